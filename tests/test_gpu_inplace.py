"""In-place merge steps against the general merge and the oracle.

A fan-out step whose merge groups all hold every letter their tables produce
(the RZ layer after the T layer on the same wires) runs in place through a
full-key index.  Its results must equal the general merge (QX_FLAG_NO_INPLACE)
bit for bit: the same string sets and the same FP64 weights, because both
compute each weight with the same fixed-order group sum.  Steps with open
groups must fall back (or be skipped by the host pre-check) with unchanged
results.
"""
import numpy as np
import pytest

from gpu_util import compare_result
from oracle import oracle as O
from paper_2505_03307_gb300 import qx
from paper_2505_03307_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")


def _raw_sorted(res):
    x, z, w, g = (t.cpu().numpy() for t in res.raw_device())
    order = np.lexsort((z[:, 0], x[:, 0], g))
    return g[order], x[order, 0], z[order, 0], w[order]


def _same(a, b):
    ga, xa, za, wa = _raw_sorted(a)
    gb, xb, zb, wb = _raw_sorted(b)
    assert np.array_equal(ga, gb) and np.array_equal(xa, xb) and np.array_equal(za, zb)
    assert np.array_equal(wa, wb)


@pytest.mark.parametrize("precision", [64, 32])
def test_bench_workload_in_place_equals_general(precision):
    n, instrs = W.fan_in_heavy(1)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    a = qx.propagate(plan, precision=precision)
    b = qx.propagate(plan, precision=precision, inplace=False)
    sa, sb = a.stats(), b.stats()
    assert sa["inplace_steps"] == 1 and sa["inplace_fallbacks"] == 0
    assert sa["block_steps"] == 1
    assert sb["inplace_steps"] == 0
    assert sa["merge_passes"] == sb["merge_passes"] == 16
    assert a.nterms == b.nterms == 2228256
    if precision == 64:
        _same(a, b)
    else:
        _, _, _, wa = _raw_sorted(a)
        _, _, _, wb = _raw_sorted(b)
        assert np.max(np.abs(wa - wb)) <= 1e-6


def test_reduced_bench_workload_in_place_against_oracle():
    n, instrs = W.fan_in_heavy(2, n=14, n_s=6, total=400, tail=60)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    res = qx.propagate(plan)
    assert res.stats()["inplace_steps"] >= 1
    compare_result(res, O.propagate(n, instrs, mode="plan", threads=8))


def test_in_place_with_pruning_equals_general():
    n, instrs = W.fan_in_heavy(3, n=20, n_s=10, total=700, tail=100)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    a = qx.propagate(plan, eps=2e-3)
    b = qx.propagate(plan, eps=2e-3, inplace=False)
    assert a.stats()["inplace_steps"] >= 1
    _same(a, b)
    pruned = [a.info(g)["pruned_sumsq"] for g in range(n)]
    assert sum(pruned) > 0  # pruning removed strings
    for g in range(n):  # an atomic sum in either path: equal up to its order
        assert abs(pruned[g] - b.info(g)["pruned_sumsq"]) <= 1e-12 * pruned[g]


@pytest.mark.parametrize("case", ["hea", "layers", "xyz"])
def test_open_groups_fall_back_with_equal_results(case):
    if case == "hea":
        n, instrs = W.hea(2, n=10, layers=3)
    elif case == "layers":
        n, instrs = W.rotation_layers(3, n_rot=14)
    else:
        n, instrs = W.xyz_chain(1, n=8, layers=3, repeats=3)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    a = qx.propagate(plan)
    b = qx.propagate(plan, inplace=False)
    _same(a, b)
    st = a.stats()
    assert st["inplace_steps"] + st["inplace_fallbacks"] <= st["fan_steps"]


@pytest.mark.parametrize("seed", [1, 2])
def test_radix_three_blocks_equal_general(seed):
    """Every generator gets all three letters on the wires 0..4 (a full
    rotation after a CX chain spreads X), then, after a CZ on wires 5 and 6
    only, a second rotation on wires 0..4 whose table has a full X and Y row:
    closed groups of three, so the blocks have radix 3 on every merge wire."""
    n = 7
    rng = np.random.default_rng(seed)
    ins = [("H", q, -1, 0.0) for q in range(n)]
    ins += [("CX", q, q + 1, 0.0) for q in range(4)]
    wires = list(range(5))
    for q in wires:  # X -> all three letters
        ins += [("RZ", q, -1, float(rng.uniform(0.2, 1.3))), ("RY", q, -1, float(rng.uniform(0.2, 1.3)))]
    ins.append(("CZ", 5, 6, 0.0))  # ends the operator without touching a merge wire
    for q in wires:
        ins += [("RZ", q, -1, float(rng.uniform(0.2, 1.3))), ("RX", q, -1, float(rng.uniform(0.2, 1.3)))]
    plan = qx.group_ops(qx.load_circuit(n, ins))
    a = qx.propagate(plan)
    b = qx.propagate(plan, inplace=False)
    _same(a, b)
    compare_result(a, O.propagate(n, ins, mode="plan"))
    st = a.stats()
    assert st["block_steps"] == 1 and st["inplace_fallbacks"] == 0
