"""Pauli rotation steps on the GPU: the two-qubit gates beyond CX / CZ and
Clifford push-through, against the oracle.

* List-order and qubit-wise plans with SWAP and RXX ... CP against the oracle's
  plan and qubit-wise modes (the oracle applies 16 x 16 tables built from the
  4 x 4 unitaries; the library applies one to three Pauli rotation steps per
  gate): exact string sets, weights within 1e-12 |w| + 1e-15.
* Push-through plans against the oracle's push-through mode (each
  non-Clifford gate conjugated by its Clifford prefix, written out gate by
  gate): exact string sets; and against list-order grouping up to strings of
  weight 0.
* FP32 against FP64, pruning, word boundaries (W = 2).
"""
import math

import numpy as np
import pytest

from gpu_util import close, compare_result, rounding_floor
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


def _nonzero(d, tol=1e-13):
    return {s: w for s, w in d.items() if abs(w) > tol}


def _semantic(res, ref_dicts, gens, floor):
    for g in gens:
        a, b = _nonzero(res.export_dict(g)), _nonzero(ref_dicts[g])
        assert a.keys() == b.keys(), g
        for s, w in b.items():
            assert close(a[s], w, floor)


@pytest.mark.parametrize("seed", range(16))
@pytest.mark.parametrize("grouping", ["plan", "dag"])
def test_two_qubit_gates_match_oracle(seed, grouping):
    n = 2 + seed % 7
    _, instrs = W.random_small_2q(seed, n, 40, angles="quarter" if seed % 4 == 0 else "uniform")
    plan = qx.group_ops(qx.load_circuit(n, instrs), dag=(grouping == "dag"))
    res = qx.propagate(plan)
    ref = O.propagate(n, instrs, mode=grouping, threads=4)
    compare_result(res, ref)


@pytest.mark.parametrize("n", [63, 64, 65, 100, 128])
def test_two_qubit_gates_word_boundaries(n):
    """A random Clifford circuit with six two-qubit rotations and a SWAP at
    random places (wires across the 64-bit word boundary)."""
    _, base = W.random_clifford(n, n, 8 * n)
    rng = np.random.default_rng(n)
    instrs = list(base)
    for k, name in enumerate(["RZZ", "CRX", "CP", "RXX", "CRY", "SWAP", "RYY"]):
        a, b = (int(v) for v in rng.choice(n, size=2, replace=False))
        if k == 0:
            a, b = min(62, n - 2), n - 1  # across the word boundary when n > 64
        pos = int(rng.integers(0, len(instrs) + 1))
        instrs.insert(pos, (name, a, b, float(rng.uniform(0, 2 * math.pi)) if name != "SWAP" else 0.0))
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    res = qx.propagate(plan, gens=(0, 24))
    ref = O.propagate(n, instrs, mode="plan", gens=(0, 24), threads=8)
    compare_result(res, ref)


def _push_cases():
    yield "small2q", W.random_small_2q(3, 6, 50)
    yield "layers", W.random_layers(2)
    yield "rotlayers", W.rotation_layers(4)
    yield "hea8", W.hea(1, n=8, layers=3)
    yield "qaoa10", W.qaoa(2, n=10, layers=2)
    yield "brickwork50", W.brickwork(1)
    yield "fanin14", W.fan_in_heavy(2, n=14, n_s=6, total=400, tail=60)
    yield "pairs100", W.random_pairs(3, n_cliff=20000, n_rz=10)


@pytest.mark.parametrize("case", [c for c, _ in _push_cases()])
def test_pushthrough_matches_oracle(case):
    n, instrs = dict(_push_cases())[case]
    gens = (0, min(n, 16))
    plan = qx.group_ops(qx.load_circuit(n, instrs), pushthrough=True)
    assert plan.info() == (0, 0)
    res = qx.propagate(plan, gens=gens)
    ref = O.propagate(n, instrs, mode="push", gens=gens, threads=8)
    compare_result(res, ref)
    lst = qx.propagate(qx.group_ops(qx.load_circuit(n, instrs)), gens=gens)
    # push-through and list order round in different orders
    _semantic(res, {g: lst.export_dict(g) for g in range(gens[1] - gens[0])},
              range(gens[1] - gens[0]), rounding_floor(instrs))


def test_pushthrough_fp32_and_pruning():
    n, instrs = W.fan_in_heavy(3, n=20, n_s=10, total=700, tail=100)
    plan = qx.group_ops(qx.load_circuit(n, instrs), pushthrough=True)
    a = qx.propagate(plan)
    b = qx.propagate(plan, precision=32)
    for g in range(n):
        da, db = a.export_dict(g), b.export_dict(g)
        assert da.keys() == db.keys()
        for s, w in da.items():
            assert abs(db[s] - w) <= 1e-5 * abs(w) + 1e-7
    eps = 2e-3
    p = qx.propagate(plan, eps=eps)
    ref = O.propagate(n, instrs, mode="push", eps=eps, threads=8)
    for g in range(n):
        got, want = p.export_dict(g), O.as_dict(ref[g])
        # strings within rounding of eps may fall either way
        near = {s for s, w in {**got, **want}.items() if abs(abs(w) - eps) <= 1e-12 * eps}
        assert set(got) - near == set(want) - near
        for s in set(want) - near:
            assert close(got[s], want[s])


def test_rotation_step_counts_and_no_fanout_at_clifford_angles():
    """RZZ(pi/2) is Clifford: its rotation step maps every anticommuting
    string to its partner alone (sin = 1, cos = 0), creating nothing."""
    n = 4
    instrs = [("H", 0, -1, 0.0), ("RZZ", 0, 1, math.pi / 2), ("RXX", 2, 3, math.pi)]
    res = qx.propagate(qx.group_ops(qx.load_circuit(n, instrs)))
    ref = O.propagate(n, instrs, mode="plan")
    compare_result(res, ref)
    assert all(res.info(g)["nterms"] == 1 for g in range(n))
    st = res.stats()
    assert st["kernels"]["pauli_rot"]["launches"] > 0
