"""General two-qubit unitaries (QX_U4) on the GPU against the oracle.

The library replaces each U4 by 15 gates (KAK: RZ RY RZ on each wire, the
commuting RXX RYY RZZ, RZ RY RZ on each wire) and runs them with its usual
steps; the oracle applies the unitary's own 16 x 16 transfer table
Tr((C0 x C1) U (P0 x P1) U^dagger) / 4 (pinned to dense matrices on the CPU).
The two reach the same operator along different roundings, so strings of
weight exactly 0 on one side may be absent on the other: both sides drop
|w| <= 1e-13, then the string sets must be equal and the weights agree within
1e-12 |w| plus the circuit's rounding floor (each U4 counts as 15 rounding
steps).  Haar-random matrices and named ones with degenerate Cartan
coordinates, list-order, qubit-wise and push-through plans, one- and
two-word strings.
"""
import os

import numpy as np
import pytest

from gpu_util import close, rounding_floor
from oracle import oracle as O
from paper_2505_03307_gb300 import qx
from paper_2505_03307_gb300 import workloads as W

pytestmark = pytest.mark.gpu
CORES = os.cpu_count() or 1


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")


def _semantic(res, ref, gens, floor):
    for k, g in enumerate(gens):
        a = {s: w for s, w in res.export_dict(g).items() if abs(w) > 1e-13}
        b = {s: w for s, w in O.as_dict(ref[k]).items() if abs(w) > 1e-13}
        assert a.keys() == b.keys(), (g, sorted(set(a) ^ set(b))[:4])
        for s, w in b.items():
            assert close(a[s], w, floor), (g, s, a[s], w)


def _residuals(instrs):
    return max((qx.u4_decompose(g[3], g[1], g[2])[1] for g in instrs if g[0] == "U4"),
               default=0.0)


@pytest.mark.parametrize("seed", range(16))
@pytest.mark.parametrize("grouping", ["list", "dag", "push"])
def test_random_u4_circuits_match_oracle(seed, grouping):
    n = 2 + seed % 7
    _, instrs = W.random_small_u4(seed, n, 10 + 4 * n)
    assert _residuals(instrs) < 1e-13
    plan = qx.group_ops(qx.load_circuit(n, instrs), dag=grouping == "dag",
                        pushthrough=grouping == "push")
    res = qx.propagate(plan)
    ref = O.propagate(n, instrs, mode="plan", threads=CORES)
    _semantic(res, ref, range(n), rounding_floor(instrs))


@pytest.mark.parametrize("n", [20, 64, 70, 100])
def test_u4_on_wide_registers(n):
    """A Clifford circuit with Haar U4 gates across the word boundary."""
    rng = np.random.default_rng(n)
    _, base = W.random_clifford(n, n, 6 * n)
    instrs = list(base)
    for k in range(5):
        a, b = (int(v) for v in rng.choice(n, size=2, replace=False))
        if k == 0:
            a, b = min(62, n - 2), n - 1
        instrs.insert(int(rng.integers(0, len(instrs) + 1)), ("U4", a, b, W.haar_u4(rng)))
    gens = (0, min(n, 24))
    res = qx.propagate(qx.group_ops(qx.load_circuit(n, instrs)), gens=gens)
    ref = O.propagate(n, instrs, mode="plan", gens=gens, threads=CORES)
    _semantic(res, ref, range(gens[1]), rounding_floor(instrs))


def test_u4_fp32_and_pruning():
    n, instrs = W.random_small_u4(99, 6, 40)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    ref = O.propagate(n, instrs, mode="plan", threads=CORES)
    r32 = qx.propagate(plan, precision=32)
    for g in range(n):
        got = r32.export_dict(g)
        for s, w in O.as_dict(ref[g]).items():
            if abs(w) > 1e-6:
                assert abs(got.get(s, 0.0) - w) <= 1e-5 * abs(w) + 1e-7
    eps = 1e-3
    pr = qx.propagate(plan, eps=eps)
    for g in range(n):
        info = pr.info(g)
        assert abs(info["sumsq"] + info["pruned_sumsq"] - 1.0) < 1e-11
        assert all(abs(w) >= eps for w in pr.export_dict(g).values())
