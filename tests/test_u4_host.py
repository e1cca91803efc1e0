"""The host decomposition of general two-qubit unitaries (qx_u4_decompose).

Each QX_U4 gate enters the library as 15 gates (RZ RY RZ on each wire, the
commuting RXX RYY RZZ, RZ RY RZ on each wire).  Their product, rebuilt here
from textbook matrices (tests/refs.py, independent of the library), must equal
the given unitary up to a global phase, for Haar-random matrices and for the
named gates whose Cartan coordinates are degenerate (local gates, CX, SWAP,
iSWAP, sqrt(SWAP), controlled phases), on either wire order.  Non-unitary
input is rejected.  No GPU is needed.
"""
import numpy as np
import pytest

import refs
from paper_2505_03307_gb300 import qx
from paper_2505_03307_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _phase_distance(a, b):
    tr = np.vdot(b, a)
    ph = tr / abs(tr) if abs(tr) > 0 else 1.0
    return float(np.max(np.abs(a - ph * b)))


def _check(u, q0, q1):
    gates, res = qx.u4_decompose(u, q0, q1)
    assert len(gates) == 15 and res <= 1e-10
    names = [g[0] for g in gates]
    assert names == ["RZ", "RY", "RZ"] * 2 + ["RXX", "RYY", "RZZ"] + ["RZ", "RY", "RZ"] * 2
    n = max(q0, q1) + 1
    # the same gates as a dense circuit on n qubits against U on (q0, q1)
    want = refs.dense_unitary(n, [("U4", q0, q1, u)])
    got = refs.dense_unitary(n, gates)
    assert _phase_distance(got, want) < 1e-9


@pytest.mark.parametrize("seed", range(25))
def test_haar_unitaries(seed):
    rng = np.random.default_rng(seed)
    u = W.haar_u4(rng)
    _check(u, 0, 1)
    _check(u, 1, 0)
    _check(u, 2, 0)


@pytest.mark.parametrize("name", sorted(W.special_u4()))
def test_degenerate_unitaries(name):
    u = W.special_u4()[name]
    _check(u, 0, 1)
    _check(u, 1, 0)


def test_non_unitary_is_rejected():
    with pytest.raises(qx.QxError) as e:
        qx.u4_decompose(np.eye(4) * 1.1)
    assert e.value.name == "QX_EINVAL"
    with pytest.raises(qx.QxError):
        qx.load_circuit(2, [("U4", 0, 1, np.ones((4, 4)))])


def test_circuit_with_u4_loads_its_decomposition():
    n, instrs = W.random_small_u4(3, 4, 20)
    c = qx.load_circuit(n, instrs)
    plan = qx.group_ops(c)
    k = sum(1 for g in instrs if g[0] == "U4")
    assert k > 0
    # every U4 became its 15 gates
    assert len(plan.order()) == len(instrs) - k + 15 * k
