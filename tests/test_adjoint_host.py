"""Host-side parts of the gradient path (no GPU needed).

qx_plan_derivative returns D = T^T dT/dtheta for the wire of a rotation in
its operator U_k.  It is checked against central finite differences of the
composed tables that qx_plan_lut returns (Algorithm 1), against the closed
form for a lone rotation, and for its structure: T^T T = I implies that D is
antisymmetric.  The calls that need a device fail loudly here.
"""
import math

import numpy as np
import pytest

from paper_2505_03307_gb300 import qx
from paper_2505_03307_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _op_of(plan, instrs, i):
    """Index of the chain operator holding instruction i."""
    ops = plan.ops()
    k = -1
    prev_two = None
    for j in range(i + 1):
        two = instrs[j][0] in ("CX", "CZ")
        if two != prev_two:
            k += 1
            prev_two = two
    assert ops[k] == "U"
    return k


def _lut(n, instrs, k):
    return qx.group_ops(qx.load_circuit(n, instrs)).lut(k)


@pytest.mark.parametrize("seed", [1, 2])
def test_derivative_matches_finite_differences(seed):
    n, ins = W.rotation_layers(seed)
    plan = qx.group_ops(qx.load_circuit(n, ins))
    h = 1e-6
    for i, (g, q0, q1, th) in enumerate(ins):
        if g not in ("RX", "RY", "RZ"):
            continue
        D, q, end = qx.plan_derivative(plan, i)
        assert q == q0
        assert end > i and (end == len(ins) or ins[end][0] in ("CX", "CZ"))
        assert all(ins[j][0] not in ("CX", "CZ") for j in range(i, end))
        k = _op_of(plan, ins, i)
        T = plan.lut(k)[q]
        plus, minus = list(ins), list(ins)
        plus[i] = (g, q0, q1, th + h)
        minus[i] = (g, q0, q1, th - h)
        dT = (_lut(n, plus, k)[q] - _lut(n, minus, k)[q]) / (2 * h)
        assert np.allclose(D, T.T @ dT, atol=1e-8), (i, D, T.T @ dT)
        assert np.allclose(D, -D.T, atol=1e-12)


@pytest.mark.parametrize("gate,axis", [("RX", 0), ("RY", 1), ("RZ", 2)])
def test_lone_rotation_closed_form(gate, axis):
    """For T = R_a(t) alone, T^T dT/dt is the generator: the axis row and
    column are zero, and the two other letters b -> d (+1) and d -> b (-1),
    with (b, d) the letters after a in cyclic (X, Y, Z) order."""
    plan = qx.group_ops(qx.load_circuit(1, [(gate, 0, -1, 0.77)]))
    D, q, end = qx.plan_derivative(plan, 0)
    b, d = (axis + 1) % 3, (axis + 2) % 3
    want = np.zeros((3, 3))
    want[b, d] = 1.0
    want[d, b] = -1.0
    assert q == 0 and end == 1
    assert np.allclose(D, want, atol=1e-15)


def test_derivative_rejects_non_rotations():
    plan = qx.group_ops(qx.load_circuit(2, [("H", 0, -1, 0.0), ("RZ", 1, -1, 0.3)]))
    with pytest.raises(qx.QxError) as e:
        qx.plan_derivative(plan, 0)
    assert e.value.name == "QX_EINVAL"
    with pytest.raises(qx.QxError):
        qx.plan_derivative(plan, 5)


def test_gradient_calls_fail_loudly_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    plan = qx.group_ops(qx.load_circuit(2, [("RY", 0, -1, 0.3), ("CX", 0, 1, 0.0)]))
    with pytest.raises(qx.QxError) as e:
        qx.Tape(plan, [0], ["ZI"])
    assert e.value.name == "QX_EUNSUPPORTED"
    with pytest.raises(qx.QxError) as e:
        qx.result_from_terms(2, 1, [0], ["XZ"], [1.0])
    assert e.value.name == "QX_EUNSUPPORTED"


def test_from_terms_validates_before_the_device():
    with pytest.raises(qx.QxError) as e:
        qx.result_from_terms(2, 1, [1], ["XZ"], [1.0])  # generator 1 of 1
    assert e.value.name == "QX_EINVAL"
    with pytest.raises(ValueError):
        qx.result_from_terms(2, 1, [0, 0], ["XZ"], [1.0])
    with pytest.raises(qx.QxError) as e:
        qx.result_from_terms(2, 1, [0], ["XZ"], [1.0], precision=16)
    assert e.value.name == "QX_EINVAL"
    plan = qx.group_ops(qx.load_circuit(2, [("RY", 0, -1, 0.3)]))
    with pytest.raises(qx.QxError) as e:
        qx.Tape(plan, [2], ["ZI"])  # query generator out of range
    assert e.value.name == "QX_EINVAL"
    assert math.isfinite(qx.plan_derivative(plan, 0)[0].sum())
