"""Pins of the oracle's gradient (parameter-shift rule on oracle propagations).

The gradient of L = sum_k a_k c_{g_k}(P_k) with respect to a rotation angle is
checked against facts that do not come from the oracle:
  * closed forms of one and two rotations on one qubit, derived by hand from
    exp(-i t s / 2) P exp(i t s / 2) (Sec. II.C images);
  * central finite differences of the dense 2^n x 2^n unitaries of tests/refs.py
    (n = 3 random circuits and the n = 8 rotation-layer workload);
  * the norm invariant: sum_P c_g(P)^2 = 1 for every angle (conjugation is
    orthogonal), so the gradient of that sum vanishes.
"""
import math

import numpy as np
import pytest

import refs
from oracle import oracle as O
from paper_2505_03307_gb300 import workloads as W


def _dense_functional(n, instrs, queries, a):
    U = refs.dense_unitary(n, instrs)
    mats = {}
    total = 0.0
    for (g, p), ak in zip(queries, a):
        if g not in mats:
            mats[g] = refs.generator_matrix(U, n, g)
        c = refs.coeff(mats[g], p)
        assert abs(c.imag) < 1e-12
        total += ak * c.real
    return total


def _dense_fd(n, instrs, queries, a, positions, h=1e-6):
    out = []
    for i in positions:
        g, q0, q1, th = instrs[i]
        plus = list(instrs)
        minus = list(instrs)
        plus[i] = (g, q0, q1, th + h)
        minus[i] = (g, q0, q1, th - h)
        out.append((_dense_functional(n, plus, queries, a) -
                     _dense_functional(n, minus, queries, a)) / (2 * h))
    return np.array(out)


@pytest.mark.parametrize("theta", [0.0, 0.37, 1.9, -2.6])
def test_single_rotation_closed_forms(theta):
    s, c = math.sin(theta), math.cos(theta)
    # RY on Z: Z -> cos t Z + sin t X
    ins = [("RY", 0, -1, theta)]
    assert np.allclose(O.grad_shift(1, ins, [(0, "Z")], [1.0]), [-s], atol=1e-14)
    assert np.allclose(O.grad_shift(1, ins, [(0, "X")], [1.0]), [c], atol=1e-14)
    # RX on Z: Z -> cos t Z - sin t Y
    ins = [("RX", 0, -1, theta)]
    assert np.allclose(O.grad_shift(1, ins, [(0, "Y")], [1.0]), [-c], atol=1e-14)
    # H then RZ: Z -> X -> cos t X + sin t Y
    ins = [("H", 0, -1, 0.0), ("RZ", 0, -1, theta)]
    g = O.grad_shift(1, ins, [(0, "X"), (0, "Y")], [2.0, -0.5])
    assert np.allclose(g, [2.0 * -s - 0.5 * c], atol=1e-14)


def test_two_rotation_chain_closed_form():
    """RX(al) then RY(be) on Z: cos al cos be Z + cos al sin be X - sin al Y."""
    al, be = 0.81, -1.3
    ins = [("RX", 0, -1, al), ("RY", 0, -1, be)]
    ca, sa, cb, sb = math.cos(al), math.sin(al), math.cos(be), math.sin(be)
    assert np.allclose(O.coeffs(1, ins, [(0, "Z"), (0, "X"), (0, "Y")]),
                       [ca * cb, ca * sb, -sa], atol=1e-15)
    for p, dal, dbe in [("Z", -sa * cb, -ca * sb), ("X", -sa * sb, ca * cb), ("Y", -ca, 0.0)]:
        assert np.allclose(O.grad_shift(1, ins, [(0, p)], [1.0]), [dal, dbe], atol=1e-14)


def _random_rot_circuit(seed, n, m):
    rng = np.random.default_rng(seed)
    ins = []
    for _ in range(m):
        k = int(rng.integers(0, 6))
        q = int(rng.integers(0, n))
        if k < 3:
            ins.append((("RX", "RY", "RZ")[k], q, -1, float(rng.uniform(0, 2 * math.pi))))
        elif k == 3:
            t = int((q + 1 + rng.integers(0, n - 1)) % n)
            ins.append(("CX", q, t, 0.0))
        else:
            ins.append((("H", "S")[k - 4], q, -1, 0.0))
    return ins


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_grad_matches_dense_finite_differences(seed):
    n = 3
    ins = _random_rot_circuit(seed, n, 14)
    rng = np.random.default_rng(100 + seed)
    strings = ["".join(p) for p in np.array(list("IXYZ"))[rng.integers(0, 4, size=(12, n))]]
    queries = [(int(rng.integers(0, n)), s) for s in strings]
    a = rng.normal(size=len(queries))
    pos = O.rotation_positions(ins)
    assert len(pos) >= 3
    for mode in ("gate", "plan"):
        g = O.grad_shift(n, ins, queries, a, mode=mode)
        fd = _dense_fd(n, ins, queries, a, pos)
        assert np.allclose(g, fd, atol=1e-8), (mode, g, fd)


def test_grad_rotation_layers_n8_matches_dense():
    n, ins = W.rotation_layers(2)
    ref = [O.as_dict(r) for r in O.propagate(n, ins, mode="plan", gens=(0, 3))]
    rng = np.random.default_rng(9)
    queries = []
    for g in range(3):
        keys = sorted(ref[g])
        for k in rng.choice(len(keys), size=min(6, len(keys)), replace=False):
            queries.append((g, keys[int(k)]))
    a = rng.normal(size=len(queries))
    pos = O.rotation_positions(ins)
    g = O.grad_shift(n, ins, queries, a, workers=4)
    fd = _dense_fd(n, ins, queries, a, pos)
    assert np.allclose(g, fd, atol=1e-8)
    assert np.max(np.abs(g)) > 1e-3  # not vacuous


def test_norm_gradient_vanishes():
    """sum_P c(P)^2 = 1 at every angle; with a = c(theta) over the support,
    dL/dtheta = 0.5 d(sum c^2)/dtheta = 0."""
    n = 3
    ins = _random_rot_circuit(5, n, 12)
    for g0 in range(n):
        d = O.as_dict(O.propagate(n, ins, mode="plan", gens=(g0, g0 + 1))[0])
        # support at generic angles: every string reachable from the shifted circuits too
        support = set(d)
        for i in O.rotation_positions(ins):
            for s in (1, -1):
                sh = list(ins)
                gname, q0, q1, th = sh[i]
                sh[i] = (gname, q0, q1, th + s * math.pi / 2)
                support |= set(O.as_dict(O.propagate(n, sh, mode="plan", gens=(g0, g0 + 1))[0]))
        queries = [(g0, p) for p in sorted(support)]
        a = [d.get(p, 0.0) for _, p in queries]
        assert abs(sum(v * v for v in a) - 1.0) < 1e-12
        g = O.grad_shift(n, ins, queries, a)
        assert np.max(np.abs(g)) < 1e-12


def test_shift_sign_mutation_is_caught():
    """A flipped shift direction (a plausible slip) fails the closed form."""
    ins = [("RY", 0, -1, 0.37)]
    good = O.grad_shift(1, ins, [(0, "Z")], [1.0])
    plus = O.functional(1, [("RY", 0, -1, 0.37 + math.pi / 2)], [(0, "Z")], [1.0])
    minus = O.functional(1, [("RY", 0, -1, 0.37 - math.pi / 2)], [(0, "Z")], [1.0])
    flipped = (minus - plus) / 2
    assert abs(good[0] + math.sin(0.37)) < 1e-14
    assert abs(flipped + math.sin(0.37)) > 0.5


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_two_qubit_gradients_match_dense_finite_differences(seed):
    """RXX / RYY / RZZ by the shift rule (one Pauli rotation each), the
    controlled rotations and CP by central differences of the oracle, both
    against central differences of the dense unitaries."""
    n = 3
    _, ins = W.random_small_2q(seed, n, 16, p2=0.5)
    rng = np.random.default_rng(200 + seed)
    strings = ["".join(p) for p in np.array(list("IXYZ"))[rng.integers(0, 4, size=(12, n))]]
    queries = [(int(rng.integers(0, n)), s) for s in strings]
    a = rng.normal(size=len(queries))
    single = [i for i, g in enumerate(ins) if g[0] in O.ROTATIONS + O.PAULI_ROTATIONS_2Q]
    split = [i for i, g in enumerate(ins) if g[0] in O.SPLIT_ROTATIONS_2Q]
    assert single
    assert np.allclose(O.grad_shift(n, ins, queries, a, positions=single),
                       _dense_fd(n, ins, queries, a, single), atol=1e-8)
    if split:
        assert np.allclose(O.grad_fd(n, ins, queries, a, split),
                           _dense_fd(n, ins, queries, a, split), atol=1e-7)
