"""Independent references that pin the oracle: dense matrices and a CHP row.

Neither the oracle nor the CUDA library is used here.  ``dense_*`` builds the
circuit unitary gate by gate from the textbook 2x2 / 4x4 matrices and reads a
Pauli coefficient as Tr(P M) / 2^n.  ``chp_*`` propagates one signed Pauli
through Clifford gates with the Aaronson-Gottesman bit rules ("Improved
simulation of stabilizer circuits", PRA 70, 052328, 2004).

Conventions: character i of a Pauli string is qubit i; basis index bit q is
qubit q.  Rotations are exp(-i theta sigma / 2).
"""
from __future__ import annotations

import cmath
import math

import numpy as np

I2 = np.eye(2, dtype=complex)
PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]], dtype=complex)
PZ = np.array([[1, 0], [0, -1]], dtype=complex)
PAULI = {"I": I2, "X": PX, "Y": PY, "Z": PZ}


def gate_matrix(name, theta=0.0):
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    r = 1 / math.sqrt(2)
    if name == "H":
        return np.array([[r, r], [r, -r]], dtype=complex)
    if name == "S":
        return np.diag([1, 1j])
    if name == "SDG":
        return np.diag([1, -1j])
    if name == "X":
        return PX.copy()
    if name == "Y":
        return PY.copy()
    if name == "Z":
        return PZ.copy()
    if name == "SX":
        return 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]])
    if name == "SXDG":
        return 0.5 * np.array([[1 - 1j, 1 + 1j], [1 + 1j, 1 - 1j]])
    if name == "T":
        return np.diag([1, cmath.exp(1j * math.pi / 4)])
    if name == "TDG":
        return np.diag([1, cmath.exp(-1j * math.pi / 4)])
    if name == "RX":
        return np.array([[c, -1j * s], [-1j * s, c]])
    if name == "RY":
        return np.array([[c, -s], [s, c]], dtype=complex)
    if name == "RZ":
        return np.diag([cmath.exp(-1j * theta / 2), cmath.exp(1j * theta / 2)])
    raise KeyError(name)


def conj_table(name, theta=0.0):
    """3x3 table T[p][c] = Tr(c g p g^dagger) / 2 from the 2x2 matrices."""
    g = gate_matrix(name, theta)
    out = np.zeros((3, 3))
    for a, p in enumerate("XYZ"):
        img = g @ PAULI[p] @ g.conj().T
        for b, c in enumerate("XYZ"):
            v = np.trace(PAULI[c] @ img) / 2
            assert abs(v.imag) < 1e-14
            out[a, b] = v.real
    return out


def _apply_1q(M, n, q, G):
    K = M.shape[1]
    T = M.reshape(2 ** (n - 1 - q), 2, 2 ** q, K)
    T = np.einsum("ij,ajbk->aibk", G, T)
    return T.reshape(2 ** n, K)


def gate_matrix_2q(name, theta=0.0):
    """4 x 4 matrix on (q0, q1), basis index 2 b(q0) + b(q1) (q0 is the control
    of the controlled gates)."""
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    I4 = np.eye(4, dtype=complex)
    if name == "SWAP":
        return np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=complex)
    if name in ("RXX", "RYY", "RZZ"):
        P = PAULI[name[1]]
        return c * I4 - 1j * s * np.kron(P, P)
    if name in ("CRX", "CRY", "CRZ"):
        m = np.eye(4, dtype=complex)
        m[2:, 2:] = gate_matrix("R" + name[2], theta)
        return m
    if name == "CP":
        return np.diag([1, 1, 1, cmath.exp(1j * theta)])
    raise KeyError(name)


def _apply_2q(M, n, a, b, G):
    """G (4 x 4 on qubits a, b; local index 2 b_a + b_b) applied to the rows of M."""
    idx = np.arange(2 ** n)
    base = idx[(((idx >> a) & 1) == 0) & (((idx >> b) & 1) == 0)]
    out = np.zeros_like(M)
    for lo in range(4):
        tgt = base | (((lo >> 1) & 1) << a) | ((lo & 1) << b)
        for li in range(4):
            if G[lo, li] != 0:
                src = base | (((li >> 1) & 1) << a) | ((li & 1) << b)
                out[tgt] += G[lo, li] * M[src]
    return out


def dense_unitary(n, instrs):
    """2^n x 2^n unitary of the circuit (first instruction applied first)."""
    D = 2 ** n
    U = np.eye(D, dtype=complex)
    idx = np.arange(D)
    for g, a, b, th in instrs:
        if g == "CX":
            perm = idx ^ (((idx >> a) & 1) << b)
            U = U[perm]
        elif g == "CZ":
            sign = np.where(((idx >> a) & 1) & ((idx >> b) & 1), -1.0, 1.0)
            U = U * sign[:, None]
        elif g == "U4":  # a general two-qubit unitary (its matrix in place of theta)
            U = _apply_2q(U, n, a, b, np.asarray(th, dtype=complex).reshape(4, 4))
        elif b >= 0:
            U = _apply_2q(U, n, a, b, gate_matrix_2q(g, th))
        else:
            U = _apply_1q(U, n, a, gate_matrix(g, th))
    return U


def pauli_xz(s):
    x = sum(1 << q for q, ch in enumerate(s) if ch in "XY")
    z = sum(1 << q for q, ch in enumerate(s) if ch in "YZ")
    return x, z


def coeff(M, s):
    """Tr(P M) / 2^n for the Hermitian Pauli string s."""
    n = len(s)
    x, z = pauli_xz(s)
    c = np.arange(2 ** n)
    par = np.array([bin(v).count("1") & 1 for v in (c & z)])
    sign = 1.0 - 2.0 * par
    ph = 1j ** bin(x & z).count("1")
    return ph * np.sum(sign * M[c, c ^ x]) / 2 ** n


def generator_matrix(U, n, j):
    zdiag = np.where((np.arange(2 ** n) >> j) & 1, -1.0, 1.0)
    return (U * zdiag[None, :]) @ U.conj().T


def pauli_matrix(s):
    M = np.array([[1.0 + 0j]])
    for ch in reversed(s):  # qubit n-1 is the most significant factor
        M = np.kron(M, PAULI[ch])
    return M


def dense_expval(n, instrs, q):
    psi = dense_unitary(n, instrs)[:, 0]
    return float(np.real(psi.conj() @ (pauli_matrix(q) @ psi)))


# --- CHP: one signed Pauli row ----------------------------------------------

def chp_row(n, j):
    """Z_j as (x bits, z bits, sign bit)."""
    x = [0] * n
    z = [0] * n
    z[j] = 1
    return [x, z, 0]


def _chp_h(r, q):
    x, z, _ = r
    r[2] ^= x[q] & z[q]
    x[q], z[q] = z[q], x[q]


def _chp_s(r, q):
    x, z, _ = r
    r[2] ^= x[q] & z[q]
    z[q] ^= x[q]


def _chp_cx(r, c, t):
    x, z, _ = r
    r[2] ^= x[c] & z[t] & (x[t] ^ z[c] ^ 1)
    x[t] ^= x[c]
    z[c] ^= z[t]


def chp_apply(r, g, a, b):
    if g == "H":
        _chp_h(r, a)
    elif g == "S":
        _chp_s(r, a)
    elif g == "SDG":
        for _ in range(3):
            _chp_s(r, a)
    elif g == "Z":
        _chp_s(r, a)
        _chp_s(r, a)
    elif g == "X":
        _chp_h(r, a)
        chp_apply(r, "Z", a, b)
        _chp_h(r, a)
    elif g == "Y":
        chp_apply(r, "Z", a, b)
        chp_apply(r, "X", a, b)
    elif g == "SX":
        _chp_h(r, a)
        _chp_s(r, a)
        _chp_h(r, a)
    elif g == "SXDG":
        _chp_h(r, a)
        chp_apply(r, "SDG", a, b)
        _chp_h(r, a)
    elif g == "CX":
        _chp_cx(r, a, b)
    elif g == "CZ":
        _chp_h(r, b)
        _chp_cx(r, a, b)
        _chp_h(r, b)
    else:
        raise KeyError(g)


def chp_string(r):
    x, z, s = r
    letters = "".join("IXZY"[xi + 2 * zi] for xi, zi in zip(x, z))
    return letters, -1.0 if s else 1.0
