"""Python access to the CPU oracle (``qx_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the bench's
CPU-baseline leg use this module; the CUDA library never imports it.

``build()`` compiles the oracle with the host C++ compiler into
``oracle/_build/liboracle.so`` (recompiled when the source is newer).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qx_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

GATE_CODES = {
    "H": 0, "S": 1, "SDG": 2, "X": 3, "Y": 4, "Z": 5, "SX": 6, "SXDG": 7,
    "T": 8, "TDG": 9, "RX": 10, "RY": 11, "RZ": 12, "CX": 13, "CZ": 14,
    "SWAP": 15, "RXX": 16, "RYY": 17, "RZZ": 18, "CRX": 19, "CRY": 20, "CRZ": 21, "CP": 22,
    "U4": 23,
}

_MODES = {"gate": 0, "plan": 1, "dag": 2, "push": 3}
_c_int_p = ctypes.POINTER(ctypes.c_int)
_c_dbl_p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle if needed; return the shared-library path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC",
               "-pthread", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_run.restype = ctypes.c_void_p
            lib.oracle_run.argtypes = [ctypes.c_int, ctypes.c_long, _c_int_p, _c_int_p, _c_int_p,
                                       _c_dbl_p, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_char_p, _c_dbl_p,
                                       ctypes.c_int]
            lib.oracle_run_u4.restype = ctypes.c_void_p
            lib.oracle_run_u4.argtypes = lib.oracle_run.argtypes + [_c_dbl_p, ctypes.c_long]
            lib.oracle_run_sum.restype = ctypes.c_void_p
            lib.oracle_run_sum.argtypes = [ctypes.c_int, ctypes.c_long, _c_int_p, _c_int_p,
                                           _c_int_p, _c_dbl_p, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_long, ctypes.c_char_p, _c_dbl_p]
            lib.oracle_num_gens.argtypes = [ctypes.c_void_p]
            lib.oracle_num_terms.restype = ctypes.c_long
            lib.oracle_num_terms.argtypes = [ctypes.c_void_p, ctypes.c_int]
            lib.oracle_terms.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_char_p,
                                         _c_dbl_p, _c_dbl_p]
            lib.oracle_pruned_sumsq.restype = ctypes.c_double
            lib.oracle_pruned_sumsq.argtypes = [ctypes.c_void_p, ctypes.c_int]
            lib.oracle_free.argtypes = [ctypes.c_void_p]
            lib.oracle_gate_table.argtypes = [ctypes.c_int, ctypes.c_double, _c_dbl_p]
            lib.oracle_cx.restype = ctypes.c_int
            lib.oracle_cx.argtypes = [ctypes.c_char, ctypes.c_char, ctypes.c_char_p]
            lib.oracle_plan.restype = ctypes.c_void_p
            lib.oracle_plan.argtypes = [ctypes.c_int, ctypes.c_long, _c_int_p, _c_int_p, _c_int_p,
                                        _c_dbl_p, ctypes.c_int]
            lib.oracle_plan_num_ops.restype = ctypes.c_long
            lib.oracle_plan_num_ops.argtypes = [ctypes.c_void_p]
            lib.oracle_plan_op_kind.argtypes = [ctypes.c_void_p, ctypes.c_long]
            lib.oracle_plan_lut.argtypes = [ctypes.c_void_p, ctypes.c_long, _c_dbl_p]
            lib.oracle_plan_free.argtypes = [ctypes.c_void_p]
            lib.oracle_flatten.restype = ctypes.c_void_p
            lib.oracle_flatten.argtypes = [ctypes.c_int, ctypes.c_int, _c_dbl_p, _c_dbl_p]
            lib.oracle_expval.argtypes = [ctypes.c_int, ctypes.c_long, _c_int_p, _c_int_p,
                                          _c_int_p, _c_dbl_p, ctypes.c_char_p, _c_dbl_p]
            _lib = lib
    return _lib


def _arrays(instrs):
    """Column arrays of a circuit; a U4 instruction's matrix (4 x 4 complex, in
    place of theta) goes to a side array and theta becomes its index."""
    m = len(instrs)
    mats = []
    thetas = []
    for i in instrs:
        if i[0] == "U4":
            u = np.asarray(i[3], dtype=complex).reshape(4, 4)
            v = np.empty(32)
            v[0::2], v[1::2] = u.real.reshape(-1), u.imag.reshape(-1)
            thetas.append(float(len(mats)))
            mats.append(v)
        else:
            thetas.append(i[3])
    g = np.array([GATE_CODES[i[0]] for i in instrs], dtype=np.int32).reshape(m)
    a = np.array([i[1] for i in instrs], dtype=np.int32).reshape(m)
    b = np.array([i[2] for i in instrs], dtype=np.int32).reshape(m)
    t = np.array(thetas, dtype=np.float64).reshape(m)
    u = np.concatenate(mats) if mats else None
    return m, g, a, b, t, u


def _ip(a):
    return a.ctypes.data_as(_c_int_p)


def _dp(a):
    return a.ctypes.data_as(_c_dbl_p)


def _collect(lib, h, n):
    out = []
    try:
        for g in range(lib.oracle_num_gens(h)):
            k = lib.oracle_num_terms(h, g)
            buf = ctypes.create_string_buffer(max(1, k * n))
            re = np.empty(k, np.float64)
            im = np.empty(k, np.float64)
            lib.oracle_terms(h, g, buf, _dp(re), _dp(im))
            raw = buf.raw[: k * n].decode("ascii")
            strings = [raw[i * n:(i + 1) * n] for i in range(k)]
            out.append({"strings": strings, "re": re, "im": im,
                        "pruned_sumsq": lib.oracle_pruned_sumsq(h, g)})
    finally:
        lib.oracle_free(h)
    return out


def propagate(n, instrs, mode="plan", eps=0.0, gens=None, init=None, threads=1):
    """Propagate generators through ``instrs``.

    mode: "gate", "plan", "dag" (plan mode with qubit-wise grouping) or "push"
    (non-Clifford gates conjugated by their Clifford prefix, then all Clifford
    gates).
    gens: (begin, end) range of Z_j generators (default
    all n).  init: optional list of (string, weight) initial generators.
    Returns one dict per generator: strings (base-4 order), re, im, pruned_sumsq.
    """
    lib = _load()
    m, g, a, b, t, u = _arrays(instrs)
    gb, ge = (0, n) if gens is None else gens
    mats = (_dp(u), len(u) // 32) if u is not None else (None, 0)
    if init:
        s = "".join(p for p, _ in init).encode("ascii")
        wts = np.array([w for _, w in init], np.float64)
        h = lib.oracle_run_u4(n, m, _ip(g), _ip(a), _ip(b), _dp(t), _MODES[mode],
                              float(eps), 0, 0, len(init), s, _dp(wts), int(threads), *mats)
    else:
        h = lib.oracle_run_u4(n, m, _ip(g), _ip(a), _ip(b), _dp(t), _MODES[mode],
                              float(eps), int(gb), int(ge), 0, None, None, int(threads), *mats)
    if not h:
        raise ValueError("oracle rejected the circuit")
    return _collect(lib, h, n)


def propagate_sum(n, instrs, strings, weights, mode="gate", eps=0.0):
    """One generator starting as sum_i weights[i] strings[i]; returns its result dict."""
    lib = _load()
    m, g, a, b, t, _ = _arrays(instrs)
    s = "".join(strings).encode("ascii")
    w = np.ascontiguousarray(weights, np.float64)
    h = lib.oracle_run_sum(n, m, _ip(g), _ip(a), _ip(b), _dp(t), _MODES[mode],
                           float(eps), len(strings), s, _dp(w))
    if not h:
        raise ValueError("oracle rejected the input")
    return _collect(lib, h, n)[0]


def as_dict(gen):
    """{string: real weight} of one generator result (asserts im == 0)."""
    assert np.all(gen["im"] == 0.0)
    return dict(zip(gen["strings"], gen["re"].tolist()))


def gate_table(name, theta=0.0):
    lib = _load()
    out = np.zeros(9, np.float64)
    lib.oracle_gate_table(GATE_CODES[name], float(theta), _dp(out))
    return out.reshape(3, 3)


def cx(c, t):
    """(control, target) letters -> (pair, sign) under CX."""
    lib = _load()
    buf = ctypes.create_string_buffer(2)
    s = lib.oracle_cx(c.encode(), t.encode(), buf)
    return buf.raw.decode(), s


def plan(n, instrs, dag=False):
    """[(kind, lut)] per operator: kind 'U' with an n x 3 x 3 table, or 'V' with None.
    dag=True: qubit-wise grouping (one-qubit gates move past gates on other wires)."""
    lib = _load()
    m, g, a, b, t, _ = _arrays(instrs)
    h = lib.oracle_plan(n, m, _ip(g), _ip(a), _ip(b), _dp(t), 1 if dag else 0)
    if not h:
        raise ValueError("oracle rejected the circuit")
    out = []
    try:
        for k in range(lib.oracle_plan_num_ops(h)):
            if lib.oracle_plan_op_kind(h, k):
                lut = np.zeros((n, 3, 3), np.float64)
                lib.oracle_plan_lut(h, k, _dp(lut))
                out.append(("U", lut))
            else:
                out.append(("V", None))
    finally:
        lib.oracle_plan_free(h)
    return out


def flatten(lambdas, w4):
    """Eq. 3 on an explicit complex form: w4 has shape (parents, n, 4) over (I,X,Y,Z)."""
    lib = _load()
    w4 = np.ascontiguousarray(w4, np.float64)
    lam = np.ascontiguousarray(lambdas, np.float64)
    npar, n, _ = w4.shape
    h = lib.oracle_flatten(n, npar, _dp(lam), _dp(w4))
    return _collect(lib, h, n)[0]


def expval(n, instrs, q):
    """<0|U^dagger Q U|0> for one Pauli string q."""
    lib = _load()
    m, g, a, b, t, _ = _arrays(instrs)
    out = np.zeros(1, np.float64)
    rc = lib.oracle_expval(n, m, _ip(g), _ip(a), _ip(b), _dp(t), q.encode("ascii"), _dp(out))
    if rc:
        raise ValueError("oracle rejected the circuit")
    return float(out[0])


# ---- gradients of output weights (parameter-shift rule) ----------------------
#
# Conjugation by a rotation exp(-i theta s / 2) maps each Pauli letter to a
# combination whose coefficients are 1, cos(theta) or sin(theta) (the images of
# Sec. II.C).  Every output weight c_g(P) is therefore a + b cos(theta) +
# c sin(theta) as a function of one rotation angle, and for such a function
# f'(theta) = (f(theta + pi/2) - f(theta - pi/2)) / 2 holds exactly.  The
# oracle's gradient is that identity applied to two oracle propagations per
# rotation; the paper has no gradient, so this is parity by definition of the
# derivative.

ROTATIONS = ("RX", "RY", "RZ")
# one Pauli rotation each: the shift rule is exact for these too
PAULI_ROTATIONS_2Q = ("RXX", "RYY", "RZZ")
# two or three commuting rotations by theta/2: the weights hold frequencies
# 1/2 and 1 in theta, so the two-point shift rule does not apply to these
SPLIT_ROTATIONS_2Q = ("CRX", "CRY", "CRZ", "CP")


def rotation_positions(instrs):
    """Indices of the RX / RY / RZ instructions."""
    return [i for i, ins in enumerate(instrs) if ins[0] in ROTATIONS]


def angle_positions(instrs):
    """Indices of every instruction with an angle (one- and two-qubit rotations)."""
    names = ROTATIONS + PAULI_ROTATIONS_2Q + SPLIT_ROTATIONS_2Q
    return [i for i, ins in enumerate(instrs) if ins[0] in names]


def coeffs(n, instrs, queries, mode="plan", threads=1):
    """c_g(P) after the circuit for queries [(g, P)] (g: generator Z_g)."""
    gs = sorted({g for g, _ in queries})
    if not gs:
        return np.zeros(0)
    lo, hi = gs[0], gs[-1] + 1
    res = propagate(n, instrs, mode=mode, gens=(lo, hi), threads=threads)
    maps = {g: as_dict(res[g - lo]) for g in gs}
    return np.array([maps[g].get(p, 0.0) for g, p in queries], np.float64)


def functional(n, instrs, queries, a, mode="plan", threads=1):
    """L = sum_k a[k] c_{g_k}(P_k)."""
    return float(np.dot(np.asarray(a, np.float64), coeffs(n, instrs, queries, mode, threads)))


def grad_shift(n, instrs, queries, a, positions=None, mode="plan", threads=1, workers=1):
    """dL/dtheta_i by the parameter-shift rule for each rotation position i
    (default: every RX / RY / RZ).  workers > 1 runs the shifted propagations
    in threads (the C oracle releases the interpreter lock)."""
    if positions is None:
        positions = rotation_positions(instrs)

    def shifted(i, s):
        g, a_, b, th = instrs[i]
        if g not in ROTATIONS + PAULI_ROTATIONS_2Q:
            raise ValueError(f"instruction {i} is not a single Pauli rotation")
        ins = list(instrs)
        ins[i] = (g, a_, b, th + s * np.pi / 2)
        return functional(n, ins, queries, a, mode, threads)

    jobs = [(i, s) for i in positions for s in (1, -1)]
    if workers > 1:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(workers) as ex:
            vals = list(ex.map(lambda js: shifted(*js), jobs))
    else:
        vals = [shifted(i, s) for i, s in jobs]
    return np.array([(vals[2 * k] - vals[2 * k + 1]) / 2 for k in range(len(positions))])


def grad_fd(n, instrs, queries, a, positions, h=1e-5, mode="plan", threads=1, workers=1):
    """dL/dtheta_i by central differences of oracle propagations (any angle;
    error about h^2 times the third derivative plus rounding / h)."""
    def shifted(i, s):
        g, a_, b, th = instrs[i]
        ins = list(instrs)
        ins[i] = (g, a_, b, th + s * h)
        return functional(n, ins, queries, a, mode, threads)

    jobs = [(i, s) for i in positions for s in (1, -1)]
    if workers > 1:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(workers) as ex:
            vals = list(ex.map(lambda js: shifted(*js), jobs))
    else:
        vals = [shifted(i, s) for i, s in jobs]
    return np.array([(vals[2 * k] - vals[2 * k + 1]) / (2 * h) for k in range(len(positions))])
