"""Python binding of libqx (ctypes): argument marshalling only.

Every step of the propagation runs in libqx's CUDA kernels; this module
converts circuits and Pauli strings to the C structures, passes PyTorch's
current CUDA stream, and raises on any non-OK status.  There is no CPU
fallback: without the built library or a GPU the calls raise.

Pauli strings are given either as "IXYZ" letter strings (character i =
qubit i) or as (x, z) integer bit masks (bit q = qubit q).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

GATE_CODES = {
    "H": 0, "S": 1, "SDG": 2, "X": 3, "Y": 4, "Z": 5, "SX": 6, "SXDG": 7,
    "T": 8, "TDG": 9, "RX": 10, "RY": 11, "RZ": 12, "CX": 13, "CZ": 14,
    "SWAP": 15, "RXX": 16, "RYY": 17, "RZZ": 18, "CRX": 19, "CRY": 20, "CRZ": 21, "CP": 22,
    "U4": 23,
}
STATUS = {0: "QX_OK", 1: "QX_EINVAL", 2: "QX_ENOMEM", 3: "QX_EBUDGET", 4: "QX_ECAP",
          5: "QX_ECUDA", 6: "QX_ETIMEOUT", 7: "QX_EUNSUPPORTED"}

#: Every symbol that include/qx.h declares.
EXPORTED = (
    "qx_default_opts", "qx_load_circuit", "qx_group_ops", "qx_plan_info", "qx_plan_op",
    "qx_plan_lut", "qx_plan_clifford_passes", "qx_plan_clifford_apply", "qx_propagate",
    "qx_propagate_from", "qx_result_shape", "qx_result_info", "qx_result_stats",
    "qx_result_export", "qx_result_raw", "qx_coeff", "qx_coeff_batch", "qx_expval",
    "qx_free_circuit", "qx_free_plan", "qx_free_result", "qx_last_error",
    "qx_kernel_class_name", "qx_merge_qubit_static", "qx_server_default_opts", "qx_server_create",
    "qx_server_submit", "qx_server_poll", "qx_server_wait", "qx_server_stats", "qx_server_destroy",
    "qx_result_from_terms", "qx_propagate_result", "qx_plan_derivative", "qx_adjoint_dot",
    "qx_tape_forward", "qx_tape_backward", "qx_tape_info", "qx_free_tape",
    "qx_group_ops_dag", "qx_plan_order", "qx_group_ops_pushthrough", "qx_adjoint_dot_pauli",
    "qx_wait_selftest", "qx_load_circuit_u4", "qx_u4_decompose", "qx_reserve_device_memory",
)


class QxError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class Instr(ctypes.Structure):
    _fields_ = [("gate", ctypes.c_uint32), ("q0", ctypes.c_int32), ("q1", ctypes.c_int32),
                ("theta", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class PropOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("eps", ctypes.c_double),
                ("gen_begin", ctypes.c_int), ("gen_end", ctypes.c_int),
                ("hbm_budget", ctypes.c_size_t), ("max_terms", ctypes.c_size_t),
                ("stream", ctypes.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_ctx", ctypes.c_void_p), ("timeout_ms", ctypes.c_uint32),
                ("flags", ctypes.c_uint32)]

FLAG_KERNEL_TIMING = 1
FLAG_NO_INPLACE = 2
KC_COUNT = 15


_SCALARS = ("K", "Kp", "term_updates", "children", "alg_bytes", "kernel_launches", "host_syncs",
            "final_terms", "peak_terms", "fan_steps", "merge_passes", "clifford_passes",
            "inplace_steps", "inplace_fallbacks", "block_steps", "guesses_held",
            "guesses_missed")


class ServerOpts(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int), ("hbm_budget", ctypes.c_size_t),
                ("precision", ctypes.c_int), ("eps", ctypes.c_double),
                ("max_queue", ctypes.c_size_t), ("max_batch", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("alone", ctypes.c_uint64), ("queued", ctypes.c_uint64),
                ("running", ctypes.c_uint64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("batches", ctypes.c_uint64), ("mean_batch", ctypes.c_double),
                ("peak_reserved", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PropStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in _SCALARS] + [
        ("kc_launches", ctypes.c_uint64 * 16), ("kc_bytes", ctypes.c_uint64 * 16),
        ("kc_ms", ctypes.c_double * 16)]

    def as_dict(self):
        d = {k: int(getattr(self, k)) for k in _SCALARS}
        lib = load_library()
        d["kernels"] = {
            lib.qx_kernel_class_name(k).decode(): {
                "launches": int(self.kc_launches[k]), "alg_bytes": int(self.kc_bytes[k]),
                "ms": float(self.kc_ms[k])}
            for k in range(KC_COUNT)}
        return d


_lib = None
_P = ctypes.c_void_p
_U64P = ctypes.POINTER(ctypes.c_uint64)
_DP = ctypes.POINTER(ctypes.c_double)
_SZ = ctypes.c_size_t


def library_path() -> str:
    return _build.LIB


def load_library():
    """Load libqx.so (built by ``__graft_entry__.build()``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libqx is not built ({path} missing): run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    sig = {
        "qx_default_opts": (None, [ctypes.POINTER(PropOpts)]),
        "qx_load_circuit": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(Instr), _SZ,
                                           ctypes.POINTER(_P)]),
        "qx_load_circuit_u4": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(Instr), _SZ, _DP, _SZ,
                                              ctypes.POINTER(_P)]),
        "qx_u4_decompose": (ctypes.c_int, [_DP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Instr),
                                           ctypes.POINTER(_SZ), _DP]),
        "qx_group_ops": (ctypes.c_int, [_P, ctypes.POINTER(_P)]),
        "qx_group_ops_dag": (ctypes.c_int, [_P, ctypes.POINTER(_P)]),
        "qx_group_ops_pushthrough": (ctypes.c_int, [_P, ctypes.POINTER(_P)]),
        "qx_plan_order": (ctypes.c_int, [_P, ctypes.POINTER(_SZ), _P]),
        "qx_plan_info": (ctypes.c_int, [_P, ctypes.POINTER(_SZ), ctypes.POINTER(_SZ)]),
        "qx_plan_op": (ctypes.c_int, [_P, _SZ, ctypes.POINTER(ctypes.c_int)]),
        "qx_plan_lut": (ctypes.c_int, [_P, _SZ, _DP]),
        "qx_plan_clifford_passes": (ctypes.c_int, [_P, ctypes.POINTER(_SZ)]),
        "qx_plan_clifford_apply": (ctypes.c_int, [_P, _SZ, _U64P, _U64P,
                                                  ctypes.POINTER(ctypes.c_int)]),
        "qx_propagate": (ctypes.c_int, [_P, ctypes.POINTER(PropOpts), ctypes.POINTER(_P)]),
        "qx_propagate_from": (ctypes.c_int, [_P, ctypes.c_int, _U64P, _U64P, _DP,
                                             ctypes.POINTER(PropOpts), ctypes.POINTER(_P)]),
        "qx_result_shape": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_SZ)]),
        "qx_result_info": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_SZ), _DP, _DP]),
        "qx_result_stats": (ctypes.c_int, [_P, ctypes.POINTER(PropStats)]),
        "qx_result_export": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _SZ, ctypes.c_int]),
        "qx_result_raw": (ctypes.c_int, [_P, _P, _P, _P, _P, _SZ]),
        "qx_coeff": (ctypes.c_int, [_P, ctypes.c_int, _U64P, _U64P, _DP, _DP]),
        "qx_coeff_batch": (ctypes.c_int, [_P, _SZ, _P, _P, _P, _P, ctypes.c_int]),
        "qx_expval": (ctypes.c_int, [_P, _SZ, _U64P, _U64P, ctypes.POINTER(PropOpts), _DP]),
        "qx_free_circuit": (None, [_P]),
        "qx_free_plan": (None, [_P]),
        "qx_free_result": (None, [_P]),
        "qx_last_error": (ctypes.c_char_p, []),
        "qx_kernel_class_name": (ctypes.c_char_p, [ctypes.c_int]),
        "qx_server_default_opts": (None, [ctypes.POINTER(ServerOpts)]),
        "qx_server_create": (ctypes.c_int, [ctypes.POINTER(ServerOpts), ctypes.POINTER(_P)]),
        "qx_server_submit": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(Instr), _SZ,
                                            ctypes.POINTER(ctypes.c_uint64)]),
        "qx_server_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)]),
        "qx_server_wait": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(_P),
                                          ctypes.POINTER(ctypes.c_double)]),
        "qx_server_stats": (ctypes.c_int, [_P, ctypes.POINTER(ServerStats)]),
        "qx_server_destroy": (None, [_P]),
        "qx_result_from_terms": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _SZ, _P, _P, _P, _P,
                                                ctypes.c_int, ctypes.POINTER(_P)]),
        "qx_propagate_result": (ctypes.c_int, [_P, _P, ctypes.POINTER(PropOpts), ctypes.POINTER(_P)]),
        "qx_plan_derivative": (ctypes.c_int, [_P, _SZ, _DP, ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(_SZ)]),
        "qx_adjoint_dot": (ctypes.c_int, [_P, _P, _P, _SZ, _P, _P, _P]),
        "qx_adjoint_dot_pauli": (ctypes.c_int, [_P, _P, _P, _SZ, _P, _P, _P]),
        "qx_tape_forward": (ctypes.c_int, [_P, ctypes.POINTER(PropOpts), ctypes.c_int, _SZ, _P, _P,
                                           _P, _P, ctypes.POINTER(_P)]),
        "qx_tape_backward": (ctypes.c_int, [_P, _P, _P]),
        "qx_tape_info": (ctypes.c_int, [_P, ctypes.POINTER(_SZ), ctypes.POINTER(_SZ),
                                        ctypes.POINTER(_SZ), ctypes.POINTER(_SZ)]),
        "qx_free_tape": (None, [_P]),
        "qx_wait_selftest": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_int]),
        "qx_reserve_device_memory": (ctypes.c_int, [_SZ, _P]),
        "qx_merge_qubit_static": (ctypes.c_int, [ctypes.c_int, _SZ, ctypes.c_int, _P, _P, _P, _P,
                                                 ctypes.c_int, _DP, _P, _P, _P, _P, _SZ,
                                                 ctypes.POINTER(_SZ), _P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status):
    if status != 0:
        raise QxError(status, load_library().qx_last_error().decode(errors="replace"))


def words(n: int) -> int:
    return (n + 63) // 64


def pauli_to_words(p, n):
    """'IXYZ...' string or (x, z) ints -> (x words, z words) as uint64 arrays."""
    W = words(n)
    if isinstance(p, str):
        if len(p) != n:
            raise ValueError("Pauli string length must equal n")
        x = sum(1 << q for q, c in enumerate(p) if c in "XY")
        z = sum(1 << q for q, c in enumerate(p) if c in "YZ")
    else:
        x, z = int(p[0]), int(p[1])
    mask = (1 << 64) - 1
    xw = np.array([(x >> (64 * k)) & mask for k in range(W)], dtype=np.uint64)
    zw = np.array([(z >> (64 * k)) & mask for k in range(W)], dtype=np.uint64)
    return xw, zw


def words_to_pauli(xw, zw, n):
    x = sum(int(v) << (64 * k) for k, v in enumerate(xw))
    z = sum(int(v) << (64 * k) for k, v in enumerate(zw))
    return "".join("IXZY"[((x >> q) & 1) + 2 * ((z >> q) & 1)] for q in range(n))


def _stream_ptr(stream):
    if stream is not None:
        return int(stream)
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return 0


class _TorchAllocator:
    """Routes libqx device allocations to PyTorch's caching allocator."""

    def __init__(self):
        import torch
        self._torch = torch
        self.alloc = ALLOC_FN(self._alloc)
        self.free = FREE_FN(self._free)

    def _alloc(self, nbytes, ctx, stream):
        try:
            return self._torch.cuda.caching_allocator_alloc(int(nbytes), stream=stream or 0)
        except Exception:  # noqa: BLE001 - report as NULL to the library
            return None

    def _free(self, ptr, ctx, stream):
        self._torch.cuda.caching_allocator_delete(ptr)


_torch_alloc = None


def make_opts(eps=0.0, gens=None, hbm_budget=0, max_terms=0, stream=None, timeout_ms=0,
              torch_allocator=False, kernel_timing=False, precision=64, inplace=True,
              allocator=None):
    """qx_prop_opts from keyword arguments.  ``allocator``: an object with
    ``alloc`` / ``free`` ctypes callbacks (ALLOC_FN / FREE_FN) that the library
    calls for every device allocation of the call."""
    o = PropOpts()
    load_library().qx_default_opts(ctypes.byref(o))
    o.precision = int(precision)
    o.eps = float(eps)
    if gens is not None:
        o.gen_begin, o.gen_end = int(gens[0]), int(gens[1])
    o.hbm_budget = int(hbm_budget)
    o.max_terms = int(max_terms)
    o.stream = _stream_ptr(stream)
    o.timeout_ms = int(timeout_ms)
    o.flags = (FLAG_KERNEL_TIMING if kernel_timing else 0) | (0 if inplace else FLAG_NO_INPLACE)
    if torch_allocator:
        global _torch_alloc
        if _torch_alloc is None:
            _torch_alloc = _TorchAllocator()
        o.alloc = _torch_alloc.alloc
        o.free = _torch_alloc.free
    if allocator is not None:
        o.alloc = allocator.alloc
        o.free = allocator.free
    return o


#: numpy layout of qx_instr (uint32 gate, int32 q0, int32 q1, double theta).
INSTR_DTYPE = np.dtype({"names": ["gate", "q0", "q1", "theta"],
                        "formats": [np.uint32, np.int32, np.int32, np.float64],
                        "offsets": [0, 4, 8, 16], "itemsize": 24})
assert INSTR_DTYPE.itemsize == ctypes.sizeof(Instr)


def instr_records(names, q0, q1, theta):
    """qx_instr records from column arrays (gate names, wires, angles), without
    a Python loop over instructions."""
    names = np.asarray(names)
    rec = np.zeros(len(names), INSTR_DTYPE)
    uniq, inv = np.unique(names, return_inverse=True)
    rec["gate"] = np.array([GATE_CODES[str(u)] for u in uniq], np.uint32)[inv]
    rec["q0"] = q0
    rec["q1"] = q1
    rec["theta"] = theta
    return rec


def u4_array(u):
    """A 4 x 4 complex matrix as the 32 doubles of the C interface (row-major,
    real and imaginary parts interleaved)."""
    u = np.asarray(u, dtype=complex).reshape(4, 4)
    out = np.empty(32, np.float64)
    out[0::2] = u.real.reshape(-1)
    out[1::2] = u.imag.reshape(-1)
    return out


def u4_decompose(u, q0=0, q1=1):
    """qx_u4_decompose: the 15 gates (name, q0, q1, theta) that replace a
    two-qubit unitary, and the residual of their product."""
    inv = {v: k for k, v in GATE_CODES.items()}
    arr = (Instr * 16)()
    cnt, res = _SZ(), ctypes.c_double()
    a = u4_array(u)
    _check(load_library().qx_u4_decompose(a.ctypes.data_as(_DP), int(q0), int(q1), arr,
                                           ctypes.byref(cnt), ctypes.byref(res)))
    return [(inv[arr[k].gate], arr[k].q0, arr[k].q1, arr[k].theta) for k in range(cnt.value)], \
        res.value


class Circuit:
    def __init__(self, n, instrs, records=None):
        """instrs: (gate, q0, q1, theta) tuples; or records: an INSTR_DTYPE
        array (then instrs is None)."""
        lib = load_library()
        h = _P()
        if records is not None:
            rec = np.ascontiguousarray(records, INSTR_DTYPE)
            _check(lib.qx_load_circuit(int(n), ctypes.cast(rec.ctypes.data, ctypes.POINTER(Instr)),
                                       len(rec), ctypes.byref(h)))
            self.instrs = None
            self.ninstr = len(rec)
        else:
            # a U4 instruction carries its 4 x 4 matrix in place of theta: the
            # matrices go to a side array and theta becomes the index
            mats = []
            rows = []
            for g, a, b, th in instrs:
                if g == "U4":
                    rows.append((GATE_CODES[g], a, b, float(len(mats))))
                    mats.append(u4_array(th))
                else:
                    rows.append((GATE_CODES[g], a, b, th))
            rec = np.array(rows, INSTR_DTYPE).reshape(-1)
            ptr = ctypes.cast(rec.ctypes.data, ctypes.POINTER(Instr))
            if mats:
                m = np.ascontiguousarray(np.concatenate(mats), np.float64)
                _check(lib.qx_load_circuit_u4(int(n), ptr, len(rec), m.ctypes.data_as(_DP),
                                              len(mats), ctypes.byref(h)))
            else:
                _check(lib.qx_load_circuit(int(n), ptr, len(rec), ctypes.byref(h)))
            self.instrs = list(instrs)
            self.ninstr = len(instrs)
        self.n = n
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.qx_free_circuit(self._h)
            self._h = None


class Plan:
    def __init__(self, circuit: Circuit, dag=False, pushthrough=False):
        lib = load_library()
        h = _P()
        if dag and pushthrough:
            raise ValueError("choose one of dag and pushthrough")
        fn = (lib.qx_group_ops_dag if dag else
              lib.qx_group_ops_pushthrough if pushthrough else lib.qx_group_ops)
        _check(fn(circuit._h, ctypes.byref(h)))
        self._h = h
        self.n = circuit.n
        self.W = words(circuit.n)
        self.ninstr = circuit.ninstr

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.qx_free_plan(self._h)
            self._h = None

    def order(self):
        """order[k] = circuit index of the plan's k-th applied instruction."""
        m = _SZ()
        _check(load_library().qx_plan_order(self._h, ctypes.byref(m), None))
        out = np.zeros(max(int(m.value), 1), np.uint64)
        _check(load_library().qx_plan_order(self._h, ctypes.byref(m), out.ctypes.data))
        return out[:int(m.value)].astype(np.int64)

    def info(self):
        K, Kp = _SZ(), _SZ()
        _check(load_library().qx_plan_info(self._h, ctypes.byref(K), ctypes.byref(Kp)))
        return int(K.value), int(Kp.value)

    def ops(self):
        K, Kp = self.info()
        out = []
        for k in range(K + Kp):
            kind = ctypes.c_int()
            _check(load_library().qx_plan_op(self._h, k, ctypes.byref(kind)))
            out.append("U" if kind.value else "V")
        return out

    def lut(self, op):
        out = np.zeros((self.n, 3, 3), np.float64)
        _check(load_library().qx_plan_lut(self._h, op, out.ctypes.data_as(_DP)))
        return out

    def clifford_passes(self):
        c = _SZ()
        _check(load_library().qx_plan_clifford_passes(self._h, ctypes.byref(c)))
        return int(c.value)

    def clifford_apply(self, k, pauli):
        """Image (string, sign) of a Pauli string under fused Clifford pass k (host)."""
        xw, zw = pauli_to_words(pauli, self.n)
        sign = ctypes.c_int(1)
        _check(load_library().qx_plan_clifford_apply(
            self._h, k, xw.ctypes.data_as(_U64P), zw.ctypes.data_as(_U64P), ctypes.byref(sign)))
        return words_to_pauli(xw, zw, self.n), int(sign.value)


class Result:
    def __init__(self, h, n):
        self._h = h
        self.n = n
        g, w, t = ctypes.c_int(), ctypes.c_int(), _SZ()
        _check(load_library().qx_result_shape(h, ctypes.byref(g), ctypes.byref(w), ctypes.byref(t)))
        self.ngen, self.W, self.nterms = int(g.value), int(w.value), int(t.value)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.qx_free_result(self._h)
            self._h = None
            self._allocator = None

    def free(self):
        self.__del__()

    def info(self, g):
        n, s, p = _SZ(), ctypes.c_double(), ctypes.c_double()
        _check(load_library().qx_result_info(self._h, int(g), ctypes.byref(n), ctypes.byref(s),
                                              ctypes.byref(p)))
        return {"nterms": int(n.value), "sumsq": s.value, "pruned_sumsq": p.value}

    def stats(self):
        s = PropStats()
        _check(load_library().qx_result_stats(self._h, ctypes.byref(s)))
        return s.as_dict()

    def export(self, g):
        """(x words [k, W] uint64, z words, weights) of generator g in base-4 order (host)."""
        k = self.info(g)["nterms"]
        x = np.zeros((max(k, 1), self.W), np.uint64)
        z = np.zeros((max(k, 1), self.W), np.uint64)
        w = np.zeros(max(k, 1), np.float64)
        _check(load_library().qx_result_export(self._h, int(g), x.ctypes.data, z.ctypes.data,
                                                w.ctypes.data, k, 0))
        return x[:k], z[:k], w[:k]

    def export_dict(self, g):
        x, z, w = self.export(g)
        return {words_to_pauli(x[i], z[i], self.n): float(w[i]) for i in range(len(w))}

    def export_strings(self, g):
        x, z, w = self.export(g)
        return [words_to_pauli(x[i], z[i], self.n) for i in range(len(w))], w

    def export_device(self, g):
        """Generator g in base-4 order into new torch CUDA tensors (x, z, w)."""
        import torch
        k = self.info(g)["nterms"]
        x = torch.zeros((max(k, 1), self.W), dtype=torch.int64, device="cuda")
        z = torch.zeros_like(x)
        w = torch.zeros(max(k, 1), dtype=torch.float64, device="cuda")
        _check(load_library().qx_result_export(self._h, int(g), x.data_ptr(), z.data_ptr(),
                                                w.data_ptr(), k, 1))
        return x[:k], z[:k], w[:k]

    def raw_device(self):
        """All terms in device order as torch CUDA tensors (x, z, w, generator)."""
        import torch
        k = self.nterms
        x = torch.zeros((max(k, 1), self.W), dtype=torch.int64, device="cuda")
        z = torch.zeros_like(x)
        w = torch.zeros(max(k, 1), dtype=torch.float64, device="cuda")
        g = torch.zeros(max(k, 1), dtype=torch.int32, device="cuda")
        _check(load_library().qx_result_raw(self._h, x.data_ptr(), z.data_ptr(), w.data_ptr(),
                                             g.data_ptr(), k))
        return x[:k], z[:k], w[:k], g[:k]

    def raw_into(self, x, z, w, g):
        """All terms in device order into the given torch tensors (CUDA, or
        pinned CPU tensors, which the export kernel writes directly): x, z
        int64 (>= nterms, W), w float64, g int32.  Returns nterms."""
        k = self.nterms
        for t in (x, z, w, g):
            if not (t.is_cuda or t.is_pinned()) or not t.is_contiguous():
                raise ValueError("buffers must be contiguous CUDA or pinned CPU tensors")
        cap = min(x.shape[0], z.shape[0], w.shape[0], g.shape[0])
        if cap < k:
            raise ValueError("buffers are smaller than the result")
        _check(load_library().qx_result_raw(self._h, x.data_ptr(), z.data_ptr(), w.data_ptr(),
                                             g.data_ptr(), cap))
        return k

    def coeff(self, g, pauli):
        xw, zw = pauli_to_words(pauli, self.n)
        re, im = ctypes.c_double(), ctypes.c_double()
        _check(load_library().qx_coeff(self._h, int(g), xw.ctypes.data_as(_U64P),
                                        zw.ctypes.data_as(_U64P), ctypes.byref(re),
                                        ctypes.byref(im)))
        return re.value

    def coeff_batch(self, gens, paulis):
        nq = len(paulis)
        g = np.ascontiguousarray(gens, dtype=np.int32)
        x = np.zeros((max(nq, 1), self.W), np.uint64)
        z = np.zeros((max(nq, 1), self.W), np.uint64)
        for i, p in enumerate(paulis):
            x[i], z[i] = pauli_to_words(p, self.n)
        out = np.zeros(max(nq, 1), np.float64)
        _check(load_library().qx_coeff_batch(self._h, nq, g.ctypes.data, x.ctypes.data,
                                              z.ctypes.data, out.ctypes.data, 0))
        return out[:nq]


def load_circuit(n, instrs) -> Circuit:
    return Circuit(n, instrs)


def load_circuit_records(n, records) -> Circuit:
    """Circuit from an INSTR_DTYPE array (see instr_records)."""
    return Circuit(n, None, records=records)


def group_ops(circuit: Circuit, dag=False, pushthrough=False) -> Plan:
    """List-order grouping (Sec. III.A); qubit-wise dependency-graph grouping
    with dag=True (qx_group_ops_dag); Clifford push-through with
    pushthrough=True (qx_group_ops_pushthrough)."""
    return Plan(circuit, dag=dag, pushthrough=pushthrough)


def propagate(plan: Plan, **kw) -> Result:
    o = make_opts(**kw)
    h = _P()
    _check(load_library().qx_propagate(plan._h, ctypes.byref(o), ctypes.byref(h)))
    r = Result(h, plan.n)
    # the result frees its arrays through the allocator's callbacks
    r._allocator = kw.get("allocator")
    return r


def propagate_from(plan: Plan, paulis, weights=None, **kw) -> Result:
    W = plan.W
    G = len(paulis)
    x = np.zeros((max(G, 1), W), np.uint64)
    z = np.zeros((max(G, 1), W), np.uint64)
    for i, p in enumerate(paulis):
        x[i], z[i] = pauli_to_words(p, plan.n)
    wp = None
    if weights is not None:
        warr = np.ascontiguousarray(weights, np.float64)
        wp = warr.ctypes.data_as(_DP)
    o = make_opts(**kw)
    h = _P()
    _check(load_library().qx_propagate_from(plan._h, G, x.ctypes.data_as(_U64P),
                                             z.ctypes.data_as(_U64P), wp, ctypes.byref(o),
                                             ctypes.byref(h)))
    return Result(h, plan.n)


def expval(plan: Plan, paulis, **kw):
    W = plan.W
    G = len(paulis)
    x = np.zeros((max(G, 1), W), np.uint64)
    z = np.zeros((max(G, 1), W), np.uint64)
    for i, p in enumerate(paulis):
        x[i], z[i] = pauli_to_words(p, plan.n)
    out = np.zeros(max(G, 1), np.float64)
    o = make_opts(**kw)
    _check(load_library().qx_expval(plan._h, G, x.ctypes.data_as(_U64P), z.ctypes.data_as(_U64P),
                                     ctypes.byref(o), out.ctypes.data_as(_DP)))
    return out[:G]


def wait_selftest(timeout_ms=100, publish=False):
    """qx_wait_selftest: raises QxError (QX_ETIMEOUT) when the wait gave up."""
    _check(load_library().qx_wait_selftest(int(timeout_ms), 1 if publish else 0))


def reserve_device_memory(nbytes, stream=None):
    """qx_reserve_device_memory: grow the current device's default memory pool
    to hold at least ``nbytes`` (kept until exit), on ``stream`` (default:
    PyTorch's current stream).  Raises QxError (QX_ENOMEM) if it cannot."""
    _check(load_library().qx_reserve_device_memory(int(nbytes), _stream_ptr(stream) or None))


def paulis_to_arrays(paulis, n):
    """Pauli strings -> (x, z) uint64 arrays of shape [len, W] (at least one row)."""
    W = words(n)
    x = np.zeros((max(len(paulis), 1), W), np.uint64)
    z = np.zeros((max(len(paulis), 1), W), np.uint64)
    for i, p in enumerate(paulis):
        x[i], z[i] = pauli_to_words(p, n)
    return x, z


def result_from_terms(n, ngen, gens, paulis, weights, precision=64) -> Result:
    """A state of `ngen` generators holding the given terms (summed where
    repeated); see qx_result_from_terms."""
    g = np.ascontiguousarray(gens, np.int32)
    w = np.ascontiguousarray(weights, np.float64)
    if not (len(g) == len(w) == len(paulis)):
        raise ValueError("gens, paulis and weights must have the same length")
    x, z = paulis_to_arrays(paulis, n)
    h = _P()
    _check(load_library().qx_result_from_terms(int(n), int(ngen), len(paulis), x.ctypes.data,
                                                z.ctypes.data, w.ctypes.data, g.ctypes.data,
                                                int(precision), ctypes.byref(h)))
    return Result(h, n)


def propagate_result(plan: Plan, start: Result, **kw) -> Result:
    """Propagation of every term of `start` through `plan` (start is unchanged)."""
    o = make_opts(**kw)
    h = _P()
    _check(load_library().qx_propagate_result(plan._h, start._h, ctypes.byref(o), ctypes.byref(h)))
    return Result(h, plan.n)


def plan_derivative(plan: Plan, instr):
    """(D [3, 3], wire, op_end) of rotation instruction `instr` (qx_plan_derivative)."""
    d = np.zeros(9, np.float64)
    q, e = ctypes.c_int(), _SZ()
    _check(load_library().qx_plan_derivative(plan._h, int(instr), d.ctypes.data_as(_DP),
                                              ctypes.byref(q), ctypes.byref(e)))
    return d.reshape(3, 3), int(q.value), int(e.value)


def adjoint_dot(m: Result, lam: Result, lam_gen, qubits, dmats):
    """<M D_r, Lambda> for each rotation r (qx_adjoint_dot)."""
    lg = np.ascontiguousarray(lam_gen, np.int32)
    if len(lg) != m.ngen:
        raise ValueError("lam_gen needs one entry per generator of m")
    q = np.ascontiguousarray(qubits, np.int32)
    d = np.ascontiguousarray(dmats, np.float64).reshape(-1)
    if d.size != 9 * len(q):
        raise ValueError("need one 3x3 matrix per rotation")
    out = np.zeros(max(len(q), 1), np.float64)
    _check(load_library().qx_adjoint_dot(m._h, lam._h, lg.ctypes.data, len(q), q.ctypes.data,
                                          d.ctypes.data, out.ctypes.data))
    return out[:len(q)]


class Tape:
    """Forward pass with per-operator checkpoints and reverse passes
    (qx_tape_forward / qx_tape_backward).

    ``values`` holds c_{query_gens[k]}(paulis[k]) after the circuit (generator
    indices relative to the ``gens`` range of the options);
    ``backward(a)`` returns dL/dtheta_i for L = sum_k a[k] values[k] and every
    instruction i (0 where the instruction is not a rotation)."""

    def __init__(self, plan: Plan, query_gens, paulis, ckpt_stride=1, **kw):
        self.plan = plan
        self.m = plan.ninstr
        g = np.ascontiguousarray(query_gens, np.int32)
        if len(g) != len(paulis):
            raise ValueError("query_gens and paulis must have the same length")
        x, z = paulis_to_arrays(paulis, plan.n)
        self.nq = len(paulis)
        vals = np.zeros(max(self.nq, 1), np.float64)
        o = make_opts(**kw)
        self._h = None
        h = _P()
        _check(load_library().qx_tape_forward(plan._h, ctypes.byref(o), int(ckpt_stride), self.nq,
                                               g.ctypes.data, x.ctypes.data, z.ctypes.data,
                                               vals.ctypes.data, ctypes.byref(h)))
        self._h = h
        self.values = vals[:self.nq]

    def backward(self, a):
        a = np.ascontiguousarray(a, np.float64).reshape(-1)
        if a.size != self.nq:
            raise ValueError("need one cotangent per query")
        grad = np.zeros(max(self.m, 1), np.float64)
        _check(load_library().qx_tape_backward(self._h, a.ctypes.data, grad.ctypes.data))
        return grad[:self.m]

    def info(self):
        r, k, h, b = _SZ(), _SZ(), _SZ(), _SZ()
        _check(load_library().qx_tape_info(self._h, ctypes.byref(r), ctypes.byref(k),
                                            ctypes.byref(h), ctypes.byref(b)))
        return {"rotations": int(r.value), "ops": int(k.value), "held": int(h.value),
                "held_bytes": int(b.value)}

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.qx_free_tape(self._h)
            self._h = None

    def free(self):
        self.__del__()


def merge_qubit_static(n, ngen, x, z, w, gen, q, table, out_x, out_z, out_w, out_gen,
                       stream=None):
    """qx_merge_qubit_static on torch CUDA tensors (planar layout, see include/qx.h).

    x, z: int64 [W, N]; w: float64 [N]; gen: int32 [N]; outputs likewise with
    capacity out_w.numel().  Returns the number of output terms."""
    t = np.ascontiguousarray(table, np.float64).reshape(9)
    nout = _SZ()
    _check(load_library().qx_merge_qubit_static(
        int(n), int(w.numel()), int(ngen), x.data_ptr(), z.data_ptr(), w.data_ptr(),
        gen.data_ptr(), int(q), t.ctypes.data_as(_DP), out_x.data_ptr(), out_z.data_ptr(),
        out_w.data_ptr(), out_gen.data_ptr(), int(out_w.numel()), ctypes.byref(nout),
        _stream_ptr(stream)))
    return int(nout.value)


def _instr_array(instrs):
    arr = (Instr * max(1, len(instrs)))()
    for i, (g, a, b, th) in enumerate(instrs):
        arr[i] = Instr(GATE_CODES[g], int(a), int(b), float(th))
    arr.count = len(instrs)
    return arr


def instr_array(instrs):
    """C instruction array of a circuit, for Server.submit."""
    return _instr_array(instrs)


class Server:
    """Request loop with continuous batching (qx_server_*): submit circuits as
    they arrive, wait for their results; planned requests are admitted by
    the HBM ledger into batches that share one term store, `slots` batches at
    a time."""

    def __init__(self, slots=2, hbm_budget=0, precision=64, eps=0.0, max_queue=0, max_batch=0):
        lib = load_library()
        o = ServerOpts()
        lib.qx_server_default_opts(ctypes.byref(o))
        o.slots, o.hbm_budget, o.precision = int(slots), int(hbm_budget), int(precision)
        o.eps, o.max_queue = float(eps), int(max_queue)
        if max_batch:
            o.max_batch = int(max_batch)
        h = _P()
        _check(lib.qx_server_create(ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self._n = {}

    def submit(self, n, instrs):
        """Queue a circuit: a list of (gate, q0, q1, theta), or an array made
        beforehand with instr_array (no marshalling at submission time)."""
        t = ctypes.c_uint64()
        arr = instrs if isinstance(instrs, ctypes.Array) else _instr_array(instrs)
        m = getattr(instrs, "count", None) if isinstance(instrs, ctypes.Array) else len(instrs)
        _check(load_library().qx_server_submit(self._h, int(n), arr, int(m), ctypes.byref(t)))
        self._n[t.value] = n
        return int(t.value)

    def poll(self, ticket):
        d = ctypes.c_int()
        _check(load_library().qx_server_poll(self._h, ticket, ctypes.byref(d)))
        return bool(d.value)

    def wait(self, ticket):
        """(Result, latency in ms); raises QxError if the request failed."""
        h = _P()
        lat = ctypes.c_double()
        n = self._n.pop(ticket, 0)
        _check(load_library().qx_server_wait(self._h, ticket, ctypes.byref(h), ctypes.byref(lat)))
        return Result(h, n), lat.value

    def stats(self):
        st = ServerStats()
        _check(load_library().qx_server_stats(self._h, ctypes.byref(st)))
        return st.as_dict()

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.qx_server_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


def coeff(result: Result, g, pauli):
    return result.coeff(g, pauli)
