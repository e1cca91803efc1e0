"""qx_merge_qubit_static, the entry point that allocates nothing, against qx_propagate.

Some callers cannot allocate device memory: their GPU memory already belongs
to another allocator, or they run a loop where a cudaMalloc (which may
synchronise the device) is not acceptable.  For them the one-qubit expansion
with index-based accumulation keeps its scratch in a fixed array inside the
library.  This test hands it the terms of a propagated circuit and checks, on
two calls in a row (the second reuses the scratch the first left behind),
that it gives the same generators as qx_propagate of the circuit followed by
the same one-qubit gate, and the same as the oracle's plan mode within the
FP64 tolerance.  This file is collected last on purpose.
"""
import ctypes
import os

import numpy as np
import pytest

from gpu_util import compare_gen
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


def _as_dicts(n, x, z, w, g, cnt, ngen):
    """Planar torch outputs -> one {string: weight} dict per generator."""
    xs = x[:, :cnt].cpu().numpy().astype(np.uint64)
    zs = z[:, :cnt].cpu().numpy().astype(np.uint64)
    ws = w[:cnt].cpu().numpy()
    gs = g[:cnt].cpu().numpy()
    out = [dict() for _ in range(ngen)]
    for i in range(cnt):
        s = qx.words_to_pauli(xs[:, i], zs[:, i], n)
        assert s not in out[gs[i]], "duplicate string in the output"
        out[gs[i]][s] = float(ws[i])
    return out


def _base_circuit(n):
    """A circuit that ends with a two-qubit gate, so the extra gate is its own U_k."""
    if n <= 16:
        return W.hea(11, n=n, layers=2)[1]  # ends with the CX ring
    _, instrs = W.random_clifford(n, n, 6 * n)
    rng = np.random.default_rng(n)
    for q in rng.choice(n, size=8, replace=False):
        instrs.insert(int(rng.integers(0, len(instrs))), ("RY", int(q), -1, 0.4 + 0.1 * int(q)))
    # rotations on the top wires just before the last two-qubit gate: the extra
    # gate then meets strings with mixed letters there and has to merge them
    return instrs + [("RY", q, -1, 0.3) for q in range(n - 8, n)] + [("CX", 0, 1, 0.0)]


@pytest.mark.parametrize("n,q", [(10, 4), (70, 66)])
def test_static_merge_matches_propagate(n, q):
    import torch
    base = _base_circuit(n)
    extra = ("RY", q, -1, 0.9)
    plan_a = qx.group_ops(qx.load_circuit(n, base))
    res_a = qx.propagate(plan_a)
    x, z, w, g = res_a.raw_device()
    xp, zp = x.t().contiguous(), z.t().contiguous()  # planar: word k of term i at [k, i]
    plan_b = qx.group_ops(qx.load_circuit(n, base + [extra]))
    table = plan_b.lut(len(plan_b.ops()) - 1)[q]
    res_b = qx.propagate(plan_b)
    want = [res_b.export_dict(j) for j in range(n)]
    ref = O.propagate(n, base + [extra], mode="plan", threads=os.cpu_count() or 1)
    oracle_dicts = [O.as_dict(r) for r in ref]
    N = w.numel()
    cap = 3 * N
    for _ in range(2):
        ox = torch.zeros((xp.shape[0], cap), dtype=torch.int64, device="cuda")
        oz = torch.zeros_like(ox)
        ow = torch.zeros(cap, dtype=torch.float64, device="cuda")
        og = torch.zeros(cap, dtype=torch.int32, device="cuda")
        cnt = qx.merge_qubit_static(n, n, xp, zp, w, g, q, table, ox, oz, ow, og)
        assert cnt == res_b.nterms
        got = _as_dicts(n, ox, oz, ow, og, cnt, n)
        for j in range(n):
            compare_gen(got[j], want[j], f"generator {j}")
            compare_gen(got[j], oracle_dicts[j], f"generator {j} against the oracle")


def test_static_merge_rejects_sizes_beyond_its_limit():
    lib = qx.load_library()
    nout = ctypes.c_size_t(0)
    table = (ctypes.c_double * 9)(1, 0, 0, 0, 1, 0, 0, 0, 1)
    rc = lib.qx_merge_qubit_static(8, (1 << 18) + 1, 1, None, None, None, None, 0, table, None,
                                   None, None, None, 0, ctypes.byref(nout), None)
    assert qx.STATUS[rc] == "QX_EINVAL"
    assert b"static scratch limit" in lib.qx_last_error()
    rc = lib.qx_merge_qubit_static(8, 10, 5000, None, None, None, None, 0, table, None, None, None,
                                   None, 0, ctypes.byref(nout), None)
    assert qx.STATUS[rc] == "QX_EINVAL"


def test_static_merge_rejects_generator_ids_beyond_ngen():
    """An id at or above ngen is caught on the device before any merge
    kernel uses it as an index (QX_EINVAL, nothing written).  The bad id 7
    with ngen = 5 stays inside the scratch's per-generator region, so the
    access would be in bounds even without the check."""
    import torch
    n, q = 10, 3
    N = 6
    x = torch.zeros((1, N), dtype=torch.int64, device="cuda")
    z = torch.zeros((1, N), dtype=torch.int64, device="cuda")
    x[0, :] = torch.tensor([1 << q | 1 << k for k in range(N)], dtype=torch.int64)
    w = torch.full((N,), 0.5, dtype=torch.float64, device="cuda")
    g = torch.tensor([0, 1, 2, 3, 4, 7], dtype=torch.int32, device="cuda")
    table = np.array([[0.6, 0.8, 0.0], [-0.8, 0.6, 0.0], [0.0, 0.0, 1.0]])
    ox = torch.full((1, 3 * N), -1, dtype=torch.int64, device="cuda")
    oz = torch.full_like(ox, -1)
    ow = torch.full((3 * N,), 7.0, dtype=torch.float64, device="cuda")
    og = torch.full((3 * N,), -1, dtype=torch.int32, device="cuda")
    with pytest.raises(qx.QxError, match="generator id"):
        qx.merge_qubit_static(n, 5, x, z, w, g, q, table, ox, oz, ow, og)
    torch.cuda.synchronize()
    assert torch.all(ow == 7.0) and torch.all(og == -1)
    # the same call with valid ids works right after
    g[5] = 4
    cnt = qx.merge_qubit_static(n, 5, x, z, w, g, q, table, ox, oz, ow, og)
    assert cnt == 2 * N
