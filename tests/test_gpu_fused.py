"""The fused expansion of small fan-out steps against the oracle.

A fan-out step with at most 8 wires and at most 16 children per parent whose
wires need no merge runs as one pass over its parents: count per tile, scan,
and an emission that also applies the Clifford pass before the step when
that pass acts on other qubits (and, for the last step, the program's last
pass).  These cases put each form of that pass (none, gate list, chunk
tables of 4 and 3 qubits), the absorbed last pass, a last pass on the step's
own wire (not absorbed), steps that turn out to need a merge, FP32, pruning
and generator ranges through it, against the oracle's plan mode: exact string
sets, weights within 1e-12 |w| + 1e-15 (FP32: 1e-5 |w| + 1e-7).
"""
import math
import os

import numpy as np
import pytest

from gpu_util import compare_gen, compare_result
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


def _check(n, instrs, **kw):
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    res = qx.propagate(plan, **kw)
    gens = kw.get("gens")
    ref = O.propagate(n, instrs, mode="plan", threads=CORES, eps=kw.get("eps", 0.0), gens=gens)
    compare_result(res, ref, offset=0)
    return plan, res


@pytest.mark.parametrize("n,n_s,total", [(40, 10, 4000), (100, 8, 12000), (70, 6, 3000)])
def test_deep_chain_of_single_wire_steps(n, n_s, total):
    """Rotation steps on one wire each between long Clifford blocks on the
    other qubits (chunk-table passes fused into the expansion once there are
    64 terms per generator, on their own before; the last pass absorbed into
    the last step)."""
    _, instrs = W.fan_in_deep(3, n=n, n_s=n_s, total=total)
    plan, res = _check(n, instrs)
    st = res.stats()
    assert st["kernels"]["expand_emit"]["launches"] == n_s
    # n_s + 1 Clifford blocks (the first one after the H/CX prefix joins
    # it): before step k there are at least (n - n_s) 2^k terms, so the
    # passes of the steps where that reaches 64 per generator run inside
    # the expansions
    small = sum(1 for k in range(n_s) if (n - n_s) * 2 ** k < 64 * n)
    assert st["kernels"]["clifford_pass"]["launches"] <= 1 + small
    again = qx.propagate(plan)  # on the plan's records
    compare_result(again, O.propagate(n, instrs, mode="plan", threads=CORES))
    # the last expansion counted its children per generator (no statistics
    # pass over the final terms): counts and norms equal the exported terms'
    for r in (res, again, qx.propagate(plan), qx.propagate(plan, precision=32)):
        assert r.stats()["kernels"]["gen_stats"]["launches"] == 0
        for g in range(n):
            info = r.info(g)
            w = np.array(list(r.export_dict(g).values()))
            assert info["nterms"] == len(w)
            assert abs(info["sumsq"] - float(np.sum(w * w))) <= 1e-12 * max(1.0, info["sumsq"])


def _short_pass_circuit(seed, n, rounds, tail_on_wire):
    """Few Clifford gates between rotations (gate-list passes), rotations on
    two wires per operator at times; the last pass optionally acts on the
    last step's wire (it cannot be absorbed then)."""
    rng = np.random.default_rng(seed)
    instrs = [("H", q, -1, 0.0) for q in range(n)]
    last_q = None
    for r in range(rounds):
        a, b = (int(v) for v in rng.choice(n, size=2, replace=False))
        instrs.append(("CX", a, b, 0.0))
        instrs.append(("S", int(rng.integers(0, n)), -1, 0.0))
        qs = rng.choice(n, size=1 + int(rng.integers(0, 2)), replace=False)
        for q in qs:
            instrs.append(("RZ" if rng.integers(0, 2) else "T", int(q), -1,
                           float(rng.uniform(0, 2 * math.pi))))
            last_q = int(q)
    other = (last_q + 1) % n
    instrs.append(("CX", last_q if tail_on_wire else other, (other + 1) % n if not tail_on_wire
                   else other, 0.0))
    instrs.append(("H", other, -1, 0.0))
    return instrs


@pytest.mark.parametrize("tail_on_wire", [False, True])
@pytest.mark.parametrize("n", [12, 64, 90])
def test_gate_list_passes_and_last_pass(n, tail_on_wire):
    instrs = _short_pass_circuit(n + int(tail_on_wire), n, 9, tail_on_wire)
    _check(n, instrs)


def test_steps_that_need_a_merge_leave_the_fused_path():
    """RZ on a wire whose letters differ within a generator: the masks show a
    merge, the pending pass runs first and the merge path takes the step."""
    n = 10
    instrs = [("H", q, -1, 0.0) for q in range(n)]
    # generator 0 holds X and Y on wire 0 before the last rotation there; the
    # pass before that rotation (CX(2,3), H(5)) acts on other wires
    instrs += [("RZ", 0, -1, 0.3), ("CX", 0, 1, 0.0), ("RZ", 1, -1, 0.9), ("CX", 2, 3, 0.0),
               ("H", 5, -1, 0.0), ("RZ", 0, -1, 1.1), ("CX", 7, 8, 0.0), ("S", 9, -1, 0.0)]
    _, res = _check(n, instrs)
    assert res.stats()["merge_passes"] + res.stats()["inplace_steps"] >= 1


@pytest.mark.parametrize("seed", range(4))
def test_fp32_and_pruning(seed):
    n, instrs = W.fan_in_deep(seed + 5, n=30, n_s=9, total=2500)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    r32 = qx.propagate(plan, precision=32)
    ref = O.propagate(n, instrs, mode="plan", threads=CORES)
    for g in range(n):
        got, want = r32.export_dict(g), O.as_dict(ref[g])
        assert got.keys() == want.keys()
        for s, w in want.items():
            assert abs(got[s] - w) <= 1e-5 * abs(w) + 1e-7
    eps = 1e-3
    pr = qx.propagate(plan, eps=eps)
    ref = O.propagate(n, instrs, mode="plan", threads=CORES, eps=eps)
    for g in range(n):
        got, want = pr.export_dict(g), O.as_dict(ref[g])
        near = {s for s, w in {**got, **want}.items() if abs(abs(w) - eps) <= 1e-12 * eps}
        assert set(got) - near == set(want) - near
        compare_gen({s: got[s] for s in set(want) - near}, {s: want[s] for s in set(want) - near},
                    f"gen {g}")


def test_generator_ranges_on_one_plan():
    n, instrs = W.fan_in_deep(9, n=50, n_s=10, total=5000)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    for gens in [(0, 50), (10, 30), (0, 5), (0, 50), (0, 50), (0, 50), (30, 50)]:
        res = qx.propagate(plan, gens=gens)
        ref = O.propagate(n, instrs, mode="plan", threads=CORES, gens=gens)
        compare_result(res, ref)


class _OffsetAllocator:
    """A caller allocator whose blocks start 8 bytes past a 256-byte boundary
    (PyTorch's caching allocator underneath), as any allocator that promises
    only the size may."""

    def __init__(self):
        import torch
        self.torch = torch
        self.base = {}
        self.handed = []
        self.alloc = qx.ALLOC_FN(self._alloc)
        self.free = qx.FREE_FN(self._free)

    def _alloc(self, nbytes, ctx, stream):
        try:
            raw = self.torch.cuda.caching_allocator_alloc(int(nbytes) + 8, stream=stream or 0)
        except Exception:  # noqa: BLE001 - NULL tells the library
            return None
        self.base[raw + 8] = raw
        self.handed.append(raw + 8)
        return raw + 8

    def _free(self, ptr, ctx, stream):
        self.torch.cuda.caching_allocator_delete(self.base.pop(ptr))


@pytest.mark.parametrize("precision", [64, 32])
def test_caller_memory_off_16_byte_boundaries(precision):
    """The fused expansion stages tiles with bulk copies, which need 16-byte
    aligned planes; the library moves every block of a caller's allocator up
    to a 256-byte boundary, so a block 8 bytes off one gives the same result,
    bit for bit, as the default allocation, and every block goes back."""
    _, instrs = W.fan_in_deep(7, n=70, n_s=8, total=6000)
    n = 70
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    ref = qx.propagate(plan, precision=precision)
    al = _OffsetAllocator()
    for _ in range(3):  # the first run counts; later runs use the plan's record
        res = qx.propagate(plan, precision=precision, allocator=al)
        assert res.stats()["kernels"]["expand_emit"]["launches"] == 8
        a, b = (r.raw_device() for r in (res, ref))
        for u, v in zip(a, b):
            assert bool((u == v).all())
        res.free()
    assert al.handed and all(p % 256 == 8 for p in al.handed)
    assert not al.base  # every block was freed with the pointer it came from
    if precision == 64:
        compare_result(ref, O.propagate(n, instrs, mode="plan", threads=CORES))
    ref.free()


def test_final_clifford_block_on_all_qubits():
    """A Clifford block on every qubit after the last rotation (it touches the
    fan-out wires, so the last expansion cannot absorb it): the table-form
    pass runs over all terms on its own, against the oracle, in both
    precisions."""
    n = 100
    _, instrs = W.fan_in_deep(4, n=n, n_s=9, total=12000, final_mix=400)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    ref = O.propagate(n, instrs, mode="plan", threads=CORES)
    for _ in range(2):  # the count path, then the plan's record
        res = qx.propagate(plan)
        assert res.stats()["kernels"]["clifford_pass"]["launches"] >= 1
        compare_result(res, ref)
        res.free()
    r32 = qx.propagate(plan, precision=32)
    for g in (0, 9, 50, 99):
        got, want = r32.export_dict(g), O.as_dict(ref[g])
        assert got.keys() == want.keys()
        for s, w in want.items():
            assert abs(got[s] - w) <= 1e-5 * abs(w) + 1e-7


@pytest.mark.parametrize("n,n_s,total,mix", [(40, 12, 600, 60), (70, 11, 800, 80)])
def test_large_table_pass_in_tiles(n, n_s, total, mix):
    """A table-form pass over more than 65,536 terms runs in tiles staged by
    bulk copies (k_clifford_tiles): an all-qubit Clifford block after the
    last rotation of a chain with 2^n_s terms per heavy generator, one- and
    two-word strings, against the oracle in both precisions."""
    _, instrs = W.fan_in_deep(6, n=n, n_s=n_s, total=total, final_mix=mix)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    ref = O.propagate(n, instrs, mode="plan", threads=CORES)
    res = qx.propagate(plan)
    assert res.nterms >= (1 << 16)
    assert res.stats()["kernels"]["clifford_pass"]["launches"] >= 1
    compare_result(res, ref)
    res.free()
    r32 = qx.propagate(plan, precision=32)
    for g in (0, n_s, n - 1):
        got, want = r32.export_dict(g), O.as_dict(ref[g])
        assert got.keys() == want.keys()
        for s, w in want.items():
            assert abs(got[s] - w) <= 1e-5 * abs(w) + 1e-7
