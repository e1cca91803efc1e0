"""Fan-out steps launched on the plan's record of its last run.

A plan remembers, per fan-out step, whether its last run was a pure expansion
(with its output size) or block-ordered merges over a set of wires, and the
next run launches that work before the per-generator letter masks come back.
These tests run one plan repeatedly with options that change the outcome
(generator ranges that change the output size or the merge wires, in-place
merges switched off, FP32), so that each kind of wrong guess happens, and
compare every result with a fresh plan (which has no record) bit for bit and
with the oracle.
"""
import numpy as np
import pytest

from gpu_util import compare_result
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


def _sorted(res):
    x, z, w, g = (t.cpu().numpy() for t in res.raw_device())
    keys = [g] + [x[:, k] for k in range(x.shape[1])] + [z[:, k] for k in range(z.shape[1])]
    order = np.lexsort(tuple(reversed(keys)))
    return g[order], x[order], z[order], w[order]


def _same(a, b):
    ga, xa, za, wa = _sorted(a)
    gb, xb, zb, wb = _sorted(b)
    assert np.array_equal(ga, gb) and np.array_equal(xa, xb) and np.array_equal(za, zb)
    assert np.array_equal(wa, wb)


def _fresh(n, instrs, **kw):
    return qx.propagate(qx.group_ops(qx.load_circuit(n, instrs)), **kw)


def test_second_run_keeps_the_guesses_and_the_result():
    n, instrs = W.fan_in_heavy(2, n=20, n_s=8, total=500, tail=80)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    first = qx.propagate(plan)
    second = qx.propagate(plan)
    s1, s2 = first.stats(), second.stats()
    assert s1["guesses_held"] == 0 and s1["guesses_missed"] == 0
    # the T layer (an expansion) and the RZ layer (block-ordered merges)
    assert s2["guesses_held"] == 2 and s2["guesses_missed"] == 0
    assert s2["host_syncs"] == s1["host_syncs"] - 2
    _same(first, second)
    compare_result(second, O.propagate(n, instrs, mode="plan", threads=8))


def test_generator_ranges_change_sizes_and_merge_wires():
    """Generators inside the fan-out set S have two strings and merge on one
    wire each; those outside have 2^8 and merge on all eight wires.  Changing
    the range makes the recorded output size too small or too large.  (A
    block-ordered guess is decided by the device alone: over generators
    inside S its blocks on the other wires have one member and are complete,
    which is exact.  Misses are covered by the tests below.)"""
    n, instrs = W.fan_in_heavy(3, n=20, n_s=8, total=500, tail=80)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    held = missed = 0
    for gens in [(0, 4), (0, 20), (12, 20), (2, 6), (0, 20), (0, 20)]:
        res = qx.propagate(plan, gens=gens)
        st = res.stats()
        held += st["guesses_held"]
        missed += st["guesses_missed"]
        _same(res, _fresh(n, instrs, gens=gens))
        compare_result(res, O.propagate(n, instrs, mode="plan", gens=gens, threads=8))
    assert held > 0


def test_options_that_disable_the_recorded_path():
    n, instrs = W.fan_in_heavy(4, n=20, n_s=8, total=500, tail=80)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    base = qx.propagate(plan)
    # in-place merges off: the block record must not be used
    off = qx.propagate(plan, inplace=False)
    assert off.stats()["block_steps"] == 0
    _same(off, _fresh(n, instrs, inplace=False))
    # FP32 on the same plan, then FP64 again
    f32 = qx.propagate(plan, precision=32)
    _same(f32, _fresh(n, instrs, precision=32))
    again = qx.propagate(plan)
    _same(again, base)
    # pruning: the records hold output sizes before pruning
    pr = qx.propagate(plan, eps=1e-3)
    _same(pr, _fresh(n, instrs, eps=1e-3))


@pytest.mark.parametrize("seed", range(6))
def test_random_circuits_repeated(seed):
    """Random small circuits with T / RZ layers on random subsets, one plan
    propagated over a sequence of generator ranges."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(6, 13))
    _, instrs = W.random_small_2q(seed, n, 60, p2=0.2)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    for _ in range(4):
        a = int(rng.integers(0, n))
        b = int(rng.integers(a + 1, n + 1))
        res = qx.propagate(plan, gens=(a, b))
        _same(res, _fresh(n, instrs, gens=(a, b)))
        compare_result(res, O.propagate(n, instrs, mode="plan", gens=(a, b), threads=4))


def test_block_count_beyond_the_recorded_table():
    """Blocks of 16 (RZ on 4 of 12 fan-out wires): a run over one generator
    records 256 blocks, and the block table of the next run, over 28
    generators (7,168 blocks), is sized from that record.  The claim gives up
    early, the step is repeated at full size, and the result is unchanged."""
    import math
    n, S = 40, list(range(12))
    rest = [q for q in range(n) if q not in S]
    rng = np.random.default_rng(11)
    instrs = [("H", q, -1, 0.0) for q in range(n)]
    instrs += [("CX", i, q, 0.0) for i in rest for q in S]
    instrs += [("T", q, -1, 0.0) for q in S]
    instrs += [("CX", n - 2, n - 1, 0.0)]  # closes the T operator (as in fan_in_heavy)
    instrs += [("RZ", q, -1, float(rng.uniform(0, 2 * math.pi))) for q in S[:4]]
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    one = qx.propagate(plan, gens=(20, 21))
    assert one.stats()["block_steps"] == 1
    many = qx.propagate(plan, gens=(12, 40))
    st = many.stats()
    assert st["block_steps"] == 1 and st["guesses_missed"] >= 1
    _same(many, _fresh(n, instrs, gens=(12, 40)))
    compare_result(many, O.propagate(n, instrs, mode="plan", gens=(12, 40), threads=8))
    again = qx.propagate(plan, gens=(12, 40))  # now recorded at full count
    assert again.stats()["guesses_missed"] == 0
    _same(again, many)


def test_checks_at_the_end_of_the_run():
    """After two runs that kept a step's guess, the next run launches the step
    without any read-back and checks it at the end of the run (one host
    round trip in all); a run whose end-of-run check fails is repeated with
    every check on the spot, and its result equals a fresh plan's."""
    n, instrs = W.fan_in_heavy(6, n=20, n_s=8, total=500, tail=80)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    runs = [qx.propagate(plan) for _ in range(4)]
    syncs = [r.stats()["host_syncs"] for r in runs]
    assert syncs[1] == syncs[0] - 2 and syncs[2] == syncs[1]
    assert syncs[3] == 1  # both fan-out steps checked at the end
    assert runs[3].stats()["guesses_held"] == 2
    for r in runs[1:]:
        _same(r, runs[0])
    # other generators: the recorded sizes and merge wires are wrong
    other = qx.propagate(plan, gens=(0, 6))
    st = other.stats()
    assert st["guesses_missed"] >= 1
    _same(other, _fresh(n, instrs, gens=(0, 6)))
    compare_result(other, O.propagate(n, instrs, mode="plan", gens=(0, 6), threads=8))
    # FP32 with the records of FP64 runs, then FP64 again
    for _ in range(3):
        f32 = qx.propagate(plan, precision=32)
    _same(f32, _fresh(n, instrs, precision=32))
    for _ in range(3):
        again = qx.propagate(plan)
    _same(again, runs[0])


def test_checks_at_the_end_on_the_large_workload_shape():
    """A chain of expansions (one fan-out qubit per step, 12 steps) where every
    step is checked at the end of the run after two runs; then a generator
    range that changes every output size."""
    n, instrs = W.fan_in_deep(2, n=40, n_s=12, total=3000)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    a = [qx.propagate(plan) for _ in range(4)][-1]
    assert a.stats()["host_syncs"] == 1
    _same(a, _fresh(n, instrs))
    b = qx.propagate(plan, gens=(12, 20))
    _same(b, _fresh(n, instrs, gens=(12, 20)))
    compare_result(b, O.propagate(n, instrs, mode="plan", gens=(12, 20), threads=8))


class _LoggingAllocator:
    """PyTorch's caching allocator behind the library's allocator callbacks,
    logging the size of every request; with ``refuse_new`` it refuses, once,
    the first request whose size is not in that set."""

    def __init__(self, refuse_new=None):
        import torch
        self.torch = torch
        self.sizes = []
        self.refuse_new = refuse_new
        self.refused = []
        self.alloc = qx.ALLOC_FN(self._alloc)
        self.free = qx.FREE_FN(self._free)

    def _alloc(self, nbytes, ctx, stream):
        nbytes = int(nbytes)
        self.sizes.append(nbytes)
        if self.refuse_new is not None and not self.refused and nbytes not in self.refuse_new:
            self.refused.append(nbytes)
            return None
        try:
            return self.torch.cuda.caching_allocator_alloc(nbytes, stream=stream or 0)
        except Exception:  # noqa: BLE001 - NULL tells the library
            return None

    def _free(self, ptr, ctx, stream):
        self.torch.cuda.caching_allocator_delete(ptr)


def test_recorded_size_that_cannot_be_allocated_falls_back():
    """The plan's record of an expansion holds the full run's output size; a
    run over fewer generators whose allocation at that size fails goes back
    to counting first, counts the miss and gives the same result."""
    n, instrs = W.fan_in_heavy(2, n=20, n_s=8, total=500, tail=80)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    for _ in range(3):
        qx.propagate(plan).free()
    gens = (12, 20)
    fresh_log = _LoggingAllocator()
    fresh = _fresh(n, instrs, gens=gens, allocator=fresh_log)
    refusing = _LoggingAllocator(refuse_new=set(fresh_log.sizes))
    res = qx.propagate(plan, gens=gens, allocator=refusing)
    assert len(refusing.refused) == 1, refusing.refused
    assert res.stats()["guesses_missed"] >= 1
    _same(res, fresh)
    compare_result(res, O.propagate(n, instrs, mode="plan", gens=gens, threads=8))
    res.free()
    fresh.free()


def test_recorded_range_offsets_skip_the_count():
    """A chain of small expansions: the second run, whose guesses held on the
    spot, records each step's range offsets, and from the third run on every
    step is one emission on them (no count, no scan) with its checks at the
    end of the run.  The same plan started from the generators in reverse
    order has the same step sizes but other range shares: the emission flags
    the ranges, the run is repeated with every check on the spot, the result
    equals a fresh plan's, and the records that failed are retired."""
    n, instrs = W.fan_in_deep(3, n=40, n_s=12, total=3000)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    runs = [qx.propagate(plan) for _ in range(4)]
    counts = [r.stats()["kernels"]["expand_count"]["launches"] for r in runs]
    assert counts[0] == counts[1] == 12 and counts[2] == counts[3] == 0, counts
    for r in runs[2:]:
        st = r.stats()
        assert st["host_syncs"] == 1 and st["guesses_held"] == 12 and st["guesses_missed"] == 0
        assert st["kernels"]["expand_scan"]["launches"] == 0
        _same(r, runs[0])
    compare_result(runs[3], O.propagate(n, instrs, mode="plan", threads=8))
    # generators in reverse order: same totals per step, other shares per range
    rev = ["".join("Z" if q == j else "I" for q in range(n)) for j in reversed(range(n))]
    res = qx.propagate_from(plan, rev)
    st = res.stats()
    assert st["guesses_missed"] >= 1
    assert st["kernels"]["expand_count"]["launches"] == 12
    _same(res, qx.propagate_from(qx.group_ops(qx.load_circuit(n, instrs)), rev))
    # the records whose check failed are retired: later runs count those
    # steps again (their guesses still hold)
    later = [qx.propagate(plan) for _ in range(3)][-1]
    assert 0 < later.stats()["kernels"]["expand_count"]["launches"] <= 12
    assert later.stats()["guesses_missed"] == 0
    _same(later, runs[0])


def test_recorded_offsets_with_pruning_and_fp32():
    """Records are per precision and threshold: an FP64 record is not used by
    FP32 or pruned runs (their sizes differ), and each configuration's own
    runs give the fresh plan's result."""
    n, instrs = W.fan_in_deep(4, n=40, n_s=10, total=2500)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    for kw in ({}, {"precision": 32}, {"eps": 1e-3}, {"eps": 1e-3, "precision": 32}, {}):
        rs = [qx.propagate(plan, **kw) for _ in range(3)]
        _same(rs[-1], _fresh(n, instrs, **kw))
