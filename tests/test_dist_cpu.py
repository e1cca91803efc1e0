"""Multi-process host logic on CPU: gloo process groups of world size 2.

The propagation itself needs no exchange (generators are independent), so
what is tested here is the host side of N > 1: generator sharding, the gather
of a range-sharded run (checked against a single-process run, with the
oracle doing the per-rank work), and the max/sum reduction of the bench.
"""
import os
import socket

import pytest

from paper_2505_03307_gb300 import dist as qdist

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, fn, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, fn(rank, world)))
    finally:
        dist.destroy_process_group()


def _run(fn, world=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, fn, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return [out[r] for r in range(world)]


def test_shard_generators_partition():
    for n in (1, 2, 7, 50, 100):
        for world in (1, 2, 3, 8):
            ranges = [qdist.shard_generators(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            for (a, b), (c, d) in zip(ranges, ranges[1:]):
                assert b == c and a <= b
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1
    cost = [1] * 10 + [100] * 2 + [1] * 10
    ranges = [qdist.shard_generators(22, r, 2, cost) for r in range(2)]
    assert ranges[0][0] == 0 and ranges[1][1] == 22 and ranges[0][1] == ranges[1][0]
    assert 10 <= ranges[0][1] <= 12


def _sharded_oracle(rank, world):
    from oracle import oracle as O
    from paper_2505_03307_gb300 import workloads as W
    n, instrs = W.random_layers(3)
    b, e = qdist.shard_generators(n, rank, world)
    local = [O.as_dict(g) for g in O.propagate(n, instrs, mode="plan", gens=(b, e))]
    return qdist.gather_generators(local, b, n)


def test_range_sharded_run_gathers_to_full_result():
    from oracle import oracle as O
    from paper_2505_03307_gb300 import workloads as W
    n, instrs = W.random_layers(3)
    full = [O.as_dict(g) for g in O.propagate(n, instrs, mode="plan")]
    results = _run(_sharded_oracle)
    for r in results:
        assert r == full


def _reduce(rank, world):
    return qdist.reduce_step_times(10.0 + rank, 100.0 * (rank + 1))


def test_reduce_step_times_max_and_sum():
    results = _run(_reduce)
    for mx, sm in results:
        assert mx == 11.0
        assert sm == 300.0


def test_single_process_passthrough():
    assert qdist.reduce_step_times(3.0, 4.0) == (3.0, 4.0)
    assert qdist.gather_generators([1, 2], 0, 2) == [1, 2]
    with pytest.raises(ValueError):
        qdist.gather_generators([1], 0, 2)


def _split_like_the_bench(rank, world):
    """The bench's strong-scaling path (dist.run_generator_split with ranges
    balanced by an earlier run's term counts), the oracle standing in for
    each rank's propagation: per-generator (term count, sum of squares)."""
    from oracle import oracle as O
    from paper_2505_03307_gb300 import workloads as W
    n, instrs = W.fan_in_deep(2, n=24, n_s=6, total=900)
    cost = [len(O.as_dict(g)) for g in O.propagate(n, instrs, mode="plan")]

    def run_range(b, e):
        res = O.propagate(n, instrs, mode="plan", gens=(b, e))
        return [(len(O.as_dict(g)), sum(w * w for w in O.as_dict(g).values())) for g in res]

    rows, rng = qdist.run_generator_split(n, rank, world, cost, run_range)
    return rows, rng, cost


def test_generator_split_of_the_bench_gathers_every_generator():
    from oracle import oracle as O
    from paper_2505_03307_gb300 import workloads as W
    n, instrs = W.fan_in_deep(2, n=24, n_s=6, total=900)
    full = [O.as_dict(g) for g in O.propagate(n, instrs, mode="plan")]
    results = _run(_split_like_the_bench)
    (rows0, r0, cost), (rows1, r1, _) = results
    assert rows0 == rows1
    assert [c for c, _ in rows0] == [len(d) for d in full]
    assert all(abs(s2 - 1.0) < 1e-12 for _, s2 in rows0)
    assert r0[0] == 0 and r0[1] == r1[0] and r1[1] == n
    # balanced by cost: each half holds about half of the terms
    c0 = sum(cost[r0[0]:r0[1]])
    assert abs(c0 - sum(cost) / 2) <= max(cost)
