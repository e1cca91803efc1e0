"""Host-side logic of multi-process runs (one process per GPU).

The n generators evolve independently (Eq. 1: each Z_j is propagated on its
own), so the work splits across processes with no exchange during the
propagation.  Two forms are used:

* independent circuits per rank (weak scaling, the bench): each rank
  propagates its own seeded instance; only the timings are reduced;
* one circuit split by generator range (strong scaling): rank r propagates
  generators [begin_r, end_r) (``qx_prop_opts.gen_begin/gen_end``) and the
  results are gathered on the host at the end.

Nothing here touches device data: the only collectives are small host-side
reductions and gathers over ``torch.distributed`` (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations


def shard_generators(n: int, rank: int, world: int, cost=None):
    """Contiguous generator range [begin, end) of `rank` out of `world`.

    With `cost` (a predicted cost per generator, e.g. term counts), ranges are
    cut where the running cost crosses multiples of total/world; otherwise the
    n generators are split as evenly as possible.  Ranges partition [0, n).
    """
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    if cost is None:
        base, extra = divmod(n, world)
        begin = rank * base + min(rank, extra)
        return begin, begin + base + (1 if rank < extra else 0)
    if len(cost) != n:
        raise ValueError("cost must have one entry per generator")
    total = float(sum(cost))
    cuts = [0]
    run = 0.0
    k = 1
    for j, c in enumerate(cost):
        run += float(c)
        while k < world and run >= total * k / world and len(cuts) <= k:
            cuts.append(j + 1)
            k += 1
    while len(cuts) < world:
        cuts.append(n)
    cuts.append(n)
    return cuts[rank], max(cuts[rank], cuts[rank + 1])


def reduce_step_times(total_ms: float, updates: float, device=None):
    """(max of total_ms over ranks, sum of updates over ranks).

    The whole job is as slow as its slowest rank; the work is the sum.  Runs
    without a process group return the local values.
    """
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(total_ms), float(updates)
    dev = device if device is not None else "cpu"
    mx = torch.tensor([float(total_ms)], dtype=torch.float64, device=dev)
    sm = torch.tensor([float(updates)], dtype=torch.float64, device=dev)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx.item()), float(sm.item())


def gather_generators(local: list, begin: int, n: int):
    """Gather per-generator results of a range-sharded run onto every rank.

    `local` holds the results of generators [begin, begin + len(local)); the
    return value is the list of all n results in generator order.
    """
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        if begin != 0 or len(local) != n:
            raise ValueError("a single process must hold all generators")
        return list(local)
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, (begin, list(local)))
    out = [None] * n
    for b, items in parts:
        for k, item in enumerate(items):
            if out[b + k] is not None:
                raise ValueError(f"generator {b + k} was computed twice")
            out[b + k] = item
    if any(x is None for x in out):
        raise ValueError("some generators were not computed")
    return out


def run_generator_split(n: int, rank: int, world: int, cost, run_range):
    """Strong scaling of one circuit: this rank's generator range, balanced by
    `cost` (e.g. the per-generator term counts of an earlier run), is
    propagated by ``run_range(begin, end)``, which returns one row per
    generator of the range; the rows of all ranks are gathered in generator
    order.  Returns (all rows, (begin, end))."""
    begin, end = shard_generators(n, rank, world, cost)
    rows = list(run_range(begin, end))
    if len(rows) != end - begin:
        raise ValueError("run_range must return one row per generator of its range")
    return gather_generators(rows, begin, n), (begin, end)
