"""Ray-id sharding across ranks and the monitor merge (Sec. 2.2.1).

The paper runs McXtrace under MPI: the rays are split among processes and
the monitors are summed at the end.  Rays are independent and each ray's
random stream is a function of its id alone, so a rank needs nothing from
the others until the merge, and the merged monitors of any partition equal
those of one process tracing the union of the ranges (counts exactly, sums
up to the order of binary64 additions).

One process drives one GPU.  The merge is a plain sum all-reduce over
torch.distributed (NCCL on GPUs, gloo on host tensors); nothing else is
exchanged.
"""

from __future__ import annotations

import numpy as np


def split_range(begin: int, end: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous share of ray ids [begin, end) for `rank` of `world`: the
    shares tile the range in rank order and their sizes differ by at most 1."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world of {world}")
    if end < begin:
        raise ValueError("end < begin")
    n = end - begin
    q, r = divmod(n, world)
    b = begin + rank * q + min(rank, r)
    return b, b + q + (1 if rank < r else 0)


def step_range(rank: int, world: int, step: int, n_per_rank: int) -> tuple[int, int]:
    """Ray ids of `rank` in `step` when every rank traces n_per_rank rays per
    step (weak scaling): the ranks of one step cover
    [step*world*n, (step+1)*world*n) without overlap, and successive steps
    never reuse an id."""
    if world < 1 or not 0 <= rank < world or step < 0 or n_per_rank < 0:
        raise ValueError("invalid rank, world, step or ray count")
    b = (step * world + rank) * n_per_rank
    return b, b + n_per_rank


def merge_monitor(N, sw, sw2, group=None):
    """Sum one monitor's (N, sum w, sum w^2) over all ranks of `group`.

    Accepts numpy arrays (host; reduced through CPU tensors) or torch
    tensors (reduced in place on their device).  Counts travel as int64
    (a bin count below 2^63 is exact), sums as float64.  Returns the merged
    arrays in the input's kind."""
    import torch
    import torch.distributed as dist

    as_numpy = isinstance(N, np.ndarray)
    if as_numpy:
        tN = torch.from_numpy(np.ascontiguousarray(N).view(np.int64).copy())
        tsw = torch.from_numpy(np.ascontiguousarray(sw, dtype=np.float64).copy())
        tsw2 = torch.from_numpy(np.ascontiguousarray(sw2, dtype=np.float64).copy())
    else:
        tN, tsw, tsw2 = N, sw, sw2
    for t in (tN, tsw, tsw2):
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    if as_numpy:
        return (tN.numpy().view(np.asarray(N).dtype), tsw.numpy(), tsw2.numpy())
    return tN, tsw, tsw2


def merge_tallies(tallies: dict, group=None) -> dict:
    """Sum the per-component removed weight, rays emitted and weight totals
    (the dict Instrument.tallies() returns) over all ranks of `group`."""
    import torch
    import torch.distributed as dist

    lost = torch.from_numpy(np.asarray(tallies["lost"], dtype=np.float64).copy())
    sums = torch.tensor([tallies["sum_w0"], tallies["sum_wend"]], dtype=torch.float64)
    n_emit = torch.tensor([int(tallies["n_emit"])], dtype=torch.int64)
    for t in (lost, sums, n_emit):
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return {"lost": lost.numpy(), "n_emit": int(n_emit.item()), "sum_w0": float(sums[0]),
            "sum_wend": float(sums[1])}
