"""The monitor merge of the paper's MPI mode (Sec. 2.2.1: rays split among
workers, monitors summed at the end) on the GPU: instruments on one GPU
trace disjoint sub-ranges of the ray ids, as ranks would; their monitors,
read into device tensors, go through the package's all-reduce (a one-rank
NCCL group: the device code path of the merge) and are summed on the
device; the result equals one instrument tracing the union (counts exactly,
sums to rounding of the summation order)."""

import socket

import numpy as np
import pytest

from paper_2410_08747_gb300 import shard
from paper_2410_08747_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_08747_gb300 import build
    build.build()
    from paper_2410_08747_gb300 import mcx
    return mcx, torch


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_subrange_instruments_merge_on_device(env, prec):
    mcx, torch = env
    import torch.distributed as dist
    spec = wl.absorption_instrument(nx=32, ne=32)
    b, e, seed, world = 2_000_000, 2_000_000 + 3_000_001, 5, 3
    parts = [shard.split_range(b, e, r, world) for r in range(world)]
    ranks = [mcx.Instrument(spec, precision=prec) for _ in range(world)]
    for g, (pb, pe) in zip(ranks, parts):
        g.trace_range(pb, pe, seed)
    whole = mcx.Instrument(spec, precision=prec)
    whole.trace_range(b, e, seed)
    # device tensors go through NCCL, the host tallies through gloo
    dist.init_process_group("cpu:gloo,cuda:nccl", init_method=f"tcp://127.0.0.1:{_port()}", rank=0,
                            world_size=1)
    try:
        merged = None
        for g in ranks:
            N, sw, sw2 = g.monitor(2)
            t = (torch.from_numpy(N.view(np.int64).copy()).cuda(),
                 torch.from_numpy(sw.copy()).cuda(), torch.from_numpy(sw2.copy()).cuda())
            t = shard.merge_monitor(*t)                 # the device path of the merge
            merged = t if merged is None else tuple(m + x for m, x in zip(merged, t))
        tallies = [shard.merge_tallies(g.tallies()) for g in ranks]
    finally:
        dist.destroy_process_group()
    N, sw, sw2 = (m.cpu().numpy() for m in merged)
    No, swo, sw2o = whole.monitor(2)
    assert np.array_equal(N, No.view(np.int64)) and int(N.sum()) == e - b
    np.testing.assert_allclose(sw, swo, rtol=1e-12, atol=0)
    np.testing.assert_allclose(sw2, sw2o, rtol=1e-12, atol=0)
    t = whole.tallies()
    assert sum(x["n_emit"] for x in tallies) == t["n_emit"] == e - b
    # tallies: binary64 sums in the plain form, compensated binary32 per warp in the mixed one
    rt = 1e-9 if prec == "fp64" else 1e-6
    assert sum(x["sum_w0"] for x in tallies) == pytest.approx(t["sum_w0"], rel=rt)
    np.testing.assert_allclose(sum(x["lost"] for x in tallies), t["lost"], rtol=rt, atol=rt)
