"""The multi-rank path on the host: two gloo ranks each trace their share of
the ray ids (with the oracle, standing in for one GPU each), merge the
monitors with the package's all-reduce, and equal one process tracing the
whole range.  A rank that dies before the merge makes the survivor's merge
raise instead of hang."""

import datetime
import os
import pickle
import socket
import tempfile

import numpy as np
import pytest

from paper_2410_08747_gb300 import shard
from paper_2410_08747_gb300 import workloads as wl

N_RAYS = 30_001
SEED = 9


def test_split_range_tiles_in_order():
    for n in (0, 1, 7, 30_001):
        for world in (1, 2, 3, 8):
            parts = [shard.split_range(100, 100 + n, r, world) for r in range(world)]
            assert parts[0][0] == 100 and parts[-1][1] == 100 + n
            assert all(parts[i][1] == parts[i + 1][0] for i in range(world - 1))
            sizes = [e - b for b, e in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.split_range(0, 10, 2, 2)


def test_step_ranges_never_overlap():
    seen = set()
    for step in range(4):
        lo = None
        for r in range(3):
            b, e = shard.step_range(r, 3, step, 5)
            if lo is not None:
                assert b == lo
            lo = e
            ids = set(range(b, e))
            assert not ids & seen
            seen |= ids
    assert seen == set(range(60))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir, die_rank):
    import torch.distributed as dist

    from oracle import oracle
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world, timeout=datetime.timedelta(seconds=20))
    spec = wl.flat_slit_instrument()
    b, e = shard.split_range(0, N_RAYS, rank, world)
    res = oracle.trace(spec, b, e, SEED, 64)
    if rank == die_rank:
        os._exit(0)                    # leaves between steps, before the merge
    try:
        merged = {c: shard.merge_monitor(*res.monitor(c)) for c in (2, 3)}
        t = shard.merge_tallies({"lost": res.lost, "n_emit": res.n_emit,
                                 "sum_w0": res.sum_w0, "sum_wend": res.sum_wend})
        out = {"ok": True, "mon": merged, "tallies": t}
    except Exception as exc:           # noqa: BLE001 - reported to the parent
        out = {"ok": False, "error": repr(exc)}
    with open(os.path.join(out_dir, f"rank{rank}.pkl"), "wb") as f:
        pickle.dump(out, f)
    if out["ok"]:
        dist.destroy_process_group()
    else:
        # the result is written; tearing down a group whose peer died can
        # abort the interpreter at exit, which is not what this test checks
        os._exit(0)


def _spawn(world, die_rank=-1):
    import torch.multiprocessing as mp
    out = tempfile.mkdtemp()
    mp.start_processes(_worker, args=(world, _free_port(), out, die_rank), nprocs=world,
                       join=True, start_method="spawn")
    res = {}
    for r in range(world):
        p = os.path.join(out, f"rank{r}.pkl")
        if os.path.exists(p):
            with open(p, "rb") as f:
                res[r] = pickle.load(f)
    return res


def test_two_gloo_ranks_equal_one_process(orc):
    pytest.importorskip("torch")
    res = _spawn(2)
    assert res[0]["ok"] and res[1]["ok"], res
    spec = wl.flat_slit_instrument()
    ref = orc.trace(spec, 0, N_RAYS, SEED, 64)
    for c in (2, 3):
        N, sw, sw2 = ref.monitor(c)
        for r in (0, 1):
            mN, msw, msw2 = res[r]["mon"][c]
            assert np.array_equal(mN.astype(np.int64), N)
            np.testing.assert_allclose(msw, sw, rtol=1e-12, atol=0)
            np.testing.assert_allclose(msw2, sw2, rtol=1e-12, atol=0)
    t = res[0]["tallies"]
    assert t["n_emit"] == ref.n_emit == N_RAYS
    assert t["sum_w0"] == pytest.approx(ref.sum_w0, rel=1e-12)
    assert t["sum_wend"] == pytest.approx(ref.sum_wend, rel=1e-12)
    np.testing.assert_allclose(t["lost"], ref.lost, rtol=1e-12, atol=1e-9)


def test_dead_rank_makes_merge_raise(orc):
    pytest.importorskip("torch")
    res = _spawn(2, die_rank=1)
    assert 1 not in res
    assert res[0]["ok"] is False and res[0]["error"]
