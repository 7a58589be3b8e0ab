"""Host-side sharding logic with 2 gloo ranks on CPU (no GPU): frame shards cover
every frame once, per-box results gathered from the ranks equal a single-process
run (the oracle stands in for the device path here), and the reported time is
the slowest rank's."""
import os
import socket

import numpy as np
import pytest

from paper_2604_07980_gb300 import dist as D


def test_frame_shards_partition():
    for n in (0, 1, 5, 32, 33):
        for world in (1, 2, 3, 8):
            got = [list(D.frame_shard(n, world, r)) for r in range(world)]
            flat = [f for g in got for f in g]
            assert flat == list(range(n))
            sizes = [len(g) for g in got]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        D.frame_shard(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist

    from oracle import oracle as orc
    from paper_2604_07980_gb300 import workloads as wl
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = wl.batch32x1200(n_frames=3, W=320, H=200, mean_boxes=6, side_range=(12, 80))
        frames = D.frame_shard(len(w.frames), world, rank)
        local, pos = D.boxes_of_frames(w.boxes, frames)
        fr = [(f.left, f.right, f.f_px, f.baseline_m) for f in w.frames[frames.start:frames.stop]]
        res = orc.match_batch(fr, local, orc.Params(**w.params)) if len(fr) else \
            {"disp": np.zeros(0, np.float32), "depth": np.zeros(0, np.float32), "flags": np.zeros(0, np.uint8)}
        out = D.gather_outputs(res, pos, w.n_boxes, dist)
        slowest = D.max_over_ranks(1.0 + rank, dist)
        if rank == 0:
            ref = orc.match_batch([(f.left, f.right, f.f_px, f.baseline_m) for f in w.frames], w.boxes,
                                  orc.Params(**w.params))
            ok = (np.array_equal(out["flags"], ref["flags"]) and
                  np.array_equal(out["disp"], ref["disp"], equal_nan=True) and
                  slowest == float(world))
            q.put(bool(ok))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_gather_equals_single_process():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    assert q.get(timeout=5) is True
