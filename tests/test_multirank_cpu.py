"""The N > 1 path on CPU: two gloo ranks.

Clips are independent, so ranks shard by clip (weak scaling) with no
collective on the data path; the only exchange is the max-over-ranks time.
The pixel-sharded sketch (each rank sketches its pixel slab, then one sum
all-reduce) is also checked here on the oracle, since D_Y is linear in the
pixels."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    import videogen
    from oracle import cdmd as O
    from oracle import measurement as M
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # clip sharding and the job's time
        seed = bench.clip_seed(rank)
        local_s = 1.0 + rank          # rank 1 is the slow one
        job_s = bench.max_over_ranks(local_s, dist, "cpu")
        value = bench.job_throughput(200, world, job_s)
        seeds = [None] * world
        dist.all_gather_object(seeds, seed)
        # pixel-sharded sketch: rank r sketches pixels [r m / world, (r+1) m / world)
        clip = videogen.make_clip(40, 30, 12, seed=3)
        D = clip.video_matrix()
        k = 16
        Cm = M.measurement_matrix("gaussian", 11, k, clip.m)
        lo, hi = rank * clip.m // world, (rank + 1) * clip.m // world
        part = torch.from_numpy(O.sketch(Cm[:, lo:hi], D[lo:hi]))
        dist.all_reduce(part, op=dist.ReduceOp.SUM)
        full = O.sketch(Cm, D)
        out.put((rank, seeds, job_s, value, float(np.max(np.abs(part.numpy() - full)) / np.max(np.abs(full)))))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_clips_and_sketch_pixels():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, seeds, job_s, value, err in results:
        assert len(set(seeds)) == world            # every rank its own clip
        assert job_s == 2.0                         # the slowest rank's time
        assert value == pytest.approx(world * 200 / 2.0)
        assert err < 1e-13                          # sum of pixel-slab sketches = full sketch
