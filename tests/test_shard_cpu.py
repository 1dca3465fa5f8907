"""The multi-rank logic on CPU: world_size 2 gloo ranks each render their row band
of a frame with the FP64 oracle and all-gather it; the stitched frame equals the
whole-frame render.  LPT assignment of frames: every frame once, balanced."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2305_07450_b300 import scenes as S, shard


def _band_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        w = S.whitted_256()
        w.params.width, w.params.height = 48, 37
        bands = shard.row_bands(w.params.height, world)
        y0, y1 = bands[rank]
        xs, ys = np.meshgrid(np.arange(w.params.width), np.arange(y0, y1))
        px = np.stack([xs.ravel(), ys.ravel()], 1).astype(np.int32)
        local = oracle.trace(w.scene, w.camera, w.params, px, threads=1)["rgb"].reshape(y1 - y0, w.params.width, 3)
        full = shard.gather_bands(torch.from_numpy(local), bands)
        if rank == 0:
            q.put(full.numpy())
    finally:
        dist.destroy_process_group()


def test_row_bands_over_two_gloo_ranks_stitch_the_frame():
    import oracle
    port = 29500 + os.getpid() % 1000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_band_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    full = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    w = S.whitted_256()
    w.params.width, w.params.height = 48, 37
    ref = oracle.render(w.scene, w.camera, w.params, threads=1)
    assert np.array_equal(full, ref)


@pytest.mark.parametrize("H,world", [(37, 2), (2160, 3), (5, 8), (720, 4)])
def test_row_bands_cover_once(H, world):
    bands = shard.row_bands(H, world)
    assert bands[0][0] == 0 and bands[-1][1] == H
    assert all(a == b0 for (_, a), (b0, _) in zip(bands, bands[1:]))
    sizes = [b - a for a, b in bands]
    assert max(sizes) - min(sizes) <= 1


def test_lpt_assigns_each_frame_once_and_balances():
    ws = S.batch_scenes()
    costs = [shard.frame_cost(w.scene, w.params) for w in ws]
    for world in (2, 4, 8):
        parts = shard.lpt(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(ws)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # LPT bound: no rank exceeds the ideal share by more than the largest item
        assert max(loads) <= sum(costs) / world + max(costs) + 1e-9
