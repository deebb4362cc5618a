"""World-size-2 gloo tests on CPU of the multi-rank host logic: a frame
sharded by tile rows renders, after one gather, exactly the single-rank
frame; the benchmark's timing aggregation takes the slowest rank."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    import sys
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _sharded_render(rank, world, port, out_path):
    _init(rank, world, port)
    try:
        import oracle
        from paper_2501_17792_gb300 import scene as S, shard
        sc = S.crowd(n_templates=2, n_gauss=512, sh_degree=1, cols=6, rows=4, width=96, height=72)
        W, H = sc.camera.width, sc.camera.height
        r0, r1 = shard.row_ranges(H, world)[rank]
        part = oracle.render(oracle.OracleScene(sc), lattice=(0, r0, 1, 1, W, r1 - r0))["rgba"]
        # gather variable-height parts: pad to the largest, then crop
        hmax = max(b - a for a, b in shard.row_ranges(H, world))
        buf = torch.zeros((hmax, W, 4), dtype=torch.float64)
        buf[: r1 - r0] = torch.from_numpy(part)
        parts = [torch.zeros_like(buf) for _ in range(world)]
        dist.all_gather(parts, buf)
        if rank == 0:
            img = np.concatenate([parts[k][: b - a].numpy() for k, (a, b) in
                                  enumerate(shard.row_ranges(H, world))], 0)
            np.save(out_path, img)
    finally:
        dist.destroy_process_group()


def test_row_sharded_frame_equals_single_rank(tmp_path):
    out = str(tmp_path / "stitched.npy")
    mp.spawn(_sharded_render, args=(2, _free_port(), out), nprocs=2, join=True)
    import oracle
    from paper_2501_17792_gb300 import scene as S
    sc = S.crowd(n_templates=2, n_gauss=512, sh_degree=1, cols=6, rows=4, width=96, height=72)
    ref = oracle.render(oracle.OracleScene(sc))["rgba"]
    got = np.load(out)
    assert ref[..., 3].max() > 0.5
    assert np.array_equal(got, ref)


def _aggregate(rank, world, port, out_path):
    _init(rank, world, port)
    try:
        import bench
        ms, value = bench.aggregate([5.0, 7.0][rank], 10, world, dist)
        if rank == 0:
            np.save(out_path, np.array([ms, value]))
    finally:
        dist.destroy_process_group()


def test_bench_aggregation_takes_the_slowest_rank(tmp_path):
    out = str(tmp_path / "agg.npy")
    mp.spawn(_aggregate, args=(2, _free_port(), out), nprocs=2, join=True)
    ms, value = np.load(out)
    assert ms == 7.0
    assert abs(value - 2 * 10 / 7e-3) < 1e-9


def test_row_ranges_cover_the_image_in_whole_tiles():
    from paper_2501_17792_gb300 import shard
    for H in (1, 15, 16, 17, 1080, 2160):
        for world in (1, 2, 3, 8):
            rr = shard.row_ranges(H, world)
            assert rr[0][0] == 0 and rr[-1][1] == H
            assert all(a <= b for a, b in rr)
            assert all(rr[k][1] == rr[k + 1][0] for k in range(world - 1))
            assert all(a % 16 == 0 or a == H for a, _ in rr)  # empty tail ranks start at H
            sizes = [(b - a + 15) // 16 for a, b in rr]
            assert max(sizes) - min(sizes) <= 1 or H < 16 * world


def test_sub_camera_maps_rows():
    from paper_2501_17792_gb300 import scene as S, shard
    cam = S.look_camera((0.0, 1.6, 0.0), 10.0, 64, 48)
    sub = shard.sub_camera(cam, 16, 32)
    assert sub.height == 16 and sub.width == 64 and sub.cy == cam.cy and sub.cx == cam.cx
    assert (sub.win_x0, sub.win_y0, sub.full_width, sub.full_height) == (0, 16, 64, 48)
    with pytest.raises(ValueError):
        shard.sub_camera(cam, 40, 60)
    with pytest.raises(ValueError):
        shard.sub_camera(cam, 8, 24)  # not on the tile grid
