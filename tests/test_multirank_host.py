"""Host logic of the multi-GPU bench path, run as world_size-2 gloo ranks on
the CPU: max/sum reductions over ranks, one camera view per rank, the
reference arm's rank-0-only rule, and one batch split into contiguous ray
ranges whose per-rank results (the oracle's march and render on each range)
concatenate to the unsplit batch's.  No GPU is touched."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        out = {
            "env": (r, w, local),
            "max": bench.reduce_max(1.5 + 10.0 * rank, dist),
            "sum": bench.reduce_sum(1000 + rank, dist),
            "view": bench.view_for_rank(rank),
        }
        # one batch split into contiguous ray ranges: each rank marches and renders its own range
        import argparse
        import numpy as np
        import oracle as orc
        a = argparse.Namespace(shard="batch", width=24, height=20)
        w = bench.rank_workload(a, rank, world)
        g, m = w.grid, w.march
        bits, _ = orc.density_grid(g, w.blobs)
        pk = orc.march(w.rays_o, w.rays_d, g.aabb_min, g.aabb_max, g.res, g.n_levels, bits, m.step, m.max_steps,
                       m.t_min, m.t_max, blobs=w.blobs, eps=m.early_stop_eps)
        sig, rgb = orc.field_samples(w.rays_o, w.rays_d, pk["ray_indices"], pk["t_starts"], pk["t_ends"], w.blobs)
        out["range"] = bench.ray_range(24 * 20, rank, world)
        out["counts"] = np.diff(pk["offsets"])
        out["rgb"] = orc.render_fwd(pk["offsets"], pk["t_starts"], pk["t_ends"], sig.astype(np.float32),
                                    rgb.astype(np.float32), w.bg)["rgb"]
        if rank != 0:
            # the reference arm prints from rank 0 only; other ranks exit 0 without work
            out["ref_rc"] = bench.main(["--impl", "reference", "--gpus", str(world), "--steps", "1",
                                        "--warmup", "0"])
        dist.barrier()
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_shard_views_and_batches():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        assert res[r]["env"] == (r, world, r)
        assert res[r]["max"] == pytest.approx(11.5)          # max over ranks of 1.5 + 10 r
        assert res[r]["sum"] == pytest.approx(2001.0)        # 1000 + 1001
    assert res[0]["view"] != res[1]["view"]                  # each rank renders its own view
    assert res[1]["ref_rc"] == 0
    # the contiguous ranges cover the batch once, and their results are the unsplit batch's
    import numpy as np
    import oracle as orc
    import workloads
    assert res[0]["range"] == (0, 240) and res[1]["range"] == (240, 480)
    w = workloads.c2_image(24, 20, view=0)
    g, m = w.grid, w.march
    bits, _ = orc.density_grid(g, w.blobs)
    pk = orc.march(w.rays_o, w.rays_d, g.aabb_min, g.aabb_max, g.res, g.n_levels, bits, m.step, m.max_steps,
                   m.t_min, m.t_max, blobs=w.blobs, eps=m.early_stop_eps)
    sig, rgb = orc.field_samples(w.rays_o, w.rays_d, pk["ray_indices"], pk["t_starts"], pk["t_ends"], w.blobs)
    full = orc.render_fwd(pk["offsets"], pk["t_starts"], pk["t_ends"], sig.astype(np.float32),
                          rgb.astype(np.float32), w.bg)["rgb"]
    np.testing.assert_array_equal(np.concatenate([res[0]["counts"], res[1]["counts"]]), np.diff(pk["offsets"]))
    np.testing.assert_array_equal(np.concatenate([res[0]["rgb"], res[1]["rgb"]]), full)
    assert np.diff(pk["offsets"]).sum() > 0


def test_single_process_reductions_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.25) == 3.25 and bench.reduce_sum(7) == 7.0


def test_ray_ranges_cover_each_ray_once():
    sys.path.insert(0, ROOT)
    import bench
    for n in (0, 1, 5, 640000, 640001):
        for world in (1, 2, 3, 8):
            rs = [bench.ray_range(n, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            sizes = [hi - lo for lo, hi in rs]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 0
