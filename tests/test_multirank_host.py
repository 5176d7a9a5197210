"""Host logic of the multi-GPU bench path, run as world_size-2 gloo ranks on
the CPU: max/sum reductions over ranks, one camera view per rank, and the
reference arm's rank-0-only rule.  No GPU is touched."""
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
        if rank != 0:
            # the reference arm prints from rank 0 only; other ranks exit 0 without work
            out["ref_rc"] = bench.main(["--impl", "reference", "--gpus", str(world), "--steps", "1",
                                        "--warmup", "0"])
        dist.barrier()
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_shard_views():
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


def test_single_process_reductions_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.25) == 3.25 and bench.reduce_sum(7) == 7.0
