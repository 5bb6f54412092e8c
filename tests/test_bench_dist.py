"""bench.py's multi-GPU host logic (replicas, weak scaling) as two gloo ranks on CPU:
disjoint source slices per rank, the max-over-ranks step time, and the barrier."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, _ = bench.dist_info()
        all_src = np.arange(100, 100 + 8 * w, dtype=np.uint32)
        mine = bench.shard_sources(all_src, r, w, 8)
        bench.barrier(w)
        slowest = bench.reduce_max(1.0 + r, w)
        out.put((r, mine.tolist(), slowest))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_sources_and_take_the_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, m0), (r1, s1, m1) = res
    assert (r0, r1) == (0, 1)
    assert len(s0) == len(s1) == 8 and not set(s0) & set(s1)
    assert sorted(s0 + s1) == list(range(100, 116))
    assert m0 == m1 == 2.0


def test_single_rank_helpers_need_no_process_group():
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    bench.barrier(1)
    assert bench.shard_sources(np.arange(8), 0, 1, 8).tolist() == list(range(8))


def test_gpus_flag_starts_that_many_ranks():
    """bench.py --gpus 2 without a torchrun environment starts 2 ranks itself (here they
    only join a gloo group and count themselves)."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items()
           if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT")}
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--gpus", "2",
                        "--launch-check"], capture_output=True, text=True, timeout=300,
                       env=env, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    assert lines == [{"launch_check": True, "world_size": 2, "ranks_counted": 2,
                      "gpus_flag": 2}]
