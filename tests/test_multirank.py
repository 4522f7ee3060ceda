"""The multi-rank host logic of bench.py on CPU: two gloo ranks agree on the
slowest rank's time, the whole-job rate counts every rank's independent work
(weak scaling, no data collective), each rank builds its own streams, and the
reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

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
    import streamgen as sg
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, local = bench.ranks()
    ms = 10.0 + 5.0 * r                         # the last rank is the slowest
    m = bench.max_over_ranks(ms, dist, "cpu")
    v = bench.whole_job_rate(w, 1000.0, m / 1e3)
    seeds = [s.seed for s in sg.batched_specs(1 + r, n_streams=4)]
    q.put((r, w, local, m, v, seeds))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, local, m, v, _ in got:
        assert w == world and local == r
        assert m == 15.0                                   # max over ranks, on every rank
        assert abs(v - world * 1000.0 / 0.015) < 1e-6     # units of all ranks / slowest time
    assert got[0][5] != got[1][5]                          # each rank its own streams


def test_reference_arm_runs_on_rank0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
