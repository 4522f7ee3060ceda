"""The multi-rank host logic of bench.py on CPU: two gloo ranks agree on the
slowest rank's time, the whole-job rate counts every rank's independent work
(weak scaling, no data collective), each rank builds its own streams, and the
reference arm runs on rank 0 only."""
import os
import socket
import subprocess
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


# ---- splitting the batched and serving workloads over ranks ------------------------------

def _shard_rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch.distributed as dist
    import streamgen as sg
    from oracle import execute
    from paper_2401_12377_b300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    specs = sg.batched_specs(3, n_streams=8, lo=40, hi=300)
    mine = shard.partition_by_size([sp.target for sp in specs], world, rank)
    outs = {}
    for i in mine:                                 # this rank's streams, run by the oracle
        sp = specs[i]
        if sp.kind == "rl":
            _, b, _ = execute.run_rlsim(sg.RLSim(sp.seed, sp.rl), emit=True)
            outs[i] = {"pos": b["pos"], "vel": b["vel"]}
        else:
            st = sg.dnn_stream(sp.seed, batch=sp.dnn_batch, blocks=sp.dnn_blocks, weight_sets=min(sp.dnn_blocks, 24))
            outs[i] = {"h": execute.run_inorder(st.buffers, st.tasks)["h"]}
    # serving: request i to rank i mod world; each rank logs a latency per request
    arrivals, kinds = sg.poisson_arrivals(5, 400, 2000.0, 16)
    req = shard.partition_round_robin(len(arrivals), world, rank)
    lat = np.sin(np.arange(len(arrivals)))[req] ** 2 + 0.01 * req       # any per-request values
    gathered = shard.gather_values(dist, lat, rank, world)
    total = shard.gather_sum(dist, float(len(req)))
    q.put((rank, mine, outs, [int(x) for x in req], gathered, total))
    dist.barrier()
    dist.destroy_process_group()


def test_batched_and_serving_split_over_two_gloo_ranks():
    """The batch's streams split by size and the serving requests round-robin
    over two ranks: the ranks' parts are disjoint and together the one-GPU
    workload, each rank's stream outputs equal the oracle's for the same
    streams run alone, the stream loads stay balanced, and the latency logs
    gathered on rank 0 give the p50 / p99 of the concatenated logs."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import streamgen as sg
    from oracle import execute
    from paper_2401_12377_b300 import shard
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=300) for _ in range(world)), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    specs = sg.batched_specs(3, n_streams=8, lo=40, hi=300)
    parts = [set(g[1]) for g in got]
    assert parts[0].isdisjoint(parts[1]) and parts[0] | parts[1] == set(range(len(specs)))
    loads = [sum(specs[i].target for i in p) for p in parts]
    assert abs(loads[0] - loads[1]) <= max(sp.target for sp in specs)
    for _, mine, outs, _, _, _ in got:
        for i in mine:
            sp = specs[i]
            if sp.kind == "rl":
                _, b, _ = execute.run_rlsim(sg.RLSim(sp.seed, sp.rl), emit=True)
                want = {"pos": b["pos"], "vel": b["vel"]}
            else:
                st = sg.dnn_stream(sp.seed, batch=sp.dnn_batch, blocks=sp.dnn_blocks,
                                   weight_sets=min(sp.dnn_blocks, 24))
                want = {"h": execute.run_inorder(st.buffers, st.tasks)["h"]}
            for k in want:
                assert np.array_equal(outs[i][k].view(np.uint8), want[k].view(np.uint8)), (i, k)
    reqs = [set(g[3]) for g in got]
    assert reqs[0].isdisjoint(reqs[1]) and reqs[0] | reqs[1] == set(range(400))
    assert got[0][5] == got[1][5] == 400.0
    r0 = got[0][4]
    assert len(r0) == 400 and len(got[1][4]) == 0        # gathered on rank 0 only
    everything = np.concatenate([np.sin(np.arange(400))[sorted(r)] ** 2 + 0.01 * np.array(sorted(r))
                                 for r in reqs])
    assert shard.percentiles(r0) == shard.percentiles(everything)


def test_partition_by_size_is_longest_first_to_the_least_loaded():
    sys.path.insert(0, ROOT)
    from paper_2401_12377_b300 import shard
    sizes = [5, 9, 1, 7, 3]
    # LPT: 9 -> r0, 7 -> r1, 5 -> r1 (7 < 9), 3 -> r0 (9 < 12), 1 -> r0 (12 = 12, lower rank)
    assert shard.partition_by_size(sizes, 2, 0) == [1, 2, 4]
    assert shard.partition_by_size(sizes, 2, 1) == [0, 3]
    assert shard.partition_by_size(sizes, 1, 0) == list(range(5))
    assert list(shard.partition_round_robin(7, 3, 1)) == [1, 4]
    with pytest.raises(ValueError):
        shard.partition_by_size(sizes, 2, 2)
