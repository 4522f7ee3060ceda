"""GPU parity: the device scheduler against the CPU oracle, through the C ABI.

For every stream: the upstream-candidate masks the scheduler logged decode to
exactly the oracle's window DAG D_W; the ticket log passes the oracle's
legality check against the full DAG E; outputs are bit-identical to the
in-order GPU run and match the oracle's in-order execution (bit for bit for the
elementwise and rigid-sphere bodies, within the GEMV bound below for the DNN).
"""
import numpy as np
import pytest
import torch

import streamgen as sg
from oracle import addresses, deps, execute

import fpcheck

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2401_12377_b300 import build
    build.build()
    from paper_2401_12377_b300 import acs, harness

# Streams with GEMV tasks: the oracle's GEMV is the exact dot product rounded
# once; the GPU's fp32 fma order differs from it by rounding. Single GEMV tasks
# and every GEMV of an unrolled DNN stream are checked element by element
# against the inner-product bound (fpcheck.check_tasks_on_own_inputs); whole
# streams element by element at 1e-5 relative with the vector-RMS cancellation
# floor of fpcheck.assert_per_element.


def oracle_dags(stream):
    segs = addresses.stream_segments(stream.tasks, stream.buffers)
    E = deps.full_dag(segs)
    return E, deps.window_dag(E, stream.window)


def check_log(masks, start, retire, E, D, W):
    got = deps.edges_from_masks([int(m) for m in masks], W)
    assert got == D, f"DAG mismatch: missing {sorted(D - got)[:5]} extra {sorted(got - D)[:5]}"
    bad = deps.check_legal(E, [int(x) for x in start], [int(x) for x in retire])
    assert not bad, bad[:5]


def assert_same(a, b, what):
    for k in a:
        assert np.array_equal(a[k].view(np.uint8), b[k].view(np.uint8)), f"{what}: buffer {k} differs"


# ---- elementwise streams (16 buffers x 4096 floats, window 8) ----------------

@pytest.mark.parametrize("seed", [0, 1, 2, 3, 7, 11, 42, 99])
@pytest.mark.parametrize("ranges", [False, True])
def test_elementwise_stream_parity(seed, ranges):
    s = sg.elementwise_stream(seed, ranges=ranges)
    E, D = oracle_dags(s)
    out, st, (masks, start, retire) = harness.run_stream(s, log=True)
    check_log(masks, start, retire, E, D, s.window)
    ref_gpu, _, _ = harness.run_stream(s, mode="inorder")
    assert_same(out, ref_gpu, "window vs in-order GPU")
    ref = execute.run_inorder(s.buffers, s.tasks)
    assert_same(out, ref, "GPU vs oracle")            # bit-exact (the bar, 1e-5 relative, is implied)
    assert st["tasks_flushed"] == len(s.tasks) and st["sched_inserts"] == len(s.tasks)


@pytest.mark.parametrize("W", [1, 2, 3, 8, 32, 33, 64])
def test_window_sizes_give_identical_outputs(W):
    s = sg.elementwise_stream(5, n_tasks=96, ranges=True)
    s.window = W
    E, D = oracle_dags(s)
    out, _, (masks, start, retire) = harness.run_stream(s, log=True)
    check_log(masks, start, retire, E, D, W)
    assert_same(out, execute.run_inorder(s.buffers, s.tasks), f"W={W}")


@pytest.mark.parametrize("slots", [1, 2, 7, 64, 200, 0])
def test_cta_slot_counts_give_identical_outputs(slots):
    """Any worker-CTA count up to the co-resident maximum (0: the maximum)."""
    s = sg.elementwise_stream(9, n_tasks=64)
    E, D = oracle_dags(s)
    out, st, (masks, start, retire) = harness.run_stream(s, log=True, cta_slots=slots)
    assert st["cta_slots"] == slots or (slots == 0 and st["cta_slots"] == st["grid"] - 1)
    check_log(masks, start, retire, E, D, s.window)
    assert_same(out, execute.run_inorder(s.buffers, s.tasks), f"slots={slots}")


# ---- static irregular DAG (randomly wired GEMV network) -------------------------------

@pytest.mark.parametrize("seed,W", [(1, 32), (2, 8), (3, 64)])
def test_random_wire_parity(seed, W):
    s = sg.random_wire_stream(seed, n_nodes=16, stages=2, window=W)
    E, D = oracle_dags(s)
    out, st, (masks, start, retire) = harness.run_stream(s, log=True)
    check_log(masks, start, retire, E, D, W)
    ref_gpu, _, _ = harness.run_stream(s, mode="inorder")
    assert_same(out, ref_gpu, "window vs in-order GPU")
    fpcheck.assert_per_element(out, execute.run_inorder(s.buffers, s.tasks), "random wire")


def test_random_wire_graph_replay_new_input():
    """The graph of a static network is built once; replaying it after the
    input changes gives the oracle's outputs for the new input."""
    s = sg.random_wire_stream(4, n_nodes=16, stages=2)
    bufs = harness.DeviceBuffers(s.buffers)
    x2 = np.random.default_rng(9).uniform(-1, 1, 256).astype(np.float32)
    with harness.Context(32, mode="graph") as ctx:
        ctx.submit(s.tasks, bufs)
        ctx.flush()
        ctx.sync()
        bufs.t["x"][:1024].copy_(torch.from_numpy(x2.view(np.uint8)))
        ctx.replay()
        ctx.sync()
        st = ctx.stats()
    assert st["launches"] == 2
    s2 = sg.random_wire_stream(4, n_nodes=16, stages=2, x=x2)
    fpcheck.assert_per_element(bufs.download(), execute.run_inorder(s2.buffers, s2.tasks), "graph replay")


# ---- the free-slot variant: W tasks in flight within a ring span M > W --------------------

@pytest.mark.parametrize("W,M", [(1, 8), (4, 16), (8, 32), (16, 64), (32, 64)])
def test_free_slot_variant(W, M):
    """Logged candidates are the oracle's D_M (masks over M - 1 predecessors),
    the ticket log is legal against E, outputs equal the oracle's, and no
    task is inserted while W others are inserted and not retired."""
    s = sg.elementwise_stream(13, n_tasks=200, ranges=True)
    segs = addresses.stream_segments(s.tasks, s.buffers)
    E = deps.full_dag(segs)
    bufs = harness.DeviceBuffers(s.buffers)
    with harness.Context(W, span=M, log=True, trace=True) as ctx:
        ids, packed = harness.pack_tasks(s.tasks, bufs)
        ctx.submit_packed(ids, packed)
        ctx.flush()
        ctx.sync()
        masks, start, retire = ctx.log(0, 0, len(ids))
        tr = ctx.trace(0, 0, len(ids)).astype(np.int64)
    check_log(masks, start, retire, E, deps.window_dag(E, M), M)
    assert_same(bufs.download(), execute.run_inorder(s.buffers, s.tasks), f"free slot W={W} M={M}")
    ins, ret = tr[:, 0], tr[:, 4]
    active = [int(np.sum(ret[:j] > ins[j])) for j in range(len(ids))]
    assert max(active) <= W - 1


def test_trace_timestamps_follow_each_task_through_its_states():
    """Per task: insertion <= publication <= first-CTA start <= last-CTA end
    <= retirement seen, on one device clock."""
    s = sg.elementwise_stream(17, n_tasks=300, ranges=True)
    bufs = harness.DeviceBuffers(s.buffers)
    with harness.Context(8, trace=True) as ctx:
        ids, packed = harness.pack_tasks(s.tasks, bufs)
        ctx.submit_packed(ids, packed)
        ctx.flush()
        ctx.sync()
        tr = ctx.trace(0, 0, len(ids)).astype(np.int64)
    assert (tr > 0).all()
    assert (np.diff(tr, axis=1) >= 0).all()


def test_free_slot_rlsim_emission():
    p = sg.RLParams(n_env=64, steps=5)
    sim = sg.RLSim(6, p)
    bufs = harness.DeviceBuffers(sim.buffers(emit=True))
    with harness.Context(16, span=64, log=True, capacity=1 << 12) as ctx:
        n = harness.RLEmitDriver(sim, bufs, ctx).run()
        masks, start, retire = ctx.log(0, 0, n)
    o_tasks, o_bufs, _ = execute.run_rlsim(sg.RLSim(6, p), emit=True)
    assert n == len(o_tasks)
    E = deps.full_dag(addresses.stream_segments(o_tasks, o_bufs))
    check_log(masks, start, retire, E, deps.window_dag(E, 64), 64)
    assert_same(bufs.download(), o_bufs, "free-slot rl vs oracle")


@pytest.mark.parametrize("every", [1, 5, 16])
def test_flush_splitting_keeps_the_window_dag(every):
    # windows continue across flushes: the logged DAG does not depend on how
    # the stream is cut into launches
    s = sg.elementwise_stream(13, n_tasks=80, ranges=True)
    E, D = oracle_dags(s)
    out, st, (masks, start, retire) = harness.run_stream(s, log=True, flush_every=every)
    check_log(masks, start, retire, E, D, s.window)
    assert st["launches"] == -(-80 // every)
    assert_same(out, execute.run_inorder(s.buffers, s.tasks), f"flush every {every}")


def test_graph_mode_matches_in_order():
    s = sg.elementwise_stream(21, ranges=True)
    out_g, st, _ = harness.run_stream(s, mode="graph")
    assert st["graph_edges"] > 0
    assert_same(out_g, execute.run_inorder(s.buffers, s.tasks), "graph vs oracle")


# ---- the paper's software scheduler (host window, K threads x one CUDA stream) ----------

@pytest.mark.parametrize("seed", [0, 5, 9])
@pytest.mark.parametrize("threads", [1, 4, 8])
def test_sw_scheduler_matches_oracle(seed, threads):
    s = sg.elementwise_stream(seed, n_tasks=120, ranges=True)
    bufs = harness.DeviceBuffers(s.buffers)
    with harness.Context(s.window, mode="sw", sw_threads=threads) as ctx:
        ids, packed = harness.pack_tasks(s.tasks, bufs)
        ctx.submit_packed(ids[:50], packed[:50])
        ctx.flush()
        ctx.submit_packed(ids[50:], packed[50:])
        ctx.flush()
        ctx.sync()
        st = ctx.stats()
    assert st["launches"] == len(s.tasks)
    assert_same(bufs.download(), execute.run_inorder(s.buffers, s.tasks), "sw vs oracle")


def test_sw_scheduler_dnn_and_streams():
    streams = [sg.dnn_stream(40 + i, batch=1 + i, blocks=6) for i in range(3)]
    bufs = [harness.DeviceBuffers(st.buffers) for st in streams]
    with harness.Context(32, mode="sw", n_streams=3, sw_threads=6) as ctx:
        for i, (st, b) in enumerate(zip(streams, bufs)):
            ctx.submit(st.tasks, b, stream=i)
        ctx.flush()
        ctx.sync()
    for st, b in zip(streams, bufs):
        fpcheck.assert_per_element(b.download(), execute.run_inorder(st.buffers, st.tasks), "sw dnn")


def test_sw_scheduler_rlsim_host_driven():
    p = sg.RLParams(n_env=64, steps=4)
    sim = sg.RLSim(4, p)
    bufs = harness.DeviceBuffers(sim.buffers())
    with harness.Context(32, mode="sw", sw_threads=8, capacity=1 << 14) as ctx:
        harness.RLDriver(sim, bufs, ctx).run()
    _, o_bufs, _ = execute.run_rlsim(sg.RLSim(4, p))
    assert_same(bufs.download(), o_bufs, "sw rl vs oracle")


def test_max_ncta_and_wide_tasks():
    s = sg.elementwise_stream(3, n_tasks=40, max_ncta=4)
    for t in s.tasks[::3]:
        t.ncta = 256
    E, D = oracle_dags(s)
    out, _, (masks, start, retire) = harness.run_stream(s, log=True)
    check_log(masks, start, retire, E, D, s.window)
    assert_same(out, execute.run_inorder(s.buffers, s.tasks), "ncta 256")


def test_empty_flush_and_single_task():
    s = sg.elementwise_stream(4, n_tasks=1)
    bufs = harness.DeviceBuffers(s.buffers)
    with harness.Context(8, log=True) as ctx:
        ctx.flush()                       # nothing submitted: a no-op
        ctx.sync()
        ctx.submit(s.tasks, bufs)
        ctx.flush()
        ctx.sync()
        masks, start, retire = ctx.log(0, 0, 1)
        assert masks[0] == 0 and start[0] < retire[0]
    assert_same(bufs.download(), execute.run_inorder(s.buffers, s.tasks), "single task")


# ---- dynamic-DNN streams (window 32) --------------------------------------------

@pytest.mark.parametrize("batch", [1, 2, 4, 8])
def test_dnn_stream_parity(batch):
    s = sg.dnn_stream(batch * 100 + 1, batch=batch)
    E, D = oracle_dags(s)
    out, _, (masks, start, retire) = harness.run_stream(s, log=True)
    check_log(masks, start, retire, E, D, s.window)
    ref_gpu, _, _ = harness.run_stream(s, mode="inorder")
    assert_same(out, ref_gpu, "window vs in-order GPU")
    stats = fpcheck.assert_per_element(out, execute.run_inorder(s.buffers, s.tasks), f"dnn b={batch}")
    print(f"dnn batch {batch}: max relative error {stats['max_rel']:.2e}, "
          f"{100 * stats['share_within_rtol']:.2f} % of elements within 1e-5 of their own magnitude")


@pytest.mark.parametrize("m,k,xoff", [
    (256, 256, 0),     # the k = 256 fast path
    (100, 384, 0),     # the float4 path, three column rounds
    (7, 200, 0),       # the float4 path, a ragged last round; fewer rows than CTAs
    (256, 255, 0),     # the scalar path: k not a multiple of 4
    (64, 256, 1),      # the scalar path: x not 16-byte aligned
])
@pytest.mark.parametrize("ncta", [1, 3, 32])
def test_gemv_task_every_element_within_the_inner_product_bound(m, k, xoff, ncta):
    """One GEMV task through the C ABI: every output element within
    gamma_k sum|w x| + u |w . x| of the exact product (oracle.bounds), on plain
    rows and on rows whose products nearly cancel (so a relative test alone
    could not hold them)."""
    rng = np.random.default_rng(m * 1000 + k * 10 + xoff)
    W = rng.uniform(-1, 1, (m, k)).astype(np.float32)
    x = rng.uniform(-1, 1, k).astype(np.float32)
    h = k // 2
    W[::2, h:2 * h] = -W[::2, :h]                  # even rows: pairs of products that cancel ...
    x[h:2 * h] = x[:h]
    W[::2, 0] *= np.float32(1.0001)                # ... up to a small remainder
    bufs = {"W": W.reshape(-1), "x": np.concatenate([np.zeros(xoff, np.float32), x]),
            "y": np.zeros(m, np.float32)}
    task = sg.Task(0, "gemv", ncta, {"W": sg.Ref("W", 0, m * k), "x": sg.Ref("x", xoff, k), "y": sg.Ref("y", 0, m)},
                   {"m": np.uint32(m), "k": np.uint32(k)})
    s = sg.Stream(bufs, [task], 8)
    out, _, _ = harness.run_stream(s)
    st = fpcheck.check_tasks_on_own_inputs(s.buffers, s.tasks, out)
    assert st["gemv_tasks"] == 1


@pytest.mark.parametrize("batch", [1, 4, 8])
def test_dnn_unrolled_every_task_on_its_own_inputs(batch):
    """The DNN computation with every intermediate kept (streamgen.dnn_stream_unrolled),
    run concurrently with window 32: its DAG and legality against the oracle,
    then every task re-evaluated by the oracle on the GPU's own inputs (each
    GEMV element within the inner-product bound, every other task bit for bit),
    and each sample's last hidden state equal, bit for bit, to what the plain
    DNN stream leaves on the GPU."""
    u = sg.dnn_stream_unrolled(batch * 100 + 1, batch=batch)
    E, D = oracle_dags(u)
    out, _, (masks, start, retire) = harness.run_stream(u, log=True)
    check_log(masks, start, retire, E, D, u.window)
    st = fpcheck.check_tasks_on_own_inputs(u.buffers, u.tasks, out)
    assert st["gemv_tasks"] == sum(t.op == "gemv" for t in u.tasks)
    plain, _, _ = harness.run_stream(sg.dnn_stream(batch * 100 + 1, batch=batch))
    hu = out["h"].reshape(batch, -1, 256)
    hp = plain["h"].reshape(batch, 256)
    for s_ in range(batch):
        assert np.array_equal(hu[s_, u.last_slot[s_]].view(np.uint8), hp[s_].view(np.uint8)), s_


def test_dnn_gemv_is_independent_of_ncta():
    s = sg.dnn_stream(77, batch=2, blocks=6)
    outs = []
    for c in (1, 3, 32, 256):
        for t in s.tasks:
            if t.op == "gemv":
                t.ncta = c
        outs.append(harness.run_stream(s)[0])
    for o in outs[1:]:
        assert_same(outs[0], o, "gemv ncta")


# ---- rigid-sphere stream (input-dependent DAG, window 32) ------------------------------

def _rl_gpu(sim_args, log=True):
    sim = sg.RLSim(*sim_args)
    bufs = harness.DeviceBuffers(sim.buffers())
    with harness.Context(sim.window, log=log, capacity=1 << 16) as ctx:
        plans = harness.RLDriver(sim, bufs, ctx).run(record_plans=True)
        n = sum(len(p.kind) for p in plans)
        lg = ctx.log(0, 0, n) if log else None
        st = ctx.stats()
    return sim, plans, bufs.download(), lg, st


@pytest.mark.parametrize("seed,n_env,steps", [(1, 16, 6), (2, 64, 4), (3, 256, 3)])
def test_rlsim_small_parity(seed, n_env, steps):
    params = sg.RLParams(n_env=n_env, steps=steps)
    sim, plans, out, (masks, start, retire), _ = _rl_gpu((seed, params))
    o_tasks, o_bufs, o_sizes = execute.run_rlsim(sg.RLSim(seed, sg.RLParams(n_env=n_env, steps=steps)))
    assert [len(p.kind) for p in plans] == o_sizes          # same input-dependent stream
    g_tasks = [t for p in plans for t in sim.tasks(p)]
    segs = addresses.stream_segments(o_tasks, o_bufs)
    E = deps.full_dag(segs)
    D = deps.window_dag(E, sim.window)
    assert [(t.op, t.ncta, t.arrays) for t in g_tasks] == [(t.op, t.ncta, t.arrays) for t in o_tasks]
    check_log(masks, start, retire, E, D, sim.window)
    assert_same(out, o_bufs, "rl GPU vs oracle")


# ---- device-side emission: the whole rigid-sphere run in one launch -------------------

def _rl_emit_gpu(seed, params, log=True):
    sim = sg.RLSim(seed, params)
    bufs = harness.DeviceBuffers(sim.buffers(emit=True))
    with harness.Context(sim.window, log=log, capacity=1 << 14) as ctx:
        drv = harness.RLEmitDriver(sim, bufs, ctx)
        n = drv.run()
        lg = ctx.log(0, 0, n) if log else None
        st = ctx.stats()
    return n, bufs.download(), lg, st


@pytest.mark.parametrize("seed,n_env,steps", [(1, 16, 6), (4, 64, 5), (5, 256, 4)])
def test_rlsim_device_emission_small(seed, n_env, steps):
    p = sg.RLParams(n_env=n_env, steps=steps)
    n, out, (masks, start, retire), st = _rl_emit_gpu(seed, p)
    o_tasks, o_bufs, _ = execute.run_rlsim(sg.RLSim(seed, sg.RLParams(n_env=n_env, steps=steps)), emit=True)
    assert n == len(o_tasks)                                  # same input-dependent stream length
    assert st["launches"] == 1 and st["tasks_emitted"] == n - st["tasks_flushed"]
    segs = addresses.stream_segments(o_tasks, o_bufs)
    E = deps.full_dag(segs)
    check_log(masks, start, retire, E, deps.window_dag(E, 32), 32)
    assert_same(out, o_bufs, "device emission vs oracle")
    # the bytes the tasks' segments name: the host counts the submitted tasks,
    # the emitters the appended ones; together, the oracle stream's sum plus,
    # per emit task, its two read-only inputs the oracle's stream leaves out
    # (the 64-byte cfg block and the CTA-count table, one byte per chunk task)
    n_emit = sum(t.op == "rl_emit" for t in o_tasks)
    extra = n_emit * (64 + (steps + 1) * 2 * (n_env // p.chunk))
    assert st["device_seg_bytes"] == sum(z for r, w in segs for _, z in r + w) + extra


def test_rlsim_device_emission_full_size():
    """256 envs x 32 spheres x 50 steps (~15 000 tasks) in one launch: the
    window DAG and outputs equal the oracle's; legality is checked on D_W
    plus in-order release (which covers every longer edge of E)."""
    n, out, (masks, start, retire), st = _rl_emit_gpu(1, sg.RLParams())
    o_tasks, o_bufs, _ = execute.run_rlsim(sg.RLSim(1, sg.RLParams()), emit=True)
    assert n == len(o_tasks)
    segs = addresses.stream_segments(o_tasks, o_bufs)
    D = deps.window_dag_direct(segs, 32)
    assert deps.edges_from_masks([int(m) for m in masks], 32) == D
    s_, r_ = [int(x) for x in start], [int(x) for x in retire]
    assert not deps.check_legal(D, s_, r_)
    assert not deps.check_release_order(s_, r_, 32)
    assert_same(out, o_bufs, "device emission vs oracle, full size")


def test_rlsim_device_emission_matches_host_driven_outputs():
    p = sg.RLParams(n_env=64, steps=8)
    _, out_emit, _, _ = _rl_emit_gpu(7, p, log=False)
    sim = sg.RLSim(7, sg.RLParams(n_env=64, steps=8))
    bufs = harness.DeviceBuffers(sim.buffers(emit=True))
    with harness.Context(32, capacity=1 << 14) as ctx:
        harness.RLDriver(sim, bufs, ctx).run()
    out_host = bufs.download()
    for k in ("pos", "vel", "cont", "nisl"):
        assert np.array_equal(out_emit[k], out_host[k]), k


def test_rlsim_device_emission_repeats_in_one_context():
    p = sg.RLParams(n_env=32, steps=4)
    sim = sg.RLSim(9, p)
    host = sim.buffers(emit=True)
    bufs = harness.DeviceBuffers(host)
    o_tasks, o_bufs, _ = execute.run_rlsim(sg.RLSim(9, sg.RLParams(n_env=32, steps=4)), emit=True)
    with harness.Context(32, capacity=256) as ctx:        # small ring: wraps, emitters wait for space
        drv = harness.RLEmitDriver(sim, bufs, ctx)
        for _ in range(3):
            bufs.upload(host)
            assert drv.run() == len(o_tasks)
            assert_same(bufs.download(), o_bufs, "repeated run")


# ---- dispatch ahead of the window (acs_config.lookahead) ------------------------------------

@pytest.mark.parametrize("W,L", [(1, 0), (1, 5), (8, 0), (8, 1), (8, 8), (8, 56), (16, 16), (32, 32), (33, 31)])
def test_dispatch_ahead_keeps_the_window_dag(W, L):
    """With lookahead L a task is dispatched up to W + L positions past the
    oldest unreleased one, and its workers wait for the W-window themselves: the
    logged masks stay the oracle's D_W, every start is legal against E, and the
    outputs equal the oracle's in-order execution."""
    for seed in (3, 8):
        s = sg.elementwise_stream(seed, n_tasks=300, ranges=True)
        s.window = W
        E, D = oracle_dags(s)
        out, st, (masks, start, retire) = harness.run_stream(s, log=True, lookahead=L)
        check_log(masks, start, retire, E, D, W)
        assert_same(out, execute.run_inorder(s.buffers, s.tasks), f"W={W} L={L} seed={seed}")


def test_dispatch_ahead_rigid_sphere_and_gated_mlp_outputs():
    """The default (lookahead on) and lookahead 0 give the oracle's rigid-sphere
    outputs with device emission, and the same gated-MLP outputs as in-order."""
    p = sg.RLParams(n_env=64, steps=6)
    o_tasks, o_bufs, _ = execute.run_rlsim(sg.RLSim(2, sg.RLParams(n_env=64, steps=6)), emit=True)
    for L in (0, None, 7):
        sim = sg.RLSim(2, p)
        bufs = harness.DeviceBuffers(sim.buffers(emit=True))
        with harness.Context(32, log=True, capacity=1 << 14, lookahead=L) as ctx:
            n = harness.RLEmitDriver(sim, bufs, ctx).run()
            masks, start, retire = ctx.log(0, 0, n)
        assert n == len(o_tasks)
        segs = addresses.stream_segments(o_tasks, o_bufs)
        E = deps.full_dag(segs)
        check_log(masks, start, retire, E, deps.window_dag(E, 32), 32)
        assert_same(bufs.download(), o_bufs, f"rl emission, lookahead {L}")
    d = sg.dnn_stream(6, batch=2, blocks=10, window=32)
    ref, _, _ = harness.run_stream(d, mode="inorder")
    for L in (0, None):
        out, _, _ = harness.run_stream(d, lookahead=L)
        assert_same(out, ref, f"dnn, lookahead {L}")


# ---- without a log the checkers skip retired candidates (windows past 32) ---------------

@pytest.mark.parametrize("W", [33, 48, 64])
def test_unlogged_windows_past_32_match_the_oracle(W):
    """With no log, a checker tests only candidates that had not retired when it
    ran (the rest would be filtered at insertion anyway). The outputs must stay
    the oracle's, bit for bit, for partially overlapping elementwise tasks, for
    the rigid-sphere stream with device emission and for the gated MLP."""
    s = sg.elementwise_stream(13, n_tasks=400, ranges=True)
    s.window = W
    out, _, _ = harness.run_stream(s, log=False)
    assert_same(out, execute.run_inorder(s.buffers, s.tasks), f"elementwise W={W}")
    p = sg.RLParams(n_env=256, steps=8)
    sim = sg.RLSim(3, p)
    bufs = harness.DeviceBuffers(sim.buffers(emit=True))
    with harness.Context(W, capacity=1 << 14) as ctx:
        n = harness.RLEmitDriver(sim, bufs, ctx).run()
    o_tasks, o_bufs, _ = execute.run_rlsim(sg.RLSim(3, sg.RLParams(n_env=256, steps=8)), emit=True)
    assert n == len(o_tasks)
    assert_same(bufs.download(), o_bufs, f"rl emission W={W}")
    d = sg.dnn_stream(5, batch=4, blocks=12, window=W)
    out, _, _ = harness.run_stream(d, log=False)
    ref, _, _ = harness.run_stream(d, mode="inorder")
    assert_same(out, ref, f"dnn W={W} vs in-order GPU")


# ---- restarting a stream's positions (acs_stream_rebase) -------------------------------------

@pytest.mark.parametrize("W,L", [(32, None), (8, None), (33, 0), (64, 0)])
def test_a_restarted_stream_keeps_the_window_dag_and_outputs(W, L):
    """One context runs the same stream from several positions: 0, just below the
    2^31 limit, 0 again and a position that is no multiple of the window, each in
    two flushes (the second launch has only 10 tasks of the stream behind it since
    the restart). Each run finds ring slots, done words and log entries of the
    previous numbering; the logged masks (by slot, seq mod W) decode to the
    oracle's D_W, every start is legal against E and the outputs equal the
    oracle's. Past the limit a submission is refused, and a stream that is not
    idle cannot be restarted."""
    s = sg.elementwise_stream(21, n_tasks=300, ranges=True)
    s.window = W
    E, D = oracle_dags(s)
    ref = execute.run_inorder(s.buffers, s.tasks)
    limit = acs.ACS_MAX_POSITION
    with harness.Context(W, log=True, capacity=1 << 12, lookahead=L) as ctx:
        for pos in (0, limit - 1000, 0, 12345):
            ctx.rebase(0, pos)
            assert ctx.tail(0) == pos
            bufs = harness.DeviceBuffers(s.buffers)
            ids, packed = harness.pack_tasks(s.tasks, bufs)
            # two flushes: the second launch starts with only 10 tasks of the
            # stream behind it since the restart (fewer than its W - 1 candidates)
            for a, b in ((0, 10), (10, len(ids))):
                ctx.submit_packed(ids[a:b], packed[a:b])
                ctx.flush()
                ctx.sync()
            masks, start, retire = ctx.log(0, pos, len(ids))
            rot = [sum(1 << ((b - pos) % W) for b in range(64) if (int(m) >> b) & 1) for m in masks]
            check_log(rot, start, retire, E, D, W)
            assert_same(bufs.download(), ref, f"W={W} L={L} from position {pos}")
        # at the limit: the last two positions below it are taken, the next is refused
        ctx.rebase(0, limit - 2)
        a = harness.pack_tasks(s.tasks[:3], harness.DeviceBuffers(s.buffers))
        ctx.submit_packed(a[0][:2], a[1][:2])
        assert acs.acs_submit_ops(ctx.h, 0, np.array([2], np.uint32), a[1][2:3]) == acs.ACS_ERR_RANGE
        assert acs.acs_stream_rebase(ctx.h, 0, 0) == acs.ACS_ERR_INVALID      # submitted, not synced
        ctx.flush()
        ctx.sync()
        ctx.rebase(0, 0)
        assert ctx.tail(0) == 0


def test_emit_driver_restarts_a_long_stream_between_runs():
    """A rigid-sphere stream placed just below harness.REBASE_AT runs across it;
    before its next run the emit driver restarts the stream's positions at 0
    (acs_stream_rebase). Both runs give the oracle's outputs, and the second
    starts at position 0."""
    p = sg.RLParams(n_env=64, steps=6)
    _, o_bufs, _ = execute.run_rlsim(sg.RLSim(4, sg.RLParams(n_env=64, steps=6)), emit=True)
    with harness.Context(32, capacity=1 << 14) as ctx:
        ctx.rebase(0, harness.REBASE_AT - 200)
        for run in range(2):
            sim = sg.RLSim(4, p)
            bufs = harness.DeviceBuffers(sim.buffers(emit=True))
            drv = harness.RLEmitDriver(sim, bufs, ctx)
            n = drv.run()
            assert n > 200
            if run == 0:
                assert ctx.tail(0) == harness.REBASE_AT - 200 + n   # the first run crossed REBASE_AT
            else:
                assert ctx.tail(0) == n                             # the second started at 0
            assert_same(bufs.download(), o_bufs, f"run {run}")
