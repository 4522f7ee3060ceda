"""C-ABI behaviour on the GPU: argument validation, sticky errors, bounded
waits that end in ACS_ERR_TIMEOUT with the device still usable, explicit
segments including the whole-memory segment, and independent streams."""
import ctypes as C
import time

import numpy as np
import pytest
import torch

import streamgen as sg
from oracle import addresses, deps, execute

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2401_12377_b300 import build
    build.build()
    from paper_2401_12377_b300 import acs, harness


def _nop_args(ncta=1):
    a = acs.acs_args()
    a.op = acs.OPS["nop"]
    a.ncta = ncta
    return a


def test_submit_validation():
    with harness.Context(8) as ctx:
        h = ctx.h
        a = _nop_args()
        seg = [(4096, 16)]
        assert acs.acs_submit(h, 1, a, seg, seg) == acs.ACS_OK
        assert acs.acs_submit(h, 1, a, seg, seg) == acs.ACS_ERR_ORDER       # not increasing
        assert acs.acs_submit(h, 0, a, seg, seg) == acs.ACS_ERR_ORDER
        assert acs.acs_submit(h, 2, a, [(4096, 16)] * 17, []) == acs.ACS_ERR_INVALID   # > 16 segments
        assert acs.acs_submit(h, 2, a, [(4096, 0)] * 20, []) == acs.ACS_OK             # empty ones dropped
        assert acs.acs_submit(h, 3, a, [((1 << 64) - 8, 16)], []) == acs.ACS_ERR_INVALID  # wraps 2^64
        assert acs.acs_submit(h, 3, a, [((1 << 64) - 16, 16)], []) == acs.ACS_OK          # ends at 2^64
        assert acs.acs_submit(h, 4, a, [acs.ACS_WHOLE_MEMORY], []) == acs.ACS_OK
        bad = _nop_args(0)
        assert acs.acs_submit(h, 5, bad, [], []) == acs.ACS_ERR_INVALID
        bad = _nop_args(257)
        assert acs.acs_submit(h, 5, bad, [], []) == acs.ACS_ERR_INVALID
        bad = _nop_args(); bad.op = 99
        assert acs.acs_submit(h, 5, bad, [], []) == acs.ACS_ERR_INVALID
        assert acs.acs_submit_stream(h, 1, 5, a, [], []) == acs.ACS_ERR_INVALID   # only stream 0
        ctx.flush()
        ctx.sync()


def test_ring_full_until_sync():
    with harness.Context(8, capacity=64) as ctx:
        a = _nop_args()
        n = 0
        while acs.acs_submit(ctx.h, n, a, [], [(4096, 4)]) == acs.ACS_OK:
            n += 1
            assert n < 64
        assert acs.acs_submit(ctx.h, n, a, [], [(4096, 4)]) == acs.ACS_ERR_FULL
        ctx.flush()
        ctx.sync()
        assert acs.acs_submit(ctx.h, n, a, [], [(4096, 4)]) == acs.ACS_OK       # room again
        ctx.flush()
        ctx.sync()


def test_timeout_is_bounded_sticky_and_leaves_the_device_usable():
    flag = torch.zeros(4, dtype=torch.int32, device="cuda")
    with harness.Context(8, timeout_s=0.2) as ctx:
        row = harness._args_row("wait_flag", 1, {"flag": flag.data_ptr(), "limit_ns": 3_000_000_000})
        ctx.submit_packed(np.array([0], np.uint32), row)
        t0 = time.time()
        ctx.flush()
        code = ctx.sync_code()
        dt = time.time() - t0
        assert code == acs.ACS_ERR_TIMEOUT, acs.acs_strerror(code)
        assert dt < 2.5
        assert acs.acs_error(ctx.h) == acs.ACS_ERR_TIMEOUT                  # sticky
        assert acs.acs_submit(ctx.h, 1, _nop_args(), [], []) == acs.ACS_ERR_TIMEOUT
    # the device is healthy: a fresh context runs a stream correctly
    s = sg.elementwise_stream(1, n_tasks=16)
    out, _, _ = harness.run_stream(s)
    ref = execute.run_inorder(s.buffers, s.tasks)
    assert all(np.array_equal(out[k], ref[k]) for k in ref)


def test_wait_flag_released_by_the_host_completes():
    flag = torch.zeros(4, dtype=torch.int32, device="cuda")
    with harness.Context(8, timeout_s=5) as ctx:
        row = harness._args_row("wait_flag", 1, {"flag": flag.data_ptr(), "limit_ns": 3_000_000_000})
        ctx.submit_packed(np.array([0], np.uint32), row)
        ctx.flush()
        side = torch.cuda.Stream()
        time.sleep(0.05)
        with torch.cuda.stream(side):
            flag.fill_(1)
        ctx.sync()


def _explicit_stream(seed):
    """Elementwise tasks plus NOP tasks with hand-given segments, including the
    whole-memory segment (indirect access, Sec. IV-A)."""
    s = sg.elementwise_stream(seed, n_tasks=40)
    return s


def test_whole_memory_segment_orders_everything():
    s = sg.elementwise_stream(31, n_tasks=30)
    bufs = harness.DeviceBuffers(s.buffers)
    ids, packed = harness.pack_tasks(s.tasks, bufs)
    W = 8
    wild_at = {7: "read", 15: "write"}
    # oracle segments with the wildcard tasks inserted
    lay = addresses.Layout(s.buffers)
    segs, n = [], 0
    with harness.Context(W, log=True) as ctx:
        tid = 0
        for i in range(len(ids)):
            if i in wild_at:
                kind = wild_at[i]
                rd = [deps.WHOLE_MEMORY] if kind == "read" else []
                wr = [deps.WHOLE_MEMORY] if kind == "write" else []
                segs.append((rd, wr))
                rc = acs.acs_submit(ctx.h, tid, _nop_args(), [acs.ACS_WHOLE_MEMORY] if rd else [],
                                    [acs.ACS_WHOLE_MEMORY] if wr else [])
                assert rc == acs.ACS_OK
                tid += 1
            segs.append(addresses.task_segments(s.tasks[i], lay))
            ctx.submit_packed(np.array([tid], np.uint32), packed[i:i + 1])
            tid += 1
        ctx.flush()
        ctx.sync()
        masks, start, retire = ctx.log(0, 0, tid)
    E = deps.full_dag(segs)
    D = deps.window_dag(E, W)
    assert deps.edges_from_masks([int(m) for m in masks], W) == D
    assert not deps.check_legal(E, [int(x) for x in start], [int(x) for x in retire])
    out = bufs.download()
    ref = execute.run_inorder(s.buffers, s.tasks)
    assert all(np.array_equal(out[k], ref[k]) for k in ref)


@pytest.mark.parametrize("lookahead", [None, 0, 8])
def test_independent_streams_in_one_launch(lookahead):
    """Five streams in one launch; with several streams the default dispatches
    without lookahead, and an explicit one applies to every stream."""
    streams = [sg.elementwise_stream(50 + i, n_tasks=20 + 13 * i, ranges=bool(i % 2)) for i in range(5)]
    bufs = [harness.DeviceBuffers(s.buffers) for s in streams]
    with harness.Context(8, n_streams=5, log=True, lookahead=lookahead) as ctx:
        for i, s in enumerate(streams):
            ctx.submit(s.tasks, bufs[i], stream=i)
        ctx.flush()
        ctx.sync()
        for i, s in enumerate(streams):
            segs = addresses.stream_segments(s.tasks, s.buffers)
            E = deps.full_dag(segs)
            masks, start, retire = ctx.log(i, 0, len(s.tasks))
            assert deps.edges_from_masks([int(m) for m in masks], 8) == deps.window_dag(E, 8)
            assert not deps.check_legal(E, [int(x) for x in start], [int(x) for x in retire])
            ref = execute.run_inorder(s.buffers, s.tasks)
            out = bufs[i].download()
            assert all(np.array_equal(out[k], ref[k]) for k in ref)
        assert ctx.stats()["launches"] == 1


@pytest.mark.parametrize("W", [8, 32, 64])
def test_tasks_with_many_segments(W):
    """NOP tasks with 1 to 16 segments each over a small address range, so
    that many pairs conflict: tasks with up to 4 segments on both sides take
    the checker's register path, the others its all-pairs path. Logged masks
    equal the oracle's D_W and the start/retire log is legal against E."""
    rng = np.random.default_rng(1234 + W)
    base = 1 << 20
    segs = []
    for _ in range(300):
        nr = int(rng.integers(0, 9))
        nw = int(rng.integers(0 if nr else 1, 9))
        def one():
            size = int(rng.integers(0, 513)) if rng.random() < 0.95 else 0
            return (base + int(rng.integers(0, 1 << 16)), size)
        segs.append(([one() for _ in range(nr)], [one() for _ in range(nw)]))
    with harness.Context(W, log=True) as ctx:
        for tid, (rd, wr) in enumerate(segs):
            assert acs.acs_submit(ctx.h, tid, _nop_args(1 + tid % 3), rd, wr) == acs.ACS_OK
        ctx.flush()
        ctx.sync()
        masks, start, retire = ctx.log(0, 0, len(segs))
    E = deps.full_dag(segs)
    assert deps.edges_from_masks([int(m) for m in masks], W) == deps.window_dag(E, W)
    assert not deps.check_legal(E, [int(x) for x in start], [int(x) for x in retire])
    assert sum(1 for rd, wr in segs if len(rd) + len(wr) > 4) > 100


def test_emit_task_with_a_zero_cta_count_fails_invalid_and_leaves_the_device_usable():
    """An emit task copies chunk CTA counts from its table into the tasks it
    appends; a 0 there would leave a task unrun. The device checks the entries
    before appending anything: the launch ends with ACS_ERR_INVALID from
    acs_sync, and a fresh context then runs the same stream to the oracle's
    result."""
    p = sg.RLParams(n_env=64, steps=5)
    sim = sg.RLSim(11, p)
    bufs = harness.DeviceBuffers(sim.buffers(emit=True))
    n_chunks = p.n_env // p.chunk
    with harness.Context(32, capacity=1 << 12, timeout_s=2) as ctx:
        drv = harness.RLEmitDriver(sim, bufs, ctx)      # the host check passes the table ...
        drv.table[(2 * 2 + 1) * n_chunks + 3] = 0       # ... then step 2's integrate, chunk 3, is spoilt
        drv.submit()
        ctx.flush()
        code = ctx.sync_code()
        assert code == acs.ACS_ERR_INVALID, acs.acs_strerror(code)
        assert acs.acs_error(ctx.h) == acs.ACS_ERR_INVALID               # sticky
    sim = sg.RLSim(11, p)
    bufs = harness.DeviceBuffers(sim.buffers(emit=True))
    with harness.Context(32, capacity=1 << 12) as ctx:
        n = harness.RLEmitDriver(sim, bufs, ctx).run()
    o_tasks, o_bufs, _ = execute.run_rlsim(sg.RLSim(11, sg.RLParams(n_env=64, steps=5)), emit=True)
    assert n == len(o_tasks)
    out = bufs.download()
    for k in ("pos", "vel", "cont", "nisl"):
        assert np.array_equal(out[k], o_bufs[k]), k


def test_host_abort_mid_stream_stops_cleanly_and_leaves_the_device_usable():
    """acs_abort while a launch runs: elementwise tasks, then a task waiting on
    a flag nothing sets, then more tasks. The launch ends well before any wait
    limit, acs_sync returns ACS_ERR_STOPPED (sticky), and a fresh context then
    runs a stream to the oracle's result."""
    flag = torch.zeros(4, dtype=torch.int32, device="cuda")
    s = sg.elementwise_stream(21, n_tasks=24)
    bufs = harness.DeviceBuffers(s.buffers)
    ids, packed = harness.pack_tasks(s.tasks, bufs)
    wait = harness._args_row("wait_flag", 1, {"flag": flag.data_ptr(), "limit_ns": 4_000_000_000})
    with harness.Context(8, timeout_s=5) as ctx:
        ctx.submit_packed(ids[:12], packed[:12])
        ctx.submit_packed(np.array([12], np.uint32), wait)
        ctx.submit_packed(ids[12:] + np.uint32(1), packed[12:])
        ctx.flush()
        time.sleep(0.05)                                  # the launch is blocked on the waiting task
        t0 = time.time()
        assert acs.acs_abort(ctx.h) == acs.ACS_OK
        code = ctx.sync_code()
        dt = time.time() - t0
        assert code == acs.ACS_ERR_STOPPED, acs.acs_strerror(code)
        assert dt < 1.0, dt
        assert acs.acs_error(ctx.h) == acs.ACS_ERR_STOPPED
        assert acs.acs_submit(ctx.h, 100, _nop_args(), [], []) == acs.ACS_ERR_STOPPED
        assert acs.acs_flush(ctx.h) == acs.ACS_ERR_STOPPED
    s2 = sg.elementwise_stream(22, n_tasks=32)
    out, _, _ = harness.run_stream(s2)
    ref = execute.run_inorder(s2.buffers, s2.tasks)
    assert all(np.array_equal(out[k], ref[k]) for k in ref)


def test_a_smaller_context_does_not_break_a_larger_one():
    """The persistent kernel's shared-memory limit is per-function state of the
    process: creating a context that needs less (a smaller window) after one
    that needs more (window 32 dispatching ahead, 64 slots) must leave the
    first one launchable."""
    s = sg.elementwise_stream(21, n_tasks=120, ranges=True)
    bufs = harness.DeviceBuffers(s.buffers)
    with harness.Context(32, log=False) as big:
        with harness.Context(4, log=False, lookahead=0) as small:
            small.submit(s.tasks[:10], bufs)
            small.flush()
            small.sync()
        bufs2 = harness.DeviceBuffers(s.buffers)
        big.submit(s.tasks, bufs2)
        big.flush()
        big.sync()
        ref = execute.run_inorder(s.buffers, s.tasks)
        out = bufs2.download()
        assert all(np.array_equal(out[k], ref[k]) for k in ref)


def test_default_lookahead_reaches_window_mode_contexts_only(monkeypatch):
    """A process-wide default lookahead (bench.py --lookahead) applies to
    window-mode contexts without a free-slot span; the host-scheduler,
    in-order and graph modes and span contexts, which take none, still open."""
    monkeypatch.setattr(harness, "DEFAULT_LOOKAHEAD", 8)
    for mode in ("window", "inorder", "graph", "sw"):
        with harness.Context(8, mode=mode) as ctx:
            assert ctx.mode == mode
    with harness.Context(8, span=32) as ctx:
        assert ctx.span == 32
    # an explicit lookahead on a mode that takes none is still refused
    with pytest.raises(acs.AcsError):
        harness.Context(8, mode="sw", lookahead=8)
