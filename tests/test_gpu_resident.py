"""Resident launches (acs_start / acs_flush / acs_progress / acs_stop): the
scheduler kernel stays on the device while the host publishes work through
mapped memory. Per stream the logged DAG equals the oracle's window DAG, the
legality log passes, and outputs equal the oracle's; work published in pieces,
to several streams at different times, with device-side emission, and after
an emitter chain finished; the idle limit ends an abandoned kernel. GPU only."""
import time

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



def _check(ctx, stream, first, tasks, buffers, W):
    """Tasks at stream positions first .. first + n - 1, sharing no bytes with
    the tasks before them: their logged DAG and legality against the oracle's.
    Window slots are position mod W, so the masks decode at their positions."""
    segs = addresses.stream_segments(tasks, buffers)
    E = deps.full_dag(segs)
    masks, start, retire = ctx.log(stream, first, len(tasks))
    got = deps.edges_from_masks([0] * first + [int(x) for x in masks], W)
    assert all(i >= first for i, _ in got), "edge to a task of an earlier request"
    assert {(i - first, j - first) for i, j in got} == deps.window_dag(E, W)
    assert not deps.check_legal(E, [int(x) for x in start], [int(x) for x in retire])


def _same(g, o):
    for k in o:
        assert np.array_equal(g[k].view(np.uint8), o[k].view(np.uint8)), k


def _close(g, o):
    fpcheck.assert_per_element(g, o, "resident")


@pytest.mark.parametrize("W", [4, 8, 32])
def test_resident_pieces_match_oracle(W):
    s = sg.elementwise_stream(21, n_tasks=400, ranges=True, window=W)
    bufs = harness.DeviceBuffers(s.buffers)
    torch.cuda.current_stream().synchronize()
    with harness.Context(W, log=True, resident=True, capacity=1 << 10) as ctx:
        cuts = [0, 1, 9, 60, 61, 200, 333, 400]
        for a, b in zip(cuts, cuts[1:]):
            ctx.submit(s.tasks[a:b], bufs)
            ctx.flush()
            if a == 61:
                time.sleep(0.01)          # let the stream go idle in between
        ctx.sync()
        head, idle = ctx.progress()
        assert int(idle[0]) == len(s.tasks) and int(head[0]) == len(s.tasks)
        _check(ctx, 0, 0, s.tasks, s.buffers, W)
        out = bufs.download()
        ctx.stop()
        assert ctx.stats()["launches"] == 1
    _same(out, execute.run_inorder(s.buffers, s.tasks))


def test_resident_streams_arrive_at_different_times():
    """DNN streams published to four slots at staggered times while earlier
    ones run; then a second request in each slot after the first completed."""
    specs = [(31 + i, 1 + i % 3, 6 + 3 * i) for i in range(4)]
    W = 16
    streams = [sg.dnn_stream(seed, batch=b, blocks=k) for seed, b, k in specs]
    bufs = [harness.DeviceBuffers(st.buffers) for st in streams]
    torch.cuda.current_stream().synchronize()
    with harness.Context(W, n_streams=4, log=True, resident=True, capacity=1 << 11) as ctx:
        for rnd in range(2):
            starts = []
            for i, st in enumerate(streams):
                if rnd:
                    bufs[i].upload(st.buffers)
                    torch.cuda.current_stream().synchronize()
                t0 = ctx.tail(i)
                starts.append(t0)
                ids, packed = harness.pack_tasks(st.tasks, bufs[i])
                ctx.submit_packed(ids + np.uint32(t0), packed, stream=i)
                ctx.flush()
                time.sleep(0.002 * i)
            ctx.sync()
            for i, st in enumerate(streams):
                assert ctx.tail(i) == starts[i] + len(st.tasks)
                _close(bufs[i].download(), execute.run_inorder(st.buffers, st.tasks))
        # the second request reused the first one's buffers: the window saw
        # both as one stream of twice the tasks
        for i, st in enumerate(streams):
            _check(ctx, i, 0, st.tasks + st.tasks, st.buffers, W)
        ctx.stop()
        assert ctx.stats()["launches"] == 1


def test_resident_emission_then_next_request():
    """A rigid-sphere request with device-side emission in a resident kernel:
    the host learns the emitted end from acs_progress; the stream then takes a
    DNN request after it."""
    p = sg.RLParams(n_env=64, steps=6)
    sim = sg.RLSim(5, p)
    host = sim.buffers(emit=True)
    bufs = harness.DeviceBuffers(host)
    o_tasks, o_bufs, _ = execute.run_rlsim(sg.RLSim(5, p), emit=True)
    dnn = sg.dnn_stream(77, batch=2, blocks=8)
    dbufs = harness.DeviceBuffers(dnn.buffers)
    torch.cuda.current_stream().synchronize()
    W = 32
    with harness.Context(W, log=True, resident=True, capacity=1 << 12) as ctx:
        drv = harness.RLEmitDriver(sim, bufs, ctx)
        start = drv.submit()
        n_first = p.n_env // p.chunk + 1          # broadphase of step 0 + the first emit task
        assert ctx.tail(0) == start + n_first
        ctx.flush()
        # poll until the emitter chain finished and everything retired: the
        # tail then moves to the emitted end
        t_end = time.time() + 10
        while True:
            head, idle = ctx.progress()
            if ctx.tail(0) != start + n_first:
                assert ctx.tail(0) == int(idle[0])
                break
            assert time.time() < t_end
            time.sleep(0.001)
        n = ctx.tail(0) - start
        assert n == len(o_tasks)
        _check(ctx, 0, start, o_tasks, o_bufs, W)
        _same(bufs.download(), o_bufs)
        t0 = ctx.tail(0)
        ids, packed = harness.pack_tasks(dnn.tasks, dbufs)
        ctx.submit_packed(ids + np.uint32(t0), packed)
        ctx.flush()
        ctx.sync()
        assert ctx.tail(0) == t0 + len(dnn.tasks)
        _close(dbufs.download(), execute.run_inorder(dnn.buffers, dnn.tasks))
        st = ctx.stats()
        ctx.stop()
    assert st["tasks_emitted"] == len(o_tasks) - n_first


def test_resident_ring_full_and_retry():
    """A small ring: submission reports ACS_ERR_FULL until the device has
    released enough tasks; progress polling frees the space."""
    s = sg.elementwise_stream(8, n_tasks=300, ranges=True, window=8)
    bufs = harness.DeviceBuffers(s.buffers)
    torch.cuda.current_stream().synchronize()
    with harness.Context(8, resident=True, capacity=64) as ctx:
        ids, packed = harness.pack_tasks(s.tasks, bufs)
        i = fulls = 0
        t_end = time.time() + 10
        while i < len(ids):
            rc = acs.load().acs_submit_ops(ctx.h, 0, 1, ids[i:i + 1].ctypes.data, packed[i:i + 1].ctypes.data)
            if rc == acs.ACS_ERR_FULL:
                fulls += 1
                ctx.flush()
                ctx.progress()
                assert time.time() < t_end
                continue
            assert rc == acs.ACS_OK
            i += 1
        ctx.flush()
        ctx.sync()
        out = bufs.download()
        ctx.stop()
    assert fulls > 0
    _same(out, execute.run_inorder(s.buffers, s.tasks))


def test_resident_then_ordinary_flush():
    s = sg.elementwise_stream(3, n_tasks=64)
    bufs = harness.DeviceBuffers(s.buffers)
    torch.cuda.current_stream().synchronize()
    with harness.Context(8, log=True, resident=True) as ctx:
        ctx.submit(s.tasks[:30], bufs)
        ctx.stop()                       # publishes the staged tasks and drains
        ctx.submit(s.tasks[30:], bufs)   # now an ordinary launch
        ctx.flush()
        ctx.sync()
        _check(ctx, 0, 0, s.tasks, s.buffers, 8)
        out = bufs.download()
        assert ctx.stats()["launches"] == 2
    _same(out, execute.run_inorder(s.buffers, s.tasks))


def test_resident_idle_limit_ends_the_kernel():
    """With no host call for longer than idle_limit_ms the kernel leaves by
    itself; the context then reports ACS_ERR_STOPPED and the device stays
    usable."""
    s = sg.elementwise_stream(4, n_tasks=16)
    bufs = harness.DeviceBuffers(s.buffers)
    torch.cuda.current_stream().synchronize()
    ctx = harness.Context(8, resident=True, idle_limit_ms=200)
    time.sleep(1.0)
    ctx.submit(s.tasks, bufs)
    with pytest.raises(acs.AcsError) as e:
        ctx.flush()
    assert e.value.code == acs.ACS_ERR_STOPPED
    ctx.close()
    out, _, _ = harness.run_stream(s)
    _same(out, execute.run_inorder(s.buffers, s.tasks))
