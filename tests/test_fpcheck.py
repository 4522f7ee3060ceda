"""The per-element checkers the GPU parity tests use (tests/fpcheck.py), run on
the CPU against a stand-in for the GPU: the same streams with their GEMVs
evaluated in a warp-like fp32 order. The stand-in passes; planted mistakes
(a dropped product, a skipped bias, one wrong element) fail. CPU only."""
import numpy as np
import pytest

import streamgen as sg
from oracle import execute

import fpcheck

f32 = np.float32


def _warp_gemv(W, x, lanes=32):
    """Lane l sums columns l, l + 32, ... with fused multiply-add (exact product,
    one rounding: emulated in fp64), then a butterfly over the lanes."""
    m, k = W.shape
    part = np.zeros((m, lanes), f32)
    for c in range(k):
        l = c % lanes
        part[:, l] = (W[:, c].astype(np.float64) * float(x[c]) + part[:, l].astype(np.float64)).astype(f32)
    off = lanes // 2
    while off:
        part = (part + np.roll(part, -off, axis=1)).astype(f32)
        off //= 2
    return part[:, 0]


def _run(stream, gemv=_warp_gemv, drop_bias_at=None):
    bufs = {k: v.copy() for k, v in stream.buffers.items()}
    n_bias = 0
    for t in stream.tasks:
        if t.op == "gemv":
            A, S = t.arrays, t.scalars
            m, k = int(S["m"]), int(S["k"])
            W = bufs[A["W"].buf][A["W"].off:A["W"].off + m * k].reshape(m, k)
            x = bufs[A["x"].buf][A["x"].off:A["x"].off + k]
            bufs[A["y"].buf][A["y"].off:A["y"].off + m] = gemv(W, x)
        elif t.op == "bias_relu" and n_bias == drop_bias_at:
            n_bias += 1
            r = t.arrays["t"]
            v = bufs[r.buf][r.off:r.off + r.n]
            v[...] = np.where(v > 0, v, f32(0))             # ReLU without the bias
        else:
            n_bias += t.op == "bias_relu"
            execute.run_task(bufs, t)
    return bufs


def test_replay_accepts_a_warp_order_gemv_and_rejects_mistakes():
    u = sg.dnn_stream_unrolled(5, batch=2, blocks=8)
    g = _run(u)
    st = fpcheck.check_tasks_on_own_inputs(u.buffers, u.tasks, g)
    assert st["gemv_tasks"] == sum(t.op == "gemv" for t in u.tasks) and st["max_err_over_bound"] < 1
    dropped = _run(u, gemv=lambda W, x: _warp_gemv(W[:, 1:], x[1:]))
    with pytest.raises(AssertionError, match="GEMV elements beyond the bound"):
        fpcheck.check_tasks_on_own_inputs(u.buffers, u.tasks, dropped)
    skipped = _run(u, drop_bias_at=3)
    with pytest.raises(AssertionError, match="differs from the oracle on its own inputs"):
        fpcheck.check_tasks_on_own_inputs(u.buffers, u.tasks, skipped)


@pytest.mark.parametrize("batch", [1, 4, 8])
def test_per_element_check_accepts_a_warp_order_gemv(batch):
    s = sg.dnn_stream(batch * 100 + 1, batch=batch)
    st = fpcheck.assert_per_element(_run(s), execute.run_inorder(s.buffers, s.tasks), "cpu stand-in")
    assert st["share_within_rtol"] > 0.95


def test_per_element_check_rejects_one_wrong_element():
    s = sg.dnn_stream(3, batch=2)
    o = execute.run_inorder(s.buffers, s.tasks)
    g = _run(s)
    rms = float(np.sqrt(np.mean(o["h"][:256].astype(np.float64) ** 2)))
    i = int(np.argmin(np.abs(o["h"][:256])))               # the entry nearest zero
    bad = {k: v.copy() for k, v in g.items()}
    bad["h"][i] = f32(float(o["h"][i]) + 3e-5 * rms)        # 3x the floor: caught
    with pytest.raises(AssertionError, match="beyond"):
        fpcheck.assert_per_element(bad, o)
    j = int(np.argmax(np.abs(o["h"][:256])))               # the largest entry
    bad = {k: v.copy() for k, v in g.items()}
    bad["h"][j] = f32(float(o["h"][j]) * (1 + 3e-5))        # 3e-5 relative: caught
    with pytest.raises(AssertionError, match="beyond"):
        fpcheck.assert_per_element(bad, o)


def test_per_element_check_wants_exact_bits_for_integer_buffers():
    o = {"n": np.arange(8, dtype=np.uint32)}
    g = {"n": o["n"].copy()}
    fpcheck.assert_per_element(g, o)
    g["n"][3] += 1
    with pytest.raises(AssertionError):
        fpcheck.assert_per_element(g, o)
