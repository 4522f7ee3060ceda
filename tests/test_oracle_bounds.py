"""Pins for oracle/bounds.py, the per-element GEMV error bound the GPU parity
tests apply to every GEMV output. CPU only.

Validity: fp32 evaluations of the same dot products in several orders (the
orders a GPU may use), on plain and on cancelling data, stay inside the bound.
Sensitivity: plausible mistakes (a dropped term, a flipped sign, a transposed
operand) leave it."""
import numpy as np
import pytest

from oracle import bounds

f32 = np.float32


def _seq(W, x):
    """Left-to-right fp32 sum of fp32 products, one rounding per operation."""
    acc = np.zeros(W.shape[0], f32)
    for j in range(W.shape[1]):
        acc = (acc + (W[:, j] * x[j]).astype(f32)).astype(f32)
    return acc


def _fma_lanes(W, x, lanes=32):
    """A warp-style order: lane l sums columns l, l + lanes, ... with fused
    multiply-add (the product unrounded: emulated in fp64, where an fp32
    product is exact), then a butterfly over the lanes."""
    m, k = W.shape
    part = np.zeros((m, lanes), f32)
    for c0 in range(0, k, lanes):
        for l in range(min(lanes, k - c0)):
            c = c0 + l
            part[:, l] = (W[:, c].astype(np.float64) * float(x[c]) + part[:, l].astype(np.float64)).astype(f32)
    off = lanes // 2
    while off:
        part = (part + np.roll(part, -off, axis=1)).astype(f32)
        off //= 2
    return part[:, 0]


def _pairwise(W, x):
    return np.sum((W * x[None, :]).astype(f32), axis=1, dtype=f32)


def _cancelling(rng, m, k):
    """Rows whose products nearly cancel: y is tiny next to sum |w x|."""
    W = rng.uniform(-1, 1, (m, k)).astype(f32)
    x = rng.uniform(-1, 1, k).astype(f32)
    h = k // 2
    W[:, h:2 * h] = -W[:, :h] * (1 + rng.uniform(-1e-4, 1e-4, (m, 1))).astype(f32)
    x[h:2 * h] = x[:h]
    return W, x


def test_gamma_matches_its_definition():
    assert bounds.gamma(1) == pytest.approx(2.0 ** -24 / (1 - 2.0 ** -24), rel=1e-15)
    assert bounds.gamma(256) == pytest.approx(256 * 2.0 ** -24 / (1 - 256 * 2.0 ** -24), rel=1e-15)


@pytest.mark.parametrize("k", [7, 33, 256, 384])
@pytest.mark.parametrize("kind", ["uniform", "cancelling"])
def test_gemv_bound_holds_for_every_evaluation_order(k, kind):
    rng = np.random.default_rng(k)
    m = 64
    if kind == "uniform":
        W = rng.uniform(-1, 1, (m, k)).astype(f32)
        x = rng.uniform(-1, 1, k).astype(f32)
    else:
        W, x = _cancelling(rng, m, k)
    o = (W.astype(np.float64) @ x.astype(np.float64)).astype(f32)       # the oracle's GEMV
    b = bounds.gemv_bound(W, x)
    for f in (_seq, _fma_lanes, _pairwise, lambda W, x: _seq(W[:, ::-1], x[::-1])):
        g = f(W, x)
        assert np.all(np.abs(g.astype(np.float64) - o) <= b)
    # and the bound is not vacuous: far below the magnitude of the sum of |w x|
    assert np.all(b <= 1e-4 * (np.abs(W.astype(np.float64)) @ np.abs(x.astype(np.float64))) + 1e-30)


def test_gemv_bound_catches_dropped_and_flipped_terms():
    rng = np.random.default_rng(5)
    W = rng.uniform(-1, 1, (256, 256)).astype(f32)
    x = rng.uniform(-1, 1, 256).astype(f32)
    o = (W.astype(np.float64) @ x.astype(np.float64)).astype(f32)
    b = bounds.gemv_bound(W, x)
    dropped = _seq(W[:, 1:], x[1:])                                      # term 0 missing
    assert np.mean(np.abs(dropped.astype(np.float64) - o) > b) > 0.9
    flipped = _seq(W, np.concatenate([-x[:1], x[1:]]))                   # sign of one term
    assert np.mean(np.abs(flipped.astype(np.float64) - o) > b) > 0.9
    transposed = _seq(W.T.copy(), x)                                     # wrong operand layout
    assert np.all(np.abs(transposed.astype(np.float64) - o) > b)
