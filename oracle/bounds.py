"""A-priori error bound between a GPU GEMV and the oracle's (test infrastructure only).

The oracle's GEMV is the exact dot product rounded once to fp32 (execute.py).
A GPU evaluates the same dot product in fp32 in some fixed order of its own, so
its result differs by accumulated rounding. The standard forward error bound
for a floating-point inner product, valid for every evaluation order and with
or without fused multiply-add (Higham, "Accuracy and Stability of Numerical
Algorithms", 2nd ed., Sec. 3.1, Eq. 3.5), is

    |fl(w . x) - w . x| <= gamma_k * sum_j |w_j x_j|,   gamma_k = k u / (1 - k u),

u = 2^-24 the unit roundoff of fp32 round-to-nearest. ``gemv_bound`` adds the
oracle's own rounding (u |w . x|), element by element. The GPU parity tests
apply it to every output element of a GEMV task, computed from that task's own
inputs.

Underflow adds at most 2^-149 per rounding (k + 2 such terms per element), and
the bound's fp64 sums are scaled by (1 + 2^-40) to cover their own rounding.
"""
from __future__ import annotations

import numpy as np

U = 2.0 ** -24            # unit roundoff, fp32 round-to-nearest
ETA = 2.0 ** -149         # smallest fp32 subnormal: the absolute error of an underflowing rounding
SAFE = 1.0 + 2.0 ** -40   # covers the fp64 rounding of the bound's own sums


def gamma(k: int) -> float:
    """gamma_k = k u / (1 - k u) (Higham, Lemma 3.1)."""
    return k * U / (1.0 - k * U)


def gemv_bound(W: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Per-element bound on |y_gpu - y_oracle| for y = W x (W: m x k, row-major),
    both sides given the same W and x: y_oracle = fl(W x) (exact, rounded once),
    y_gpu any fp32 evaluation of W x:

      |y_g - y_o| <= gamma_k |W| |x|   (the GPU's rounding, Eq. 3.5)
                   + u |W x|           (the oracle's one rounding)
    """
    m, k = W.shape
    Wd, xd = W.astype(np.float64), x.astype(np.float64)
    b = gamma(k) * (np.abs(Wd) @ np.abs(xd)) + U * np.abs(Wd @ xd) + (k + 2) * ETA
    return b * SAFE
