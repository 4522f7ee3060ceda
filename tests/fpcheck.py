"""Per-element comparison of GPU outputs with the oracle (shared by the GPU tests).

Elementwise and rigid-sphere bodies round exactly as the oracle does: their
outputs must be bit-identical. A GEMV rounds in the GPU's own order, so:

* ``check_tasks_on_own_inputs``: in a stream that keeps every GEMV output
  (and every input a task reads), every task is re-evaluated by the oracle on
  the GPU's own inputs; each GEMV output element must lie within the inner
  product bound of oracle.bounds of the exact result, and every other task's
  output must match bit for bit.

* ``assert_per_element``: a whole stream's final buffers against the oracle's
  in-order run, element by element, at 1e-5 relative with a cancellation floor:
  |g - o| <= 1e-5 * max(|o|, rms(v)), v the 256-element activation vector the
  element belongs to (one sample's hidden state). Rounding differences of the
  many GEMVs upstream of an element scale with the vectors they were computed
  from, not with the element itself, so an entry that cancels to near zero is
  held to 1e-5 of its vector's RMS instead of its own magnitude.
"""
from __future__ import annotations

from typing import Dict

import numpy as np

from oracle import bounds, execute

RTOL = 1e-5
VEC = 256


def assert_per_element(g: Dict[str, np.ndarray], o: Dict[str, np.ndarray], what: str = "", keys=None,
                       vec: int = VEC, rtol: float = RTOL) -> Dict[str, float]:
    """Every element within rtol * max(|o|, rms of its vec-element vector);
    non-float buffers (and float buffers shorter than one vector) bit for bit.
    Returns the largest plain relative error and the share of elements within
    rtol of their own magnitude, over the float buffers."""
    worst, n_all, n_ok = 0.0, 0, 0
    for k in (keys or o):
        ok_, gk = o[k], g[k]
        if ok_.dtype != np.float32 or ok_.size % vec:
            assert np.array_equal(gk.view(np.uint8), ok_.view(np.uint8)), f"{what}: buffer {k} differs"
            continue
        od = ok_.astype(np.float64).reshape(-1, vec)
        gd = gk.astype(np.float64).reshape(-1, vec)
        rms = np.sqrt(np.mean(od * od, axis=1, keepdims=True))
        err = np.abs(gd - od)
        lim = rtol * np.maximum(np.abs(od), rms)
        bad = np.argwhere(err > lim)
        if bad.size:
            r, c = (int(v) for v in bad[0])
            raise AssertionError(f"{what}: buffer {k}: {len(bad)} of {err.size} elements beyond "
                                 f"{rtol} x max(|o|, vector rms); first at {r * vec + c}: gpu {gd[r, c]!r} "
                                 f"oracle {od[r, c]!r} err {err[r, c]:.3e} limit {lim[r, c]:.3e}")
        rel = err / np.maximum(np.abs(od), 1e-30)
        worst = max(worst, float(np.max(np.where(err > 0, rel, 0.0))))
        n_all += err.size
        n_ok += int(np.count_nonzero(rel <= rtol))
    return {"max_rel": worst, "share_within_rtol": (n_ok / n_all) if n_all else 1.0}


def _view(d, ref):
    return d[ref.buf][ref.off:ref.off + ref.n]


OUT_ROLE = {"gemv": "y", "scale": "y", "axpy": "y", "add": "z", "bias_relu": "t", "resid": "h"}


def check_tasks_on_own_inputs(buffers, tasks, g: Dict[str, np.ndarray]) -> Dict[str, float]:
    """Replay a stream task by task on the oracle, each task evaluated on the
    GPU's own results for its inputs: starting from the initial ``buffers``,
    every task's output range takes the GPU's final value once the task is its
    last writer (``g`` holds the GPU's final buffers). A GEMV must be the last
    writer of its output: each element within bounds.gemv_bound of the exact
    product of the GPU's own W and x. Every other task that is the last writer
    of its range must give the GPU's value bit for bit; one that is not (a copy
    an in-place task then updates) passes the oracle's exact value on, so its
    error would surface at the last writer. Returns the number of GEMV tasks
    checked and the largest error-to-bound ratio among their elements."""
    def span(r):
        return r.buf, r.off, r.off + r.n

    outs = [span(t.arrays[OUT_ROLE[t.op]]) for t in tasks]
    last = [True] * len(tasks)
    for i in range(len(tasks)):
        b, lo, hi = outs[i]
        for j in range(i + 1, len(tasks)):
            b2, lo2, hi2 = outs[j]
            if b2 == b and lo2 < hi and lo < hi2:
                last[i] = False
                break
    cur = {k: v.copy() for k, v in buffers.items()}
    worst, n_gemv = 0.0, 0
    for i, t in enumerate(tasks):
        A, S = t.arrays, t.scalars
        o_ref = A[OUT_ROLE[t.op]]
        if t.op == "gemv":
            assert last[i], f"task {t.task_id}: a GEMV output that a later task overwrites cannot be checked"
            m, k = int(S["m"]), int(S["k"])
            W, x = _view(cur, A["W"]).reshape(m, k), _view(cur, A["x"])
            y = _view(g, o_ref).astype(np.float64)
            o = (W.astype(np.float64) @ x.astype(np.float64)).astype(np.float32).astype(np.float64)
            b = bounds.gemv_bound(W, x)
            err = np.abs(y - o)
            assert np.all(err <= b), (f"task {t.task_id}: {int(np.sum(err > b))} GEMV elements beyond the "
                                      f"bound, worst err/bound {float(np.max(err / b)):.3g}")
            worst = max(worst, float(np.max(err / b)))
            n_gemv += 1
            _view(cur, o_ref)[...] = _view(g, o_ref)
        else:
            execute.run_task(cur, t)                  # the oracle's body on the GPU's inputs
            if last[i]:
                assert np.array_equal(_view(cur, o_ref).view(np.uint8), _view(g, o_ref).view(np.uint8)), \
                    f"task {t.task_id} ({t.op}) differs from the oracle on its own inputs"
    return {"gemv_tasks": n_gemv, "max_err_over_bound": worst}
