"""In-order CPU executor of task streams (test infrastructure only).

The method is correct when concurrent issue reproduces the memory state of
running the stream one task at a time in program order: every conflicting pair
keeps its order (Sec. III-C: a kernel becomes ready only after its upstream
kernels complete) and non-conflicting tasks touch disjoint bytes. This module is
that in-order execution, one task after another, on numpy buffers.

Arithmetic is single precision with one rounding per operation (numpy float32
elementwise operations never contract into FMA). The one exception is the GEMV
of the dynamic-DNN stream, whose oracle value is the exact dot product rounded
once to fp32 (computed in fp64, where fp32 products are exact); the GPU's fp32
reduction differs from it by accumulated rounding, bounded in the tests.

The rigid-sphere bodies run in ``rlsim.c`` (compiled on first use with
``-ffp-contract=off``).

Parity: elementwise bodies and the GEMV are pinned against closed forms with
exactly representable data (tests/test_oracle_bodies.py); the stream executor is
pinned by schedule independence: executing any topological order of the
oracle's DAG E reproduces the in-order result bit for bit.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Dict, List

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rlsim.c")
_LIB = os.path.join(_HERE, "_rlsim.so")
_lib = None

CFLAGS = ["-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def build_c(force: bool = False) -> str:
    """Compile ``rlsim.c`` into ``_rlsim.so`` with gcc (no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _c():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_c())
        f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
        u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
        lib.oracle_rl_broadphase.argtypes = [f32p, f32p, u8p, u32p, ctypes.c_uint32]
        lib.oracle_rl_solve.argtypes = [f32p, f32p, u8p, f32p, ctypes.c_float, ctypes.c_float]
        lib.oracle_rl_integrate.argtypes = [f32p, f32p, f32p, ctypes.c_uint32,
                                           ctypes.c_float, ctypes.c_float, ctypes.c_float]
        for fn in (lib.oracle_rl_broadphase, lib.oracle_rl_solve, lib.oracle_rl_integrate):
            fn.restype = None
        _lib = lib
    return _lib


def _view(bufs, ref):
    return bufs[ref.buf][ref.off:ref.off + ref.n]


def _copy_in(view):
    """A contiguous scratch copy of a buffer range (C bodies take plain arrays)."""
    return np.ascontiguousarray(view).copy()


def run_task(bufs: Dict[str, np.ndarray], task) -> None:
    """Execute one task in place on ``bufs``."""
    op, A, S = task.op, task.arrays, task.scalars
    f32 = np.float32
    if op == "axpy":
        x, y = _view(bufs, A["x"]), _view(bufs, A["y"])
        ax = f32(S["a"]) * x
        y[...] = ax + y
    elif op == "scale":
        x, y = _view(bufs, A["x"]), _view(bufs, A["y"])
        y[...] = f32(S["a"]) * x
    elif op == "add":
        x, y, z = _view(bufs, A["x"]), _view(bufs, A["y"]), _view(bufs, A["z"])
        z[...] = x + y
    elif op == "gemv":
        m, k = int(S["m"]), int(S["k"])
        W = _view(bufs, A["W"]).reshape(m, k).astype(np.float64)
        x = _view(bufs, A["x"]).astype(np.float64)
        _view(bufs, A["y"])[...] = (W @ x).astype(np.float32)
    elif op == "bias_relu":
        t, b = _view(bufs, A["t"]), _view(bufs, A["b"])
        v = t + b
        t[...] = np.where(v > f32(0), v, f32(0))
    elif op == "resid":
        h, u, b = _view(bufs, A["h"]), _view(bufs, A["u"]), _view(bufs, A["b"])
        ub = u + b
        h[...] = h + ub
    elif op == "sleep":
        y = _view(bufs, A["y"])
        half = y[:1] * f32(0.5)
        y[:1] = half + f32(S["tag"])
    elif op == "rl_broadphase":
        lib = _c()
        cont = _copy_in(_view(bufs, A["cont"]))
        nisl = _copy_in(_view(bufs, A["nisl"]))
        lib.oracle_rl_broadphase(_copy_in(_view(bufs, A["pos"])), _copy_in(_view(bufs, A["prop"])),
                                 cont, nisl, ctypes.c_uint32(int(S["nenv"])))
        _view(bufs, A["cont"])[...] = cont
        _view(bufs, A["nisl"])[...] = nisl
    elif op == "rl_solve":
        lib = _c()
        vel = _copy_in(_view(bufs, A["vel"]))
        lib.oracle_rl_solve(_copy_in(_view(bufs, A["pos"])), _copy_in(_view(bufs, A["prop"])),
                            _copy_in(_view(bufs, A["cont"])), vel,
                            ctypes.c_float(S["beta_dt"]), ctypes.c_float(S["slop"]))
        _view(bufs, A["vel"])[...] = vel
    elif op == "rl_integrate":
        lib = _c()
        pos, vel = _copy_in(_view(bufs, A["pos"])), _copy_in(_view(bufs, A["vel"]))
        lib.oracle_rl_integrate(pos, vel, _copy_in(_view(bufs, A["prop"])),
                                ctypes.c_uint32(int(S["nenv"])), ctypes.c_float(S["dt"]),
                                ctypes.c_float(S["gdt"]), ctypes.c_float(S["box"]))
        _view(bufs, A["pos"])[...] = pos
        _view(bufs, A["vel"])[...] = vel
    elif op in ("nop", "rl_emit"):
        pass        # an emit task changes the stream, not the buffers
    else:
        raise ValueError(f"unknown op {op!r}")


def run_inorder(buffers: Dict[str, np.ndarray], tasks, order=None) -> Dict[str, np.ndarray]:
    """Run ``tasks`` one at a time (program order, or the index order given)
    on copies of ``buffers``; returns the final buffers."""
    bufs = {k: v.copy() for k, v in buffers.items()}
    for idx in (range(len(tasks)) if order is None else order):
        run_task(bufs, tasks[idx])
    return bufs


def run_rlsim(sim, emit: bool = False):
    """Run a ``streamgen.RLSim`` with the oracle: returns (tasks, buffers,
    batch_sizes). Each batch's tasks are emitted from the island counts the
    oracle's own broadphase wrote into ``nisl``. With ``emit`` the stream is
    the emitting variant: an emit task follows every broadphase batch."""
    bufs = {k: v.copy() for k, v in sim.buffers(emit=emit).items()}
    tasks: List = []
    sizes = []
    batch = sim.first_batch()
    if emit and sim.p.steps > 0:
        batch.append(sim.emit_task(0))
    for t in range(sim.p.steps + 1):
        if t > 0:
            batch = sim.step_batch(t - 1, bufs["nisl"].copy())
            if emit and t < sim.p.steps:
                batch.append(sim.emit_task(t))
        for task in batch:
            run_task(bufs, task)
        tasks.extend(batch)
        sizes.append(len(batch))
    return tasks, bufs, sizes
