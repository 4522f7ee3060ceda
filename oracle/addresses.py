"""Read/write segment resolution for the oracle (test infrastructure only).

Sec. IV-A ("ACS Kernel Wrappers", Fig. get_addresses): each kernel's wrapper
turns its launch arguments into ``__read_segments__`` and
``__write_segments__``, lists of ``{start_addr, size}`` byte ranges, just before
launch. The paper's worked example is matrix multiplication: inputs of m*n and
n*k elements are read, the m*k-element output is written (the listing's
comment calls the output segment "reads"; it sits in the write list, which is
the reading used).

The oracle resolves the operand roles of each op to byte ranges on a virtual
address layout: buffer number b (in sorted name order) starts at (b + 1) * 2**40.
Dependencies only depend on overlap, which any layout of disjoint buffers that
keeps in-buffer byte offsets preserves, so these edges equal the edges over real
device addresses.

Pinned by the matmul example and hand-made streams (tests/test_oracle_deps.py).
"""
from __future__ import annotations

from typing import Dict, List, Tuple

import numpy as np

# roles read and written by each op
OP_ROLES: Dict[str, Tuple[Tuple[str, ...], Tuple[str, ...]]] = {
    "axpy": (("x", "y"), ("y",)),
    "scale": (("x",), ("y",)),
    "add": (("x", "y"), ("z",)),
    "gemv": (("W", "x"), ("y",)),
    "bias_relu": (("t", "b"), ("t",)),
    "resid": (("h", "u", "b"), ("h",)),
    "rl_broadphase": (("pos", "prop"), ("cont", "nisl")),
    "rl_solve": (("pos", "prop", "cont", "vel"), ("vel",)),
    "rl_integrate": (("pos", "vel", "prop"), ("pos", "vel")),
    "sleep": ((), ("y",)),
    "rl_emit": (("nisl",), ("token",)),
}


class Layout:
    """Virtual base addresses for a dict of named numpy buffers."""

    def __init__(self, buffers: Dict[str, np.ndarray]):
        self.base = {name: (i + 1) << 40 for i, name in enumerate(sorted(buffers))}
        self.itemsize = {name: int(buffers[name].dtype.itemsize) for name in buffers}

    def segment(self, ref) -> Tuple[int, int]:
        isz = self.itemsize[ref.buf]
        return (self.base[ref.buf] + ref.off * isz, ref.n * isz)


def matmul_segments(input1: int, input2: int, output: int, m: int, n: int, k: int, elt: int):
    """The paper's get_addresses example for C(m x k) = A(m x n) B(n x k)."""
    reads = [(input1, m * n * elt), (input2, n * k * elt)]
    writes = [(output, m * k * elt)]
    return reads, writes


def task_segments(task, layout: Layout) -> Tuple[List[Tuple[int, int]], List[Tuple[int, int]]]:
    """(reads, writes) byte segments of one streamgen task."""
    rroles, wroles = OP_ROLES[task.op]
    reads = [layout.segment(task.arrays[r]) for r in rroles]
    writes = [layout.segment(task.arrays[w]) for w in wroles]
    return reads, writes


def stream_segments(tasks, buffers):
    layout = Layout(buffers)
    return [task_segments(t, layout) for t in tasks]
