"""ctypes binding of libacs.so: the C ABI of include/acs.h, same names.

Argument marshalling only -- every step of the scheduling path (descriptor
rings, window, dependency test, state machine, dispatch, task bodies) runs in
libacs.so and its CUDA kernels. Importing this module without the built
library raises; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libacs.so")

ACS_OK = 0
ACS_ERR_INVALID = -1
ACS_ERR_FULL = -2
ACS_ERR_TIMEOUT = -3
ACS_ERR_DEVICE = -4
ACS_ERR_STOPPED = -5
ACS_ERR_ORDER = -6
ACS_ERR_NOMEM = -7
ACS_ERR_RANGE = -8
ACS_MAX_POSITION = 1 << 31

ACS_MAX_WINDOW = 64
ACS_MAX_SEGS = 16
ACS_MAX_NCTA = 256
ACS_MAX_STREAMS = 256
ACS_BLOCK_THREADS = 256
ACS_WHOLE_MEMORY = (0, (1 << 64) - 1)
ACS_NOALLOC_MAX_TASKS = 4096

OPS = {"nop": 0, "axpy": 1, "scale": 2, "add": 3, "gemv": 4, "bias_relu": 5, "resid": 6,
       "rl_broadphase": 10, "rl_solve": 11, "rl_integrate": 12, "rl_emit": 13, "wait_flag": 30,
       "sleep": 31}

ACS_MODE_WINDOW, ACS_MODE_INORDER, ACS_MODE_GRAPH, ACS_MODE_SW = 0, 1, 2, 3
ACS_FLAG_LOG, ACS_FLAG_TIMING, ACS_FLAG_TRACE = 1, 2, 4

ACS_RL_SPHERES = 32
ACS_RL_REC_BYTES = 1088


class acs_segment(C.Structure):
    _fields_ = [("start", C.c_uint64), ("size", C.c_uint64)]


class acs_args(C.Structure):
    _fields_ = [("op", C.c_uint16), ("ncta", C.c_uint16), ("reserved", C.c_uint32),
                ("bytes", C.c_uint8 * 48)]


class acs_config(C.Structure):
    _fields_ = [("mode", C.c_uint32), ("n_streams", C.c_uint32), ("cta_slots", C.c_uint32),
                ("capacity", C.c_uint32), ("log_capacity", C.c_uint32), ("flags", C.c_uint32),
                ("timeout_ns", C.c_uint64), ("cuda_stream", C.c_void_p), ("device", C.c_int32),
                ("poll_ns", C.c_uint32), ("ctas_per_sm", C.c_uint32), ("idle_limit_ms", C.c_uint32),
                ("sw_threads", C.c_uint32), ("span", C.c_uint32), ("lookahead", C.c_uint32),
                ("reserved", C.c_uint32 * 1)]

LOOKAHEAD_AUTO = 0xFFFFFFFF


class acs_stats(C.Structure):
    _fields_ = [("tasks_submitted", C.c_uint64), ("tasks_flushed", C.c_uint64), ("launches", C.c_uint64),
                ("seg_bytes", C.c_uint64), ("kernel_ms", C.c_double), ("graph_build_ms", C.c_double),
                ("graph_instantiate_ms", C.c_double), ("graph_edges", C.c_uint64),
                ("sched_cycles", C.c_uint64), ("sched_busy_cycles", C.c_uint64),
                ("sched_inserts", C.c_uint64), ("sched_iterations", C.c_uint64),
                ("sched_phase_cycles", C.c_uint64 * 8), ("tasks_emitted", C.c_uint64),
                ("device_seg_bytes", C.c_uint64), ("check_cycles", C.c_uint64),
                ("starved_iters", C.c_uint64), ("cta_slots", C.c_uint32),
                ("grid", C.c_uint32)]


# numpy image of acs_args (56 bytes) for packing many tasks at once
ARGS_DTYPE = np.dtype([("op", "<u2"), ("ncta", "<u2"), ("reserved", "<u4"), ("bytes", "V48")])
assert ARGS_DTYPE.itemsize == C.sizeof(acs_args) == 56

EXPORTS = ["acs_config_default", "acs_init", "acs_get_addresses", "acs_submit", "acs_submit_stream",
           "acs_submit_ops", "acs_flush", "acs_sync", "acs_get_log", "acs_get_trace", "acs_stream_tail",
           "acs_get_stats", "acs_graph_replay", "acs_start", "acs_progress", "acs_stop",
           "acs_error", "acs_strerror", "acs_destroy", "acs_run_noalloc", "acs_abort", "acs_stream_rebase"]

_lib = None


def load(path: str = LIB_PATH):
    """Load libacs.so and declare the prototypes (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libacs.so not built at {path}: run __graft_entry__.build()")
    lib = C.CDLL(path)
    P = C.POINTER
    lib.acs_config_default.argtypes = [P(acs_config)]
    lib.acs_config_default.restype = None
    lib.acs_init.argtypes = [P(C.c_void_p), C.c_uint32, P(acs_config)]
    lib.acs_get_addresses.argtypes = [P(acs_args), P(acs_segment), P(C.c_uint32), P(acs_segment), P(C.c_uint32)]
    lib.acs_submit.argtypes = [C.c_void_p, C.c_uint32, P(acs_args), P(acs_segment), C.c_uint32,
                               P(acs_segment), C.c_uint32]
    lib.acs_submit_stream.argtypes = [C.c_void_p, C.c_uint32, C.c_uint32, P(acs_args), P(acs_segment),
                                      C.c_uint32, P(acs_segment), C.c_uint32]
    lib.acs_submit_ops.argtypes = [C.c_void_p, C.c_uint32, C.c_uint32, C.c_void_p, C.c_void_p]
    lib.acs_flush.argtypes = [C.c_void_p]
    lib.acs_sync.argtypes = [C.c_void_p]
    lib.acs_get_log.argtypes = [C.c_void_p, C.c_uint32, C.c_uint64, C.c_uint32, C.c_void_p, C.c_void_p,
                                C.c_void_p]
    lib.acs_get_trace.argtypes = [C.c_void_p, C.c_uint32, C.c_uint64, C.c_uint32, C.c_void_p]
    lib.acs_stream_tail.argtypes = [C.c_void_p, C.c_uint32, P(C.c_uint32)]
    lib.acs_stream_rebase.argtypes = [C.c_void_p, C.c_uint32, C.c_uint32]
    lib.acs_get_stats.argtypes = [C.c_void_p, P(acs_stats)]
    lib.acs_graph_replay.argtypes = [C.c_void_p]
    lib.acs_start.argtypes = [C.c_void_p]
    lib.acs_progress.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    lib.acs_stop.argtypes = [C.c_void_p]
    lib.acs_error.argtypes = [C.c_void_p]
    lib.acs_abort.argtypes = [C.c_void_p]
    lib.acs_strerror.argtypes = [C.c_int]
    lib.acs_strerror.restype = C.c_char_p
    lib.acs_run_noalloc.argtypes = [C.c_uint32, C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.acs_destroy.argtypes = [C.c_void_p]
    lib.acs_destroy.restype = None
    for name in EXPORTS:
        fn = getattr(lib, name)
        if name not in ("acs_config_default", "acs_strerror", "acs_destroy"):
            fn.restype = C.c_int
    _lib = lib
    return lib


class AcsError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = load().acs_strerror(code).decode()
        super().__init__(f"{what}: {msg} ({code})" if what else f"{msg} ({code})")


def check(code: int, what: str = "") -> int:
    if code != ACS_OK:
        raise AcsError(code, what)
    return code


# ---- thin wrappers with the C names ------------------------------------------

def acs_config_default() -> acs_config:
    cfg = acs_config()
    load().acs_config_default(C.byref(cfg))
    return cfg


def acs_init(window: int, cfg: acs_config = None) -> C.c_void_p:
    h = C.c_void_p()
    check(load().acs_init(C.byref(h), window, C.byref(cfg) if cfg is not None else None), "acs_init")
    return h


def acs_get_addresses(args: acs_args):
    r = (acs_segment * ACS_MAX_SEGS)()
    w = (acs_segment * ACS_MAX_SEGS)()
    nr, nw = C.c_uint32(), C.c_uint32()
    check(load().acs_get_addresses(C.byref(args), r, C.byref(nr), w, C.byref(nw)), "acs_get_addresses")
    return ([(r[i].start, r[i].size) for i in range(nr.value)],
            [(w[i].start, w[i].size) for i in range(nw.value)])


def _segs(lst):
    arr = (acs_segment * max(1, len(lst)))()
    for i, (a, n) in enumerate(lst):
        arr[i].start, arr[i].size = a, n
    return arr


def acs_submit(ctx, task_id: int, args: acs_args, reads, writes) -> int:
    return load().acs_submit(ctx, task_id, C.byref(args), _segs(reads), len(reads), _segs(writes), len(writes))


def acs_submit_stream(ctx, stream: int, task_id: int, args: acs_args, reads, writes) -> int:
    return load().acs_submit_stream(ctx, stream, task_id, C.byref(args), _segs(reads), len(reads),
                                    _segs(writes), len(writes))


def acs_submit_ops(ctx, stream: int, task_ids: np.ndarray, packed: np.ndarray) -> int:
    """Submit len(task_ids) tasks whose acs_args are rows of ``packed`` (ARGS_DTYPE)."""
    ids = np.ascontiguousarray(task_ids, dtype=np.uint32)
    packed = np.ascontiguousarray(packed)
    assert packed.dtype == ARGS_DTYPE and len(packed) == len(ids)
    return load().acs_submit_ops(ctx, stream, len(ids), ids.ctypes.data, packed.ctypes.data)


def acs_flush(ctx) -> int:
    return load().acs_flush(ctx)


def acs_sync(ctx) -> int:
    return load().acs_sync(ctx)


def acs_get_log(ctx, stream: int, first: int, n: int):
    masks = np.zeros(n, np.uint64)
    start = np.zeros(n, np.uint64)
    retire = np.zeros(n, np.uint64)
    check(load().acs_get_log(ctx, stream, first, n, masks.ctypes.data, start.ctypes.data, retire.ctypes.data),
          "acs_get_log")
    return masks, start, retire


def acs_get_trace(ctx, stream: int, first: int, n: int) -> np.ndarray:
    """(n, 5) globaltimer ns: insert, units published, first-CTA start, last-CTA end, retire seen."""
    t = np.zeros((n, 5), np.uint64)
    check(load().acs_get_trace(ctx, stream, first, n, t.ctypes.data), "acs_get_trace")
    return t


def acs_stream_tail(ctx, stream: int) -> int:
    v = C.c_uint32()
    check(load().acs_stream_tail(ctx, stream, C.byref(v)), "acs_stream_tail")
    return v.value


def acs_stream_rebase(ctx, stream: int, pos: int = 0) -> int:
    return load().acs_stream_rebase(ctx, stream, pos)


def acs_start(ctx) -> None:
    check(load().acs_start(ctx), "acs_start")


def acs_stop(ctx) -> None:
    check(load().acs_stop(ctx), "acs_stop")


def acs_progress(ctx, n_streams: int, head: np.ndarray = None, idle_at: np.ndarray = None):
    """(head, idle_at) uint32 arrays of n_streams (filled in place when given)."""
    if head is None:
        head = np.zeros(n_streams, np.uint32)
    if idle_at is None:
        idle_at = np.zeros(n_streams, np.uint32)
    check(load().acs_progress(ctx, head.ctypes.data, idle_at.ctypes.data), "acs_progress")
    return head, idle_at


def acs_get_stats(ctx) -> acs_stats:
    s = acs_stats()
    check(load().acs_get_stats(ctx, C.byref(s)), "acs_get_stats")
    return s


def acs_graph_replay(ctx) -> int:
    return load().acs_graph_replay(ctx)


def acs_error(ctx) -> int:
    return load().acs_error(ctx)


def acs_abort(ctx) -> int:
    """Raise the context's device stop word (any host thread); see include/acs.h."""
    return load().acs_abort(ctx)


def acs_strerror(code: int) -> str:
    return load().acs_strerror(code).decode()


def acs_run_noalloc(window: int, task_ids: np.ndarray, packed: np.ndarray, cuda_stream: int = 0) -> int:
    """Run the packed tasks with the library's fixed scratch (no allocation)."""
    ids = np.ascontiguousarray(task_ids, dtype=np.uint32)
    packed = np.ascontiguousarray(packed)
    assert packed.dtype == ARGS_DTYPE and len(packed) == len(ids)
    return load().acs_run_noalloc(window, len(ids), ids.ctypes.data, packed.ctypes.data, cuda_stream)


def acs_destroy(ctx) -> None:
    load().acs_destroy(ctx)


def stats_dict(s: acs_stats) -> dict:
    out = {k: getattr(s, k) for k, _ in acs_stats._fields_}
    out["sched_phase_cycles"] = list(s.sched_phase_cycles)
    return out
