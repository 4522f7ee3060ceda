"""Drive streamgen task streams through libacs (argument marshalling only).

Maps named streamgen buffers to CUDA tensors, packs each task's device
pointers and scalars into ``acs_args`` rows (the layouts of the acs_*_args
structs in include/acs.h), submits them with ``acs_submit_ops`` -- which
derives read/write segments in the library (acs_get_addresses) -- and runs the
rigid-sphere stream step by step, reading back the island counts its own
broadphase tasks wrote.
"""
from __future__ import annotations

import ctypes as C
from typing import Dict, List, Optional

import numpy as np
import torch

from . import acs

# per-op argument layouts (must match include/acs.h)
_U8 = "<u8"
OP_DTYPES = {
    "axpy": np.dtype([("x", _U8), ("y", _U8), ("n", "<u4"), ("a", "<f4")]),
    "scale": np.dtype([("x", _U8), ("y", _U8), ("n", "<u4"), ("a", "<f4")]),
    "add": np.dtype([("x", _U8), ("y", _U8), ("z", _U8), ("n", "<u4"), ("pad", "<u4")]),
    "gemv": np.dtype([("W", _U8), ("x", _U8), ("y", _U8), ("m", "<u4"), ("k", "<u4")]),
    "bias_relu": np.dtype([("t", _U8), ("b", _U8), ("n", "<u4"), ("pad", "<u4")]),
    "resid": np.dtype([("h", _U8), ("u", _U8), ("b", _U8), ("n", "<u4"), ("pad", "<u4")]),
    "rl_broadphase": np.dtype([("pos", _U8), ("prop", _U8), ("cont", _U8), ("nisl", _U8), ("nenv", "<u4"),
                               ("pad", "<u4")]),
    "rl_solve": np.dtype([("pos", _U8), ("prop", _U8), ("cont", _U8), ("vel", _U8), ("beta_dt", "<f4"),
                          ("slop", "<f4")]),
    "rl_integrate": np.dtype([("pos", _U8), ("vel", _U8), ("prop", _U8), ("nenv", "<u4"), ("dt", "<f4"),
                              ("gdt", "<f4"), ("box", "<f4")]),
    "rl_emit": np.dtype([("cfg", _U8), ("nisl", _U8), ("token", _U8), ("ncta_table", _U8), ("n_env", "<u4"),
                         ("step", "<u4"), ("steps", "<u4"), ("chunk", "<u4")]),
    "wait_flag": np.dtype([("flag", _U8), ("limit_ns", _U8)]),
    "sleep": np.dtype([("y", _U8), ("ns", _U8), ("tag", "<f4"), ("pad", "<u4")]),
}
for _dt in OP_DTYPES.values():
    assert _dt.itemsize <= 48


class DeviceBuffers:
    """Named streamgen buffers as CUDA byte tensors (caller-owned device memory)."""

    def __init__(self, buffers: Dict[str, np.ndarray], device: str = "cuda"):
        self.dtype = {k: v.dtype for k, v in buffers.items()}
        self.t = {k: torch.from_numpy(np.ascontiguousarray(v).view(np.uint8).copy()).to(device)
                  for k, v in buffers.items()}
        self.base = {k: int(v.data_ptr()) for k, v in self.t.items()}

    def ptr(self, ref) -> int:
        return self.base[ref.buf] + ref.off * self.dtype[ref.buf].itemsize

    def upload(self, buffers: Dict[str, np.ndarray]) -> None:
        for k, v in buffers.items():
            self.t[k].copy_(torch.from_numpy(np.ascontiguousarray(v).view(np.uint8)))

    def download(self) -> Dict[str, np.ndarray]:
        # the current stream only: a resident scheduler kernel keeps the device busy
        torch.cuda.current_stream().synchronize()
        return {k: v.cpu().numpy().view(self.dtype[k]) for k, v in self.t.items()}


def _args_row(op: str, ncta: int, fields: dict) -> np.ndarray:
    row = np.zeros(1, acs.ARGS_DTYPE)
    row["op"] = acs.OPS[op]
    row["ncta"] = ncta
    body = np.zeros(1, OP_DTYPES[op])
    for k, v in fields.items():
        body[k] = v
    raw = np.zeros(48, np.uint8)
    raw[:body.itemsize] = np.frombuffer(body.tobytes(), np.uint8)
    row["bytes"] = raw.tobytes()
    return row


def pack_task(task, bufs: DeviceBuffers) -> np.ndarray:
    """One streamgen task as a packed acs_args row."""
    A, S = task.arrays, task.scalars
    op = task.op
    if op in ("axpy", "scale"):
        f = {"x": bufs.ptr(A["x"]), "y": bufs.ptr(A["y"]), "n": A["y"].n, "a": S["a"]}
    elif op == "add":
        f = {"x": bufs.ptr(A["x"]), "y": bufs.ptr(A["y"]), "z": bufs.ptr(A["z"]), "n": A["z"].n}
    elif op == "gemv":
        f = {"W": bufs.ptr(A["W"]), "x": bufs.ptr(A["x"]), "y": bufs.ptr(A["y"]), "m": S["m"], "k": S["k"]}
    elif op == "bias_relu":
        f = {"t": bufs.ptr(A["t"]), "b": bufs.ptr(A["b"]), "n": A["t"].n}
    elif op == "resid":
        f = {"h": bufs.ptr(A["h"]), "u": bufs.ptr(A["u"]), "b": bufs.ptr(A["b"]), "n": A["h"].n}
    elif op == "rl_broadphase":
        f = {"pos": bufs.ptr(A["pos"]), "prop": bufs.ptr(A["prop"]), "cont": bufs.ptr(A["cont"]),
             "nisl": bufs.ptr(A["nisl"]), "nenv": S["nenv"]}
    elif op == "rl_solve":
        f = {"pos": bufs.ptr(A["pos"]), "prop": bufs.ptr(A["prop"]), "cont": bufs.ptr(A["cont"]),
             "vel": bufs.ptr(A["vel"]), "beta_dt": S["beta_dt"], "slop": S["slop"]}
    elif op == "rl_integrate":
        f = {"pos": bufs.ptr(A["pos"]), "vel": bufs.ptr(A["vel"]), "prop": bufs.ptr(A["prop"]),
             "nenv": S["nenv"], "dt": S["dt"], "gdt": S["gdt"], "box": S["box"]}
    elif op == "sleep":
        f = {"y": bufs.ptr(A["y"]), "ns": S["ns"], "tag": S["tag"]}
    elif op == "rl_emit":
        f = {"cfg": S["cfg"], "nisl": bufs.ptr(A["nisl"]), "token": bufs.ptr(A["token"]),
             "ncta_table": S["ncta_table"], "n_env": A["nisl"].n, "step": S["step"], "steps": S["steps"],
             "chunk": S["chunk"]}
    elif op == "wait_flag":
        f = {"flag": S["flag"], "limit_ns": S["limit_ns"]}
    else:
        raise ValueError(f"unknown op {op!r}")
    return _args_row(op, task.ncta, f)


def pack_tasks(tasks, bufs: DeviceBuffers):
    """(task_ids, packed acs_args rows) for a list of streamgen tasks."""
    if not tasks:
        return np.zeros(0, np.uint32), np.zeros(0, acs.ARGS_DTYPE)
    ids = np.array([t.task_id for t in tasks], np.uint32)
    return ids, np.concatenate([pack_task(t, bufs) for t in tasks])


MODES = {"window": acs.ACS_MODE_WINDOW, "inorder": acs.ACS_MODE_INORDER, "graph": acs.ACS_MODE_GRAPH,
         "sw": acs.ACS_MODE_SW}


# Dispatch lookahead for window-mode Contexts (no free-slot span) created
# without one (None: the library's default).
DEFAULT_LOOKAHEAD: Optional[int] = None
# a driver restarts an idle stream's positions once they pass this (the library
# takes host-submitted tasks only below 2^31 per stream)
REBASE_AT = 1 << 30


class Context:
    """An acs_ctx on the current torch CUDA stream (raises on every error)."""

    def __init__(self, window: int, mode: str = "window", n_streams: int = 1, cta_slots: int = 0,
                 capacity: int = 0, log: bool = False, timing: bool = False, trace: bool = False,
                 timeout_s: float = 5.0, poll_ns: int = 0, ctas_per_sm: int = 0,
                 cuda_stream: Optional[int] = None, resident: bool = False, idle_limit_ms: int = 0,
                 sw_threads: int = 0, span: int = 0, lookahead: Optional[int] = None):
        cfg = acs.acs_config_default()
        cfg.mode = MODES[mode]
        cfg.n_streams = n_streams
        cfg.cta_slots = cta_slots
        if capacity:
            cfg.capacity = capacity
        cfg.flags = ((acs.ACS_FLAG_LOG if log else 0) | (acs.ACS_FLAG_TIMING if timing else 0)
                     | (acs.ACS_FLAG_TRACE if trace else 0))
        cfg.timeout_ns = int(timeout_s * 1e9)
        cfg.poll_ns = poll_ns
        cfg.ctas_per_sm = ctas_per_sm
        cfg.idle_limit_ms = idle_limit_ms
        cfg.sw_threads = sw_threads
        cfg.span = span
        if lookahead is None and mode == "window" and not span:
            lookahead = DEFAULT_LOOKAHEAD
        if lookahead is not None:          # None: the library's default (dispatch ahead, auto)
            cfg.lookahead = lookahead
        # All device work of the context goes to one stream shared with torch, so
        # torch copies of the task buffers are ordered with the tasks. The legacy
        # default stream has no handle to share: then a torch stream is made
        # current for the context's lifetime.
        self._prev_stream = None
        self._lib_stream = None
        if cuda_stream is None and resident:
            # a resident kernel occupies its stream until stopped: the library
            # gets a stream of its own, torch's current stream stays free for
            # the caller's copies (which the caller completes before flushing)
            if torch.cuda.current_stream().cuda_stream == 0:
                self._prev_stream = torch.cuda.current_stream()
                torch.cuda.set_stream(torch.cuda.Stream())
            self._lib_stream = torch.cuda.Stream()
            cuda_stream = self._lib_stream.cuda_stream
        if cuda_stream is None:
            cur = torch.cuda.current_stream()
            if cur.cuda_stream == 0:
                torch.cuda.synchronize()
                self._prev_stream = cur
                self._stream = torch.cuda.Stream()
                torch.cuda.set_stream(self._stream)
                cur = self._stream
            cuda_stream = cur.cuda_stream
        cfg.cuda_stream = C.c_void_p(cuda_stream)
        self.window, self.mode, self.n_streams = window, mode, n_streams
        self.span = span or window   # ring span: logged masks are over span - 1 predecessors
        try:
            self.h = acs.acs_init(window, cfg)
        except acs.AcsError:
            if self._prev_stream is not None:     # leave torch's current stream as it was
                torch.cuda.set_stream(self._prev_stream)
            raise
        self.resident = False
        if resident:
            self.start()

    def start(self) -> None:
        """Leave the scheduler kernel resident (acs_start)."""
        acs.acs_start(self.h)
        self.resident = True

    def stop(self) -> None:
        """Drain and end the resident kernel (acs_stop)."""
        self.resident = False
        acs.acs_stop(self.h)

    def progress(self, head: Optional[np.ndarray] = None, idle_at: Optional[np.ndarray] = None):
        """(head, idle_at) per stream (acs_progress)."""
        return acs.acs_progress(self.h, self.n_streams, head, idle_at)

    def submit_packed(self, ids: np.ndarray, packed: np.ndarray, stream: int = 0) -> None:
        acs.check(acs.acs_submit_ops(self.h, stream, ids, packed), "acs_submit_ops")

    def submit(self, tasks, bufs: DeviceBuffers, stream: int = 0) -> None:
        self.submit_packed(*pack_tasks(tasks, bufs), stream=stream)

    def flush(self) -> None:
        acs.check(acs.acs_flush(self.h), "acs_flush")

    def sync(self) -> None:
        acs.check(acs.acs_sync(self.h), "acs_sync")

    def sync_code(self) -> int:
        return acs.acs_sync(self.h)

    def log(self, stream: int, first: int, n: int):
        return acs.acs_get_log(self.h, stream, first, n)

    def trace(self, stream: int, first: int, n: int) -> np.ndarray:
        return acs.acs_get_trace(self.h, stream, first, n)

    def stats(self) -> dict:
        return acs.stats_dict(acs.acs_get_stats(self.h))

    def tail(self, stream: int = 0) -> int:
        return acs.acs_stream_tail(self.h, stream)

    def rebase(self, stream: int = 0, pos: int = 0) -> None:
        """Restart an idle stream's positions at `pos` (acs_stream_rebase)."""
        acs.check(acs.acs_stream_rebase(self.h, stream, pos), "acs_stream_rebase")

    def replay(self) -> None:
        acs.check(acs.acs_graph_replay(self.h), "acs_graph_replay")

    def close(self) -> None:
        if self.h:
            acs.acs_destroy(self.h)
            self.h = None
        if self._prev_stream is not None:
            torch.cuda.synchronize()
            torch.cuda.set_stream(self._prev_stream)
            self._prev_stream = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def run_stream(stream, mode: str = "window", window: Optional[int] = None, log: bool = False,
               cta_slots: int = 0, flush_every: int = 0, lookahead: Optional[int] = None):
    """Run one streamgen Stream on the GPU; returns (buffers after, context
    stats, log or None). ``flush_every`` > 0 splits the stream into flushes."""
    bufs = DeviceBuffers(stream.buffers)
    W = window or stream.window
    with Context(W, mode=mode, log=log, cta_slots=cta_slots, lookahead=lookahead) as ctx:
        ids, packed = pack_tasks(stream.tasks, bufs)
        step = flush_every or len(ids) or 1
        for a in range(0, len(ids), step):
            ctx.submit_packed(ids[a:a + step], packed[a:a + step])
            ctx.flush()
        ctx.sync()
        lg = ctx.log(0, 0, len(ids)) if (log and mode == "window") else None
        st = ctx.stats()
    return bufs.download(), st, lg


# ---- rigid-sphere stream -------------------------------------------------------------

class RLDriver:
    """Runs a streamgen.RLSim on the GPU through one Context: per step, flush
    the batch, sync, read back nisl (4 bytes per env) and emit the next plan.
    Packing is vectorised from per-env / per-chunk templates."""

    def __init__(self, sim, bufs: DeviceBuffers, ctx: Context, stream: int = 0):
        self.sim, self.bufs, self.ctx, self.stream = sim, bufs, ctx, stream
        p = sim.p
        sc = sim.scalars()
        self.templates = {}
        for kind, op in ((0, "rl_broadphase"), (1, "rl_solve"), (2, "rl_integrate")):
            n = p.n_env if kind == 1 else p.n_env // p.chunk
            rows = []
            for idx in range(n):
                fake = sim.tasks(_one_plan(kind, idx))[0]
                fake.scalars = dict(sc[op])
                rows.append(pack_task(fake, bufs))
            self.templates[kind] = np.concatenate(rows)
        self.nisl_host = torch.empty(p.n_env, dtype=torch.int32, pin_memory=True)

    def pack(self, plan):
        rows = np.empty(len(plan.kind), acs.ARGS_DTYPE)
        for kind in (0, 1, 2):
            sel = plan.kind == kind
            if sel.any():
                rows[sel] = self.templates[kind][plan.index[sel]]
        rows["ncta"] = plan.ncta
        return plan.ids, rows

    def start_read_nisl(self) -> None:
        self.nisl_host.copy_(self.bufs.t["nisl"].view(torch.int32), non_blocking=True)

    def nisl(self) -> np.ndarray:
        """The island counts of the last start_read_nisl (after a stream sync)."""
        return self.nisl_host.numpy().view(np.uint32)

    def read_nisl(self) -> np.ndarray:
        self.start_read_nisl()
        torch.cuda.current_stream().synchronize()
        return self.nisl()

    def begin(self):
        """The first plan, numbered from the stream's current position."""
        self.sim.next_id = self.ctx.tail(self.stream)
        return self.sim.first_plan()

    def submit_plan(self, plan) -> None:
        self.ctx.submit_packed(*self.pack(plan), stream=self.stream)

    def run(self, record_plans: bool = False) -> List:
        plans = []
        plan = self.begin()
        for t in range(self.sim.p.steps + 1):
            if t > 0:
                plan = self.sim.step_plan(t - 1, self.read_nisl())
            self.submit_plan(plan)
            self.ctx.flush()
            self.ctx.sync()
            if record_plans:
                plans.append(plan)
        return plans


EMIT_CFG_DTYPE = np.dtype([("pos", _U8), ("vel", _U8), ("prop", _U8), ("cont", _U8), ("beta_dt", "<f4"),
                           ("slop", "<f4"), ("dt", "<f4"), ("gdt", "<f4"), ("box", "<f4"), ("pad", "<u4", 3)])
assert EMIT_CFG_DTYPE.itemsize == 64


class RLEmitDriver:
    """Runs a streamgen.RLSim on the GPU with device-side emission: the host
    submits the first broadphase batch and the first emit task once; every
    later task is appended on the device by emit tasks, so the whole run is one
    flush, one persistent launch and one sync."""

    def __init__(self, sim, bufs: DeviceBuffers, ctx: Context, stream: int = 0):
        table = sim.ncta_table()
        if table.size and int(table.min()) < 1:      # the device takes these CTA counts as they are
            raise ValueError("ncta_table entries must be 1 .. 255")
        self.sim, self.bufs, self.ctx, self.stream = sim, bufs, ctx, stream
        p = sim.p
        sc = sim.scalars()
        cfg = np.zeros(1, EMIT_CFG_DTYPE)
        for k in ("pos", "vel", "prop", "cont"):
            cfg[k] = bufs.base[k]
        for k in ("beta_dt", "slop"):
            cfg[k] = sc["rl_solve"][k]
        for k in ("dt", "gdt", "box"):
            cfg[k] = sc["rl_integrate"][k]
        self.cfg = torch.from_numpy(cfg.view(np.uint8).copy()).to("cuda")
        self.table = torch.from_numpy(table).to("cuda")
        self._packed = None   # the first tasks' rows: the same every run, ids aside

    def first_tasks(self):
        p = self.sim.p
        tasks = self.sim.first_batch()
        if p.steps > 0:
            e = self.sim.emit_task(0)
            e.scalars.update({"cfg": int(self.cfg.data_ptr()), "ncta_table": int(self.table.data_ptr()),
                              "steps": np.uint32(p.steps), "chunk": np.uint32(p.chunk)})
            tasks.append(e)
        return tasks

    def submit(self) -> int:
        """Submit the run's first tasks to the context (no flush); returns the
        stream position the run starts at."""
        if self.ctx.tail(self.stream) >= REBASE_AT:   # idle here: keep positions clear of 2^31
            self.ctx.rebase(self.stream)
        start = self.ctx.tail(self.stream)
        # emitted tasks take task_id = their position, so ids continue from there
        if self._packed is None:
            self.sim.next_id = 0
            self._packed = pack_tasks(self.first_tasks(), self.bufs)
        ids, rows = self._packed
        self.sim.next_id = start + len(ids)
        self.ctx.submit_packed(ids + np.uint32(start), rows, stream=self.stream)
        return start

    def run(self) -> int:
        """One complete run; returns the number of tasks the stream had."""
        start = self.submit()
        self.ctx.flush()
        self.ctx.sync()
        return self.ctx.tail(self.stream) - start


def _one_plan(kind: int, idx: int):
    import streamgen as sg
    return sg.RLPlan(np.array([kind], np.uint8), np.array([idx], np.uint32), np.array([1], np.uint16), 0,
                     np.array([0], np.uint32))


# ---- many independent streams in one persistent launch ----------------------------------

# buffers each kind of stream writes (the rest are read-only inputs)
WRITTEN = {"rl": ("pos", "vel", "cont", "nisl", "token"), "dnn": ("h", "t", "u")}
# what a caller reads back as the result of a stream
RESULTS = {"rl": ("pos", "vel"), "dnn": ("h",)}


class _Batch:
    """Device buffers of every stream of a batch, with device-side pristine
    copies of the written buffers (fast resets between runs) and pinned host
    copies of every buffer (host-to-device runs)."""

    def _add(self, kind, host, bufs, drv) -> None:
        keep = {k: bufs.t[k].clone() for k in WRITTEN[kind] if k in bufs.t}
        self.items.append((kind, host, bufs, drv))
        self._pristine.append(keep)

    def reset(self) -> None:
        """Restore every written buffer to the stream's initial state: device
        copies, or, while a resident kernel holds every SM (a device-to-device
        copy would wait for it), copies from pinned host memory."""
        if self.ctx is not None and self.ctx.resident:
            for (_, _, bufs, _), keep in zip(self.items, self.host_written()):
                for k, v in keep.items():
                    bufs.t[k].copy_(v, non_blocking=True)
            return
        for (_, _, bufs, _), keep in zip(self.items, self._pristine):
            for k, v in keep.items():
                bufs.t[k].copy_(v, non_blocking=True)

    def host_written(self):
        """Pinned host copies of each stream's written buffers, initial state
        (create them before a resident kernel starts: pinning is slow)."""
        if self._written is None:
            self._written = [{k: torch.from_numpy(np.ascontiguousarray(host[k]).view(np.uint8).copy()).pin_memory()
                              for k in WRITTEN[kind] if k in host} for kind, host, _, _ in self.items]
        return self._written

    def host_inputs(self):
        if self._pinned is None:
            self._pinned = [{k: torch.from_numpy(np.ascontiguousarray(v).view(np.uint8).copy()).pin_memory()
                             for k, v in host.items()} for _, host, _, _ in self.items]
        return self._pinned

    def upload_host(self) -> int:
        """Copy every buffer of every stream from pinned host memory; returns bytes."""
        n = 0
        for (_, _, bufs, _), pin in zip(self.items, self.host_inputs()):
            for k, v in pin.items():
                bufs.t[k].copy_(v, non_blocking=True)
                n += v.numel()
        return n

    def result_buffers(self):
        """Pinned host tensors for each stream's result buffers."""
        if self._results is None:
            self._results = [{k: torch.empty(bufs.t[k].numel(), dtype=torch.uint8, pin_memory=True)
                              for k in RESULTS[kind]} for kind, _, bufs, _ in self.items]
        return self._results

    def download_results(self) -> int:
        """Start device-to-host copies of each stream's results; returns bytes."""
        n = 0
        for (_, _, bufs, _), out in zip(self.items, self.result_buffers()):
            for k, v in out.items():
                v.copy_(bufs.t[k], non_blocking=True)
                n += v.numel()
        return n

    def outputs(self):
        return [bufs.download() for _, _, bufs, _ in self.items]

    def _init_common(self, specs, ctx) -> None:
        self.specs, self.ctx = specs, ctx
        self.items, self._pristine = [], []
        self._pinned = self._results = self._written = None

    @staticmethod
    def _dnn(sp):
        import streamgen as sg
        return sg.dnn_stream(sp.seed, batch=sp.dnn_batch, blocks=sp.dnn_blocks, weight_sets=min(sp.dnn_blocks, 24))


class BatchedWorkload(_Batch):
    """The streams of ``streamgen.batched_specs`` on one device: rigid-sphere
    streams run with device-side emission, DNN streams are submitted whole;
    every stream is one of the context's independent streams, so one flush
    runs all of them in one persistent launch."""

    def __init__(self, specs, ctx: Optional[Context]):
        import streamgen as sg
        self._init_common(specs, ctx)
        for i, sp in enumerate(specs):
            if sp.kind == "rl":
                sim = sg.RLSim(sp.seed, sp.rl)
                host = sim.buffers(emit=True)
                bufs = DeviceBuffers(host)
                self._add("rl", host, bufs, RLEmitDriver(sim, bufs, ctx, stream=i))
            else:
                st = self._dnn(sp)
                bufs = DeviceBuffers(st.buffers)
                self._add("dnn", st.buffers, bufs, pack_tasks(st.tasks, bufs))

    def bind(self, ctx: Context) -> None:
        """Run the same streams (same device buffers) through another context."""
        self.ctx = ctx
        for kind, _, _, drv in self.items:
            if kind == "rl":
                drv.ctx = ctx

    def submit_all(self) -> None:
        for i, (kind, host, bufs, drv) in enumerate(self.items):
            if kind == "rl":
                drv.submit()
            else:
                ids, packed = drv
                # ids continue from the stream's position across repeated runs
                self.ctx.submit_packed(ids + np.uint32(self.ctx.tail(i)), packed, stream=i)

    def run(self) -> int:
        """One pass over every stream; returns tasks run. With an ordinary
        context: one flush, one launch. With a resident context: each stream
        is published as soon as it is submitted, longest first, so the kernel
        runs the long chains while the host still submits the short ones."""
        before = [self.ctx.tail(i) for i in range(len(self.items))]
        if self.ctx.resident:
            torch.cuda.current_stream().synchronize()    # resets and uploads are on the device
            for i in sorted(range(len(self.items)), key=lambda k: -self.specs[k].target):
                kind, _, _, drv = self.items[i]
                if kind == "rl":
                    drv.submit()
                else:
                    ids, packed = drv
                    self.ctx.submit_packed(ids + np.uint32(self.ctx.tail(i)), packed, stream=i)
                self.ctx.flush()
        else:
            self.submit_all()
            self.ctx.flush()
        self.ctx.sync()
        return sum(self.ctx.tail(i) - b for i, b in enumerate(before))


class BatchedHostDriven(_Batch):
    """The streams of ``streamgen.batched_specs`` without device-side
    emission, for the in-order and CUDA-graph baselines (which cannot emit) and
    the host-driven window arm. Streams advance in lockstep rounds: round 0
    submits every DNN stream whole and the first step of every rigid-sphere
    stream; round t > 0 reads back the island counts of every rigid-sphere
    stream that has a step t and submits that step. One flush and one sync per
    round, over all streams."""

    def __init__(self, specs, ctx: Context):
        import streamgen as sg
        self._init_common(specs, ctx)
        for i, sp in enumerate(specs):
            if sp.kind == "rl":
                sim = sg.RLSim(sp.seed, sp.rl)
                host = sim.buffers(emit=False)
                bufs = DeviceBuffers(host)
                self._add("rl", host, bufs, RLDriver(sim, bufs, ctx, stream=i))
            else:
                st = self._dnn(sp)
                bufs = DeviceBuffers(st.buffers)
                self._add("dnn", st.buffers, bufs, pack_tasks(st.tasks, bufs))
        self.rounds = 1 + max([d.sim.p.steps for k, _, _, d in self.items if k == "rl"] or [0])

    def run(self) -> int:
        """One pass over every stream; returns tasks run."""
        before = [self.ctx.tail(i) for i in range(len(self.items))]
        rl = [(i, d) for i, (k, _, _, d) in enumerate(self.items) if k == "rl"]
        for i, (kind, _, _, drv) in enumerate(self.items):
            if kind == "dnn":
                ids, packed = drv
                self.ctx.submit_packed(ids + np.uint32(self.ctx.tail(i)), packed, stream=i)
        for _, d in rl:
            d.submit_plan(d.begin())
        self.ctx.flush()
        self.ctx.sync()
        for t in range(1, self.rounds):
            live = [d for _, d in rl if d.sim.p.steps >= t]
            for d in live:
                d.start_read_nisl()
            torch.cuda.current_stream().synchronize()
            for d in live:
                d.submit_plan(d.sim.step_plan(t - 1, d.nisl()))
            self.ctx.flush()
            self.ctx.sync()
        return sum(self.ctx.tail(i) - b for i, b in enumerate(before))
