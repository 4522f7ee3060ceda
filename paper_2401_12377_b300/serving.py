"""Serving: a request loop over a resident scheduler kernel.

Requests (task streams) arrive over time. A request is admitted when a stream
slot of the context is free and its device memory fits the budget; admitted
requests wait in FIFO order otherwise. Admission allocates the request's
device block, copies its initial bytes from pinned host memory, and publishes
its descriptors to the free slot with one acs_flush: the kernel, resident
since the start, picks them up while other requests are running (continuous
batching: each slot's window lives on the device, and work of all slots
overlaps on the worker CTAs). A request is complete once its slot reports,
through acs_progress, an idle end at or past the end the request was
published with; its latency is that moment minus its arrival (host clock).

Every request is an instance of an entry of a catalogue of request types
(streamgen.serving_catalogue): one device block per instance, holding all its
buffers at fixed offsets, so descriptors are packed once per entry at offset 0
and take the block's base address at admission. Gated-MLP requests share one
copy of the model's weights.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import numpy as np
import torch

from . import acs, harness

ALIGN = 256
SHIFT = np.uint64(1 << 40)


class _AtBases:
    """pack_task's view of buffers placed at given addresses."""

    def __init__(self, base: Dict[str, int], dtype: Dict[str, np.dtype]):
        self.base, self.dtype = base, dtype

    def ptr(self, ref) -> int:
        return self.base[ref.buf] + ref.off * self.dtype[ref.buf].itemsize


def _layout(arrays: Dict[str, np.ndarray]):
    off, pos = {}, 0
    for k in sorted(arrays):
        off[k] = pos
        pos += (arrays[k].nbytes + ALIGN - 1) // ALIGN * ALIGN
    return off, max(pos, ALIGN)


@dataclass
class Entry:
    """A request type prepared for repeated admission."""
    kind: str
    spec: object
    nbytes: int                       # device block size
    init: torch.Tensor                # pinned initial bytes of the block
    ids: np.ndarray                   # task ids 0 .. n-1 (positions relative to the start)
    packed: np.ndarray                # acs_args rows, block pointers relative to 0
    patch: np.ndarray                 # u64 words of `packed` that take the block base
    init_patch: np.ndarray            # u64 words of `init` that take the block base
    results: Dict[str, tuple] = field(default_factory=dict)   # name -> (offset, nbytes, dtype)


def _patch_words(pack_a: np.ndarray, pack_b: np.ndarray) -> np.ndarray:
    wa, wb = pack_a.view(np.uint64), pack_b.view(np.uint64)
    idx = np.nonzero(wa != wb)[0]
    assert np.all(wb[idx] - wa[idx] == SHIFT)
    return idx.astype(np.int64)


def prepare_rl(spec) -> Entry:
    import streamgen as sg
    sim = sg.RLSim(spec.seed, spec.rl)
    p = sim.p
    host = sim.buffers(emit=True)
    sc = sim.scalars()
    arrays = dict(host)
    arrays["cfg"] = np.zeros(harness.EMIT_CFG_DTYPE.itemsize, np.uint8)
    arrays["table"] = sim.ncta_table()
    off, total = _layout(arrays)
    cfg = np.zeros(1, harness.EMIT_CFG_DTYPE)
    for k in ("pos", "vel", "prop", "cont"):
        cfg[k] = off[k]
    for k in ("beta_dt", "slop"):
        cfg[k] = sc["rl_solve"][k]
    for k in ("dt", "gdt", "box"):
        cfg[k] = sc["rl_integrate"][k]
    arrays["cfg"] = cfg.view(np.uint8)
    init = np.zeros(total, np.uint8)
    for k, v in arrays.items():
        b = np.ascontiguousarray(v).view(np.uint8).reshape(-1)
        init[off[k]:off[k] + b.size] = b
    dtypes = {k: v.dtype for k, v in arrays.items()}
    packs = []
    for shift in (0, 1 << 40):
        sim.next_id = 0
        tasks = sim.first_batch()
        if p.steps > 0:
            e = sim.emit_task(0)
            e.scalars.update({"cfg": off["cfg"] + shift, "ncta_table": off["table"] + shift,
                              "steps": np.uint32(p.steps), "chunk": np.uint32(p.chunk)})
            tasks.append(e)
        ids, packed = harness.pack_tasks(tasks, _AtBases({k: o + shift for k, o in off.items()}, dtypes))
        packs.append(packed)
    init_patch = (off["cfg"] // 8 + np.arange(4)).astype(np.int64)   # cfg.pos .. cfg.cont
    res = {k: (off[k], host[k].nbytes, host[k].dtype) for k in ("pos", "vel")}
    return Entry("rl", spec, total, torch.from_numpy(init).pin_memory(), ids, packs[0],
                 _patch_words(packs[0], packs[1]), init_patch, res)


def prepare_dnn(spec, shared_host, shared_dev: Dict[str, int]) -> Entry:
    import streamgen as sg
    st = sg.dnn_stream(spec.seed, batch=spec.dnn_batch, blocks=spec.dnn_blocks,
                       weight_sets=sg.DNN_SERVE_WEIGHT_SETS, shared=shared_host)
    arrays = {k: st.buffers[k] for k in ("h", "t", "u")}
    off, total = _layout(arrays)
    init = np.zeros(total, np.uint8)
    for k, v in arrays.items():
        b = v.view(np.uint8)
        init[off[k]:off[k] + b.size] = b
    dtypes = {k: v.dtype for k, v in st.buffers.items()}
    packs = []
    for shift in (0, 1 << 40):
        base = {k: o + shift for k, o in off.items()}
        base.update(shared_dev)
        ids, packed = harness.pack_tasks(st.tasks, _AtBases(base, dtypes))
        packs.append(packed)
    res = {"h": (off["h"], arrays["h"].nbytes, arrays["h"].dtype)}
    return Entry("dnn", spec, total, torch.from_numpy(init).pin_memory(), ids, packs[0],
                 _patch_words(packs[0], packs[1]), np.zeros(0, np.int64), res)


class Catalogue:
    """Prepared request types plus the shared model weights on the device."""

    def __init__(self, specs, weight_seed: int = 1234):
        import streamgen as sg
        self.specs = specs
        self.shared_host = sg.dnn_weights(weight_seed, sg.DNN_SERVE_WEIGHT_SETS)
        self.shared = {"W": torch.from_numpy(self.shared_host[0]).cuda(),
                       "B": torch.from_numpy(self.shared_host[1]).cuda()}
        dev = {k: int(v.data_ptr()) for k, v in self.shared.items()}
        self.entries: List[Entry] = [prepare_rl(sp) if sp.kind == "rl" else prepare_dnn(sp, self.shared_host, dev)
                                     for sp in specs]
        torch.cuda.current_stream().synchronize()


@dataclass
class _Live:
    idx: int
    entry: Entry
    arrival: float
    block: torch.Tensor
    start: int
    end: int
    admitted: float


def admit_fifo(waiting, free, in_use: int, budget: int, need) -> List[Tuple[int, int]]:
    """Admission, oldest first: the head of the `waiting` queue takes a slot
    from `free` while one is free and its bytes (`need(request)`) fit the
    budget beside `in_use`; the first request that does not fit stops the
    round, so no later request overtakes it. Pops what it admits and returns
    [(request, slot)]."""
    out = []
    while waiting and free:
        nb = need(waiting[0])
        if in_use + nb > budget:
            break
        out.append((waiting.popleft(), free.popleft()))
        in_use += nb
    return out


class Server:
    """The request loop over one resident context (n_streams = slots)."""

    def __init__(self, catalogue: Catalogue, ctx: harness.Context, budget_bytes: int = 20 << 30,
                 readback: bool = False):
        if not ctx.resident:
            raise ValueError("Server needs a resident context (Context(..., resident=True))")
        self.cat, self.ctx = catalogue, ctx
        self.slots = ctx.n_streams
        self.budget = budget_bytes
        # readback: every completed request's results go to pinned host memory
        # (a ring the caller would consume; here only the bytes are counted)
        self.readback = readback
        self._ring = torch.empty(64 << 20, dtype=torch.uint8).pin_memory() if readback else None
        self._ring_pos = 0
        self._cfg_stage = torch.empty((1024, 64), dtype=torch.uint8).pin_memory()
        self._head = np.zeros(self.slots, np.uint32)
        self._idle = np.zeros(self.slots, np.uint32)
        self._tail_max = max(ctx.tail(s) for s in range(self.slots))   # highest slot position
        self.restarts = 0

    def _restart_positions(self) -> None:
        """With no request in the system: end the resident launch, restart
        every slot's positions at 0 (acs_stream_rebase; the library takes
        host-submitted tasks only below 2^31 per stream) and start it again."""
        self.ctx.stop()
        for s in range(self.slots):
            self.ctx.rebase(s)
        self.ctx.start()
        self._tail_max = 0
        self.restarts += 1

    def run(self, arrivals: np.ndarray, kinds: np.ndarray, keep: Optional[set] = None,
            stall_s: float = 30.0) -> dict:
        """Serve requests arriving at `arrivals` (s, from now) of catalogue
        types `kinds`; returns latencies, tasks, throughput and the results of
        the requests named in `keep`."""
        keep = keep or set()
        ctx, cat = self.ctx, self.cat
        n = len(arrivals)
        live: Dict[int, _Live] = {}
        free = collections.deque(range(self.slots))
        waiting = collections.deque()
        in_use = 0
        peak_in_use = 0
        lat = np.zeros(n)
        queued = np.zeros(n)
        tasks = np.zeros(n, np.int64)
        results = {}
        pending_results = []
        done = 0
        nxt = 0
        h2d = d2h = 0
        busy_time = 0.0
        last_t = None
        stream = torch.cuda.current_stream()
        t0 = time.perf_counter()
        first_arrival = t0 + float(arrivals[0]) if n else t0
        last_done = t0
        last_move = t0
        while done < n:
            now = time.perf_counter()
            if live and now - last_move > stall_s:
                raise RuntimeError(f"serving stalled: {len(live)} requests made no progress for {stall_s} s")
            if last_t is not None:
                busy_time += (now - last_t) * len(live)
            last_t = now
            rel = now - t0
            while nxt < n and arrivals[nxt] <= rel:
                waiting.append(nxt)
                nxt += 1
            # completions
            if live:
                ctx.progress(self._head, self._idle)
                for s in list(live):
                    L = live[s]
                    if (int(self._idle[s]) - L.end) & 0xFFFFFFFF >= 0x80000000:
                        continue                  # idle end still before the request's end
                    t = time.perf_counter()
                    lat[L.idx] = t - (t0 + float(arrivals[L.idx]))
                    tail = ctx.tail(s)
                    tasks[L.idx] = tail - L.start
                    self._tail_max = max(self._tail_max, tail)
                    if self.readback:
                        for name, (o, nb, dt) in L.entry.results.items():
                            if self._ring_pos + nb > self._ring.numel():
                                self._ring_pos = 0
                            self._ring[self._ring_pos:self._ring_pos + nb].copy_(L.block[o:o + nb], non_blocking=True)
                            self._ring_pos += nb
                            d2h += nb
                    if L.idx in keep:
                        outs = {}
                        for name, (o, nb, dt) in L.entry.results.items():
                            h = torch.empty(nb, dtype=torch.uint8).pin_memory()
                            h.copy_(L.block[o:o + nb], non_blocking=True)
                            outs[name] = (h, dt)
                        pending_results.append((L.idx, outs))
                    in_use -= L.entry.nbytes
                    del live[s]
                    free.append(s)
                    done += 1
                    last_done = last_move = t
            # a slot past harness.REBASE_AT: restart the positions while nothing is in flight
            if not live and not waiting and self._tail_max >= harness.REBASE_AT:
                self._restart_positions()
            # admissions, oldest first
            batch = []
            for i, s in admit_fifo(waiting, free, in_use, self.budget,
                                   lambda r: cat.entries[int(kinds[r])].nbytes):
                e = cat.entries[int(kinds[i])]
                blk = torch.empty(e.nbytes, dtype=torch.uint8, device="cuda")
                base = np.uint64(blk.data_ptr())
                packed = e.packed.copy()
                packed.view(np.uint64)[e.patch] += base
                blk.copy_(e.init, non_blocking=True)
                if e.init_patch.size:
                    st = self._cfg_stage[len(batch) % len(self._cfg_stage)]
                    w = e.init[e.init_patch[0] * 8:(e.init_patch[-1] + 1) * 8].numpy().view(np.uint64) + base
                    st[:w.nbytes].copy_(torch.from_numpy(w.view(np.uint8)))
                    o = int(e.init_patch[0]) * 8
                    blk[o:o + w.nbytes].copy_(st[:w.nbytes], non_blocking=True)
                in_use += e.nbytes
                h2d += e.nbytes + 320 * len(e.ids)
                peak_in_use = max(peak_in_use, in_use)
                batch.append((i, s, e, blk, packed))
                queued[i] = time.perf_counter() - (t0 + float(arrivals[i]))
            if batch:
                stream.synchronize()          # the blocks' bytes are on the device
                ta = time.perf_counter()
                for i, s, e, blk, packed in batch:
                    start = ctx.tail(s)
                    ctx.submit_packed(e.ids + np.uint32(start), packed, stream=s)
                    live[s] = _Live(i, e, float(arrivals[i]), blk, start, start + len(e.ids), ta)
                ctx.flush()
                last_move = time.perf_counter()
        stream.synchronize()
        for i, outs in pending_results:
            results[i] = {k: h.numpy().view(dt).copy() for k, (h, dt) in outs.items()}
        span = last_done - first_arrival
        return {"latency_s": lat, "queue_s": queued, "tasks": tasks, "span_s": span,
                "tasks_per_s": float(tasks.sum()) / span if span > 0 else 0.0,
                "mean_in_flight": busy_time / max(last_done - t0, 1e-9),
                "peak_bytes": peak_in_use, "h2d_bytes": h2d, "d2h_bytes": d2h, "results": results}
