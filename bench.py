#!/usr/bin/env python
"""Benchmark of the window scheduler on the rigid-sphere RL-simulation stream.

One bench step = one complete run of the stream: 256 environments x 32 spheres,
50 simulation steps, window 32, about 300 small tasks (1-16 CTAs) per
simulation step whose task graph depends on the simulated contacts (island
counts the broadphase tasks compute decide the next step's tasks).

The method runs it with device-side emission: the host submits the first
broadphase batch and an emit task once; emit tasks append each next step's
tasks on the device; one flush, one persistent launch, one sync per run. The
host-driven arm runs the same scheduler with one flush per simulation step
(the host reads back the 1 KiB of island counts and submits the next batch),
as do the in-order and CUDA-graph arms, which cannot emit on the device.

Prints ONE JSON line (rank 0). Arms measured on the same box and workload:
  value                  window scheduler, device-side emission
  window_host_driven     window scheduler, one flush per simulation step
  inorder                one kernel launch per task on one stream
  graph_launch           CUDA graph of each batch's full DAG, launch time only
  graph_with_build       same, including host DAG build + instantiate
  sw_host_scheduler      the paper's software scheduler (host window, 8 threads x 1 stream)
``--impl reference`` times the CPU oracle (in-order executor) instead.

Timing: CUDA events on the library's stream around each bench step, L2
flushed (512 MiB write) between timed steps, W >= 3 warm-up steps; nvidia-smi
clocks sampled during the timed region.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "tasks/s & step-time speedup vs in-order stream + CUDA graph; p50/p99 latency"
WORKLOAD = "rigid-sphere RL-sim stream: 256 envs x 32 spheres, 50 steps, window 32, ~300 tasks/step of 1-16 CTAs"
WORKLOAD_DNN = ("dynamic DNN: gated residual MLP, hidden 256, 24 blocks, shared weights; {per_b} inputs for each "
                "batch size 1, 2, 4, 8, one flush per input, window 32")
WORKLOAD_STATIC = ("static irregular DAG: randomly wired network, 3 stages x 32 nodes (GEMV 256x256 of 1-8 CTAs, "
                   "bias+ReLU, input aggregation), 411 tasks per input, 100 inputs per step, window 32")
WORKLOAD_SERVING = ("serving: Poisson arrivals of rigid-sphere (64 envs, device-side emission) / gated-MLP "
                    "(batch 1-8, shared weights) requests of 100-5000 tasks, 20 GB budget, resident kernel")
WORKLOAD_BATCHED = ("batched: 64 independent streams (alternating rigid-sphere 64 envs x 32 spheres / gated "
                    "residual MLP hidden 256, batch 1-8), lengths log-uniform in [100, 5000] tasks, one launch")


def parse():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["acs", "reference"], default="acs")
    ap.add_argument("--workload", choices=["rlsim", "dnn", "static", "batched", "serving"], default="rlsim",
                    help="rlsim: one rigid-sphere stream (default); batched: 64 independent streams in one "
                         "launch; serving: Poisson arrivals over a resident kernel (steps = seconds of arrivals)")
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: mean arrivals per second")
    ap.add_argument("--slots", type=int, default=64, help="serving: stream slots (concurrent requests)")
    ap.add_argument("--window", type=int, default=0, help="window size (default: 32, or autotuned for batched)")
    ap.add_argument("--cta-slots", type=int, default=0)
    ap.add_argument("--no-tune", action="store_true", help="batched: skip the autotuner")
    ap.add_argument("--window-study", action="store_true",
                    help="rlsim: also time windows 8..64, ring and free-slot (span 64)")
    ap.add_argument("--no-baselines", action="store_true", help="skip the in-order / graph arms")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--headline-only", action="store_true",
                    help="rlsim: skip the compact runs of the other workloads (tiny, dnn, batched, serving)")
    ap.add_argument("--serving-seconds", type=float, default=2.0,
                    help="seconds of arrivals in the compact serving run of the default benchmark")
    ap.add_argument("--lookahead", type=int, default=None,
                    help="window mode: dispatch lookahead for every context (default: the library's, "
                         "min(2 window, 64 - window); 0 turns dispatch ahead off)")
    return ap.parse_args()


def effective_lookahead(window: int, span: int = 0, requested=None, n_streams: int = 1) -> int:
    """The dispatch lookahead a window-mode context runs with (as acs_init resolves it)."""
    if requested is None:
        return 0 if (span or n_streams > 1) else min(2 * window, 64 - window)
    return requested


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one persistent
# launch of the default workload, from one ncu capture of that launch; it
# applies only while the kernel's sources hash to the value it was taken with
# (else traffic is null).
KERNEL_SOURCES = ("paper_2401_12377_b300/csrc/acs_kernels.cu", "paper_2401_12377_b300/csrc/acs_bodies.cuh",
                  "paper_2401_12377_b300/csrc/acs_internal.h")
TRAFFIC_RLSIM = {"bytes_per_launch": 3698176, "sources_sha1": "6a70a08a9d4e3f0cfc1029c5fc521386a49e70b3"}


def kernel_sources_sha1() -> str:
    import hashlib
    h = hashlib.sha1()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def ranks():
    """(world, rank, local rank) from the launcher's environment (1, 0, 0 alone)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over all ranks (x itself without a process group)."""
    if not dist:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: float, max_seconds: float) -> float:
    """Units all ranks processed over the slowest rank's time (weak scaling:
    every rank processes the same amount of independent work)."""
    return world * units_per_rank / max_seconds


def rl_params(steps=50):
    import streamgen as sg
    return sg.RLParams(n_env=256, steps=steps)


# ---- CPU oracle ---------------------------------------------------------------------

def cpu_oracle_rate(budget_s: float = 10.0, max_runs: int = 20):
    """The oracle's in-order executor on full runs of the same stream."""
    import streamgen as sg
    from oracle import execute
    execute.build_c()
    tasks = 0
    runs = 0
    t0 = time.perf_counter()
    while runs < max_runs and (time.perf_counter() - t0) < budget_s:
        t, _, _ = execute.run_rlsim(sg.RLSim(1 + runs, rl_params()))
        tasks += len(t)
        runs += 1
    dt = time.perf_counter() - t0
    return {"value": tasks / dt, "unit": "tasks/s", "cores": 1, "kind": "oracle",
            "sample": f"{runs} full runs of the stream (256 envs x 32 spheres x 50 steps, {tasks} tasks), "
                      f"single-threaded numpy + C bodies, {dt:.1f} s"}


def oracle_batch(seed: int, limit_s: float = 1e9):
    """The oracle over the streams of one batch (in order, stream by stream),
    stopping after the stream that crosses limit_s; returns (tasks, streams, s)."""
    import streamgen as sg
    from oracle import execute
    execute.build_c()
    tasks = streams = 0
    t0 = time.perf_counter()
    for sp in sg.batched_specs(seed):
        if sp.kind == "rl":
            t, _, _ = execute.run_rlsim(sg.RLSim(sp.seed, sp.rl), emit=True)
        else:
            st = sg.dnn_stream(sp.seed, batch=sp.dnn_batch, blocks=sp.dnn_blocks,
                               weight_sets=min(sp.dnn_blocks, 24))
            execute.run_inorder(st.buffers, st.tasks)
            t = st.tasks
        tasks += len(t)
        streams += 1
        if time.perf_counter() - t0 > limit_s:
            break
    return tasks, streams, time.perf_counter() - t0


def oracle_serving(seed: int, n_req: int, rate: float, limit_s: float, offset: int = 0):
    """The oracle over serving requests in arrival order (from request
    offset * 97), stopping after the request that crosses limit_s; returns
    (tasks, requests, s)."""
    import streamgen as sg
    from oracle import execute
    execute.build_c()
    cat = sg.serving_catalogue(seed)
    shared = sg.dnn_weights(1234, sg.DNN_SERVE_WEIGHT_SETS)
    _, kinds = sg.poisson_arrivals(seed, n_req, rate, len(cat))
    tasks = reqs = 0
    t0 = time.perf_counter()
    for i in range(len(kinds)):
        sp = cat[int(kinds[(i + offset * 97) % len(kinds)])]
        if sp.kind == "rl":
            t, _, _ = execute.run_rlsim(sg.RLSim(sp.seed, sp.rl), emit=True)
        else:
            st = sg.dnn_stream(sp.seed, batch=sp.dnn_batch, blocks=sp.dnn_blocks,
                               weight_sets=sg.DNN_SERVE_WEIGHT_SETS, shared=shared)
            execute.run_inorder(st.buffers, st.tasks)
            t = st.tasks
        tasks += len(t)
        reqs += 1
        if time.perf_counter() - t0 > limit_s:
            break
    return tasks, reqs, time.perf_counter() - t0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import streamgen as sg
    from oracle import execute
    execute.build_c()
    if args.workload == "static":
        st = sg.random_wire_stream(1)
        execute.run_inorder(st.buffers, st.tasks)
        times = []
        for k in range(args.steps):
            t0 = time.perf_counter()
            for i in range(10):                      # a bounded sample: 10 of the step's 100 inputs
                execute.run_inorder(st.buffers, st.tasks)
            times.append(time.perf_counter() - t0)
        tasks = 10 * args.steps * len(st.tasks)
        value = tasks / sum(times)
        line = {"metric": METRIC, "value": value, "unit": "tasks/s", "n_gpus": args.gpus, "steps": args.steps,
                "warmup": 1, "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "impl": "reference",
                "config": {"workload": WORKLOAD_STATIC, "l2": "n/a (CPU)"},
                "cpu_baseline": {"value": value, "unit": "tasks/s", "cores": 1, "kind": "oracle",
                                 "sample": "each step 10 of the 100 inputs, single-threaded"},
                "e2e": {"value": value, "unit": "tasks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    if args.workload == "dnn":
        shared = sg.dnn_weights(7919, 24)
        streams = [sg.dnn_stream(100000 + b * 1000 + i, batch=b, blocks=24, weight_sets=24, shared=shared)
                   for b in (1, 2, 4, 8) for i in range(100)]
        times, tasks = [], 0
        for k in range(args.steps):
            t0 = time.perf_counter()
            n = 0
            for st in streams[k * 7 % 100::25]:      # a bounded sample: 16 inputs of every batch size
                execute.run_inorder(st.buffers, st.tasks)
                n += len(st.tasks)
            times.append(time.perf_counter() - t0)
            tasks += n
        value = tasks / sum(times)
        line = {"metric": METRIC, "value": value, "unit": "tasks/s", "n_gpus": args.gpus, "steps": args.steps,
                "warmup": 0, "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "impl": "reference",
                "config": {"workload": WORKLOAD_DNN, "l2": "n/a (CPU)"},
                "cpu_baseline": {"value": value, "unit": "tasks/s", "cores": 1, "kind": "oracle",
                                 "sample": "each step 16 of the 400 inputs (4 of each batch size), single-threaded"},
                "e2e": {"value": value, "unit": "tasks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    if args.workload == "serving":
        n_req = int(args.rate * args.steps)
        times, tasks = [], 0
        for k in range(args.steps):
            t, _, dt = oracle_serving(1, n_req, args.rate, limit_s=20.0, offset=k)
            times.append(dt)
            tasks += t
        s_tot = sum(times)
        value = tasks / s_tot
        line = {"metric": METRIC, "value": value, "unit": "tasks/s", "n_gpus": args.gpus, "steps": args.steps,
                "warmup": 0, "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "impl": "reference",
                "config": {"workload": WORKLOAD_SERVING, "l2": "n/a (CPU)"},
                "cpu_baseline": {"value": value, "unit": "tasks/s", "cores": 1, "kind": "oracle",
                                 "sample": f"requests in arrival order, about 20 s of in-order execution per step "
                                           f"({tasks} tasks in all), single-threaded"},
                "e2e": {"value": value, "unit": "tasks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    if args.workload == "batched":
        oracle_batch(100)   # warm-up: imports, compiled bodies
        times, tasks = [], 0
        for k in range(args.steps):
            tasks, _, dt = oracle_batch(1 + k)
            times.append(dt)
        ms = 1e3 * statistics.mean(times)
        value = tasks / (ms / 1e3)
        line = {"metric": METRIC, "value": value, "unit": "tasks/s", "n_gpus": args.gpus, "steps": args.steps,
                "warmup": 1, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "impl": "reference",
                "config": {"workload": WORKLOAD_BATCHED, "l2": "n/a (CPU)"},
                "cpu_baseline": {"value": value, "unit": "tasks/s", "cores": 1, "kind": "oracle",
                                 "sample": f"each step one full batch of 64 streams ({tasks} tasks), "
                                           "single-threaded"},
                "e2e": {"value": value, "unit": "tasks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    for w in range(args.warmup):
        execute.run_rlsim(sg.RLSim(100 + w, rl_params(steps=5)))
    times, tasks = [], 0
    for k in range(args.steps):
        t0 = time.perf_counter()
        t, _, _ = execute.run_rlsim(sg.RLSim(1 + k, rl_params()))
        times.append(time.perf_counter() - t0)
        tasks = len(t)
    ms = 1e3 * statistics.mean(times)
    value = tasks / (ms / 1e3)
    cores = 1
    line = {"metric": METRIC, "value": value, "unit": "tasks/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "tasks/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step one full run of the stream ({tasks} tasks), single-threaded"},
            "e2e": {"value": value, "unit": "tasks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- clocks ---------------------------------------------------------------------------

REASONS = ["clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
           "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]


class ClockSampler:
    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = "index,clocks.sm,clocks.max.sm,power.draw," + ",".join(REASONS)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except OSError:
            rows = []
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        sm, mx, reasons = [], None, set()
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for name, v in zip(REASONS, r[4:8]):
                    if v.strip().lower() == "active":
                        reasons.add(name.split(".")[-1])
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---- GPU arms ----------------------------------------------------------------------------

class RLBench:
    """One mode (window / inorder / graph) on one device state."""

    def __init__(self, mode, seed, window, cta_slots, timing=True, emit=False, span=0, traced=False,
                 lookahead=None):
        import torch
        import streamgen as sg
        from paper_2401_12377_b300 import harness
        self.torch = torch
        self.sim = sg.RLSim(seed, rl_params())
        host = self.sim.buffers(emit=emit)
        self.bufs = harness.DeviceBuffers(host)
        self.pristine = {k: v.clone() for k, v in self.bufs.t.items()}
        self.host_pinned = {k: torch.from_numpy(v.view("uint8").copy()).pin_memory() for k, v in host.items()}
        self.ctx = harness.Context(window, mode=mode, timing=timing, capacity=1 << 14, cta_slots=cta_slots,
                                   span=span, log=traced, trace=traced, lookahead=lookahead)
        self.emit = emit
        self.driver = (harness.RLEmitDriver if emit else harness.RLDriver)(self.sim, self.bufs, self.ctx)
        self.mode = mode

    def reset_device(self):
        for k, t in self.bufs.t.items():
            t.copy_(self.pristine[k], non_blocking=True)

    def upload_host(self):
        for k, t in self.bufs.t.items():
            t.copy_(self.host_pinned[k], non_blocking=True)

    def run_once(self, latencies=None):
        """One full stream; returns its number of tasks."""
        if self.emit:
            t0 = time.perf_counter()
            n = self.driver.run()
            if latencies is not None:
                latencies.append(time.perf_counter() - t0)
            return n
        before = self.ctx.stats()["tasks_submitted"]
        plan = self.sim.first_plan()
        steps = self.sim.p.steps
        for t in range(steps + 1):
            t0 = time.perf_counter()
            if t > 0:
                plan = self.sim.step_plan(t - 1, self.driver.read_nisl())
            self.ctx.submit_packed(*self.driver.pack(plan))
            self.ctx.flush()
            self.ctx.sync()
            if latencies is not None:
                latencies.append(time.perf_counter() - t0)
        return self.ctx.stats()["tasks_submitted"] - before


def l2_flush(buf):
    """Between timed steps: a 512 MiB write (or the given flush function)."""
    if buf is None:
        return
    if callable(buf):
        buf()
    else:
        buf.zero_()


# Warm-up runs go on for at least this long as well as for the requested number
# of steps: the host CPU needs a few hundred milliseconds of load to come back to
# full clock after an idle spell (measured on the B300 hosts: a run's host work,
# submit + flush, takes 25 us at full clock and 140 us right after a 2 s sleep;
# 50 ms of load recovers half of that, 500 ms all of it).
HOST_WARM_S = 0.5


def time_arm(arm, steps, warmup, flush_buf, latencies=None):
    torch = arm.torch
    k, t_warm = 0, time.perf_counter() + HOST_WARM_S
    while k < warmup or time.perf_counter() < t_warm:
        arm.reset_device()
        arm.run_once()
        k += 1
    torch.cuda.current_stream().synchronize()
    st0 = arm.ctx.stats()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    tasks = 0
    wall = 0.0
    for k in range(steps):
        arm.reset_device()
        l2_flush(flush_buf)
        torch.cuda.current_stream().synchronize()
        w0 = time.perf_counter()
        ev[k][0].record()
        tasks += arm.run_once(latencies)
        ev[k][1].record()
        torch.cuda.current_stream().synchronize()
        wall += time.perf_counter() - w0
    ms = [a.elapsed_time(b) for a, b in ev]
    st1 = arm.ctx.stats()
    fixed = ("cta_slots", "grid")
    delta = {k: (st1[k] - st0[k]) if isinstance(st1[k], (int, float)) and k not in fixed else st1[k] for k in st1}
    return {"ms": ms, "tasks": tasks, "wall_s": wall, "stats": delta}


def critical_path(ctx, stream: int, first: int, n: int):
    """Longest chain of a stream's device-logged window DAG (every conflicting
    predecessor within the ring span), each task weighted by its body time in a
    traced run (first CTA start to last CTA end). Any legal schedule respects
    these edges, so the chain bounds the run's makespan from below for zero
    scheduling overhead. Returns (us, tasks on the chain)."""
    span = ctx.span
    masks, _, _ = ctx.log(stream, first, n)
    tr = ctx.trace(stream, first, n).astype(np.int64)
    body = np.maximum(tr[:, 3] - tr[:, 2], 0) / 1e3
    fin = np.zeros(n)
    cnt = np.zeros(n, np.int64)
    for j in range(n):
        m, seq = int(masks[j]), first + j
        best, bc = 0.0, 0
        while m:
            b = (m & -m).bit_length() - 1
            m &= m - 1
            i = j - (seq - b) % span           # the predecessor in slot b
            if 0 <= i < j and fin[i] > best:
                best, bc = fin[i], cnt[i]
        fin[j] = best + body[j]
        cnt[j] = bc + 1
    k = int(np.argmax(fin)) if n else 0
    return (float(fin[k]), int(cnt[k])) if n else (0.0, 0)


def window_bound(ctx, first: int, n: int, window: int, emitter) -> dict:
    """Makespan of an as-soon-as-possible schedule of a logged, traced stream
    under the window rule with no scheduling overhead: a task starts once its
    logged conflicting predecessors and every task `window` or more positions
    back have ended (a window holds `window` tasks), and an emitted task once
    its emit task has started (optimistic) or ended. Tasks take their traced
    body times. emitter[j] is the position of the emit task that appended
    task j, or -1. Returns the two makespans in microseconds."""
    span = ctx.span
    masks, _, _ = ctx.log(0, first, n)
    tr = ctx.trace(0, first, n).astype(np.int64)
    body = np.maximum(tr[:, 3] - tr[:, 2], 0) / 1e3
    preds = []
    for j in range(n):
        m, seq, p = int(masks[j]), first + j, []
        while m:
            b = (m & -m).bit_length() - 1
            m &= m - 1
            i = j - (seq - b) % span
            if 0 <= i < j:
                p.append(i)
        preds.append(p)
    out = {}
    for release in ("start", "end"):
        S, E, runmax = np.zeros(n), np.zeros(n), np.zeros(n)
        for j in range(n):
            t = max((E[i] for i in preds[j]), default=0.0)
            if j >= window:
                t = max(t, runmax[j - window])
            e = emitter[j]
            if e >= 0:
                t = max(t, S[e] if release == "start" else E[e])
            S[j], E[j] = t, t + body[j]
            runmax[j] = max(runmax[j - 1] if j else 0.0, E[j])
        out[release] = float(E.max()) if n else 0.0
    return out


def task_segments(rows):
    """Read and write segments of packed task rows, as the library resolves
    them (acs_get_addresses)."""
    from paper_2401_12377_b300 import acs
    return [acs.acs_get_addresses(acs.acs_args.from_buffer_copy(r.tobytes())) for r in rows]


def critical_path_full(segs, body_us):
    """Longest chain of a stream's full dependency DAG (every read-after-write,
    write-after-read and write-after-write pair, however far apart), tasks
    weighted by body_us. Per byte it keeps the finish time of its last writer
    and the latest finish of its readers since: a read waits for the writer, a
    write for both, and older conflicts are implied through them. Returns
    (us, tasks on the chain)."""
    import bisect
    whole = (0, (1 << 64) - 1)
    ranges = sorted((s, s + n) for rd, wr in segs for s, n in list(rd) + list(wr) if n and (s, n) != whole)
    merged = []
    for a, b in ranges:
        if merged and a <= merged[-1][1]:
            merged[-1][1] = max(merged[-1][1], b)
        else:
            merged.append([a, b])
    starts = [a for a, _ in merged]
    base, off = [], 0
    for a, b in merged:
        base.append(off)
        off += b - a
    lw, rd = np.zeros(off), np.zeros(off)                  # finish times (us)
    lwc, rdc = np.zeros(off, np.int64), np.zeros(off, np.int64)   # chain lengths

    def slices(seg_list):
        out = []
        for s, n in seg_list:
            if (s, n) == whole:
                out.append(slice(0, off))
            elif n:
                k = bisect.bisect_right(starts, s) - 1
                lo = base[k] + (s - merged[k][0])
                out.append(slice(lo, lo + n))
        return out

    best_all, cnt_all = 0.0, 0
    for (r, w), body in zip(segs, body_us):
        rs, ws = slices(r), slices(w)
        best, bc = 0.0, 0
        for sl, arrs in [(x, ((lw, lwc),)) for x in rs] + [(x, ((lw, lwc), (rd, rdc))) for x in ws]:
            for arr, carr in arrs:
                if sl.stop > sl.start:
                    k = int(np.argmax(arr[sl]))
                    if arr[sl][k] > best:
                        best, bc = float(arr[sl][k]), int(carr[sl][k])
        f, c = best + float(body), bc + 1
        for sl in rs:
            upd = rd[sl] < f
            rd[sl][upd] = f
            rdc[sl][upd] = c
        for sl in ws:
            lw[sl], lwc[sl], rd[sl], rdc[sl] = f, c, 0.0, 0
        if f > best_all:
            best_all, cnt_all = f, c
    return best_all, cnt_all


def time_e2e(arm, steps):
    """Host buffers in, results out: H2D of the initial state from pinned
    memory, the run, D2H of the final pos / vel, all inside CUDA events."""
    torch = arm.torch
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out_pos = torch.empty_like(arm.bufs.t["pos"], device="cpu").pin_memory()
    out_vel = torch.empty_like(arm.bufs.t["vel"], device="cpu").pin_memory()

    def step():
        arm.upload_host()
        n = arm.run_once()
        out_pos.copy_(arm.bufs.t["pos"], non_blocking=True)
        out_vel.copy_(arm.bufs.t["vel"], non_blocking=True)
        return n

    k, t_warm = 0, time.perf_counter() + HOST_WARM_S      # untimed warm-up, as for every arm
    while k < 1 or time.perf_counter() < t_warm:
        step()
        k += 1
    tasks = 0
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(steps):
        tasks += step()
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    h2d_inputs = sum(t.numel() for t in arm.host_pinned.values())
    n_flush = 1 if arm.emit else arm.sim.p.steps + 1
    desc_bytes = (tasks // steps) * 320
    d2h = out_pos.numel() + out_vel.numel() + (0 if arm.emit else arm.sim.p.steps * arm.sim.p.n_env * 4)
    return {"value": (tasks / steps) / (ms / 1e3), "unit": "tasks/s",
            "h2d_bytes_per_step": int(h2d_inputs + desc_bytes), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": ms, "flushes_per_step": n_flush}


class BatchArm:
    """time_arm adapter for a batch (BatchedWorkload or BatchedHostDriven)."""

    def __init__(self, torch, wl, ctx):
        self.torch, self.wl, self.ctx = torch, wl, ctx

    def reset_device(self):
        self.wl.reset()

    def run_once(self, latencies=None):
        t0 = time.perf_counter()
        n = self.wl.run()
        if latencies is not None:
            latencies.append(time.perf_counter() - t0)
        return n


_PINNED_FLUSH = None


def copy_engine_flush(torch, flush_buf):
    """An L2 flush that needs no SM: a host-to-device copy of 512 MiB (while
    a resident kernel holds every SM, a fill kernel would wait for it)."""
    global _PINNED_FLUSH
    if _PINNED_FLUSH is None:
        _PINNED_FLUSH = torch.empty(flush_buf.numel(), dtype=torch.uint8).pin_memory()
    return lambda: flush_buf.copy_(_PINNED_FLUSH, non_blocking=True)


class DNNInputs:
    """The dynamic-DNN workload: inputs of a gated MLP with shared weights,
    run one input per flush (the DAG of each input depends on its gates).
    resident: the scheduler kernel stays on the device and every input is
    published to it (no launch per input); the activations are reset from
    pinned host memory (a device-side copy would wait for the kernel)."""

    def __init__(self, torch, mode, window, cta_slots, seed=1, per_b=100, resident=False):
        import streamgen as sg
        from paper_2401_12377_b300 import harness
        self.torch, self.resident = torch, resident
        shared = sg.dnn_weights(seed * 7919, 24)
        self.shared = shared
        self.streams = [sg.dnn_stream(seed * 100000 + b * 1000 + i, batch=b, blocks=24, weight_sets=24,
                                      shared=shared, window=window)
                        for b in (1, 2, 4, 8) for i in range(per_b)]
        wdev = {"W": torch.from_numpy(shared[0]).cuda(), "B": torch.from_numpy(shared[1]).cuda()}
        self.bufs, self.packed = [], []
        for st in self.streams:
            acts = {k: st.buffers[k] for k in ("h", "t", "u")}
            b = harness.DeviceBuffers(acts)
            b.t.update(wdev)
            b.base.update({k: int(v.data_ptr()) for k, v in wdev.items()})
            b.dtype.update({"W": np.dtype(np.float32), "B": np.dtype(np.float32)})
            self.bufs.append(b)
            self.packed.append(harness.pack_tasks(st.tasks, b))
        if resident:
            self.pristine = [{k: torch.from_numpy(st.buffers[k].view(np.uint8).copy()).pin_memory()
                              for k in ("h", "t", "u")} for st in self.streams]
        else:
            self.pristine = [{k: b.t[k].clone() for k in ("h", "t", "u")} for b in self.bufs]
        torch.cuda.current_stream().synchronize()
        self.ctx = harness.Context(window, mode=mode, timing=True, capacity=1 << 12, cta_slots=cta_slots,
                                   resident=resident)
        self.n_tasks = sum(len(st.tasks) for st in self.streams)

    def reset_device(self):
        for b, p in zip(self.bufs, self.pristine):
            for k, v in p.items():
                b.t[k].copy_(v, non_blocking=True)

    def run_once(self, latencies=None):
        if self.resident:
            self.torch.cuda.current_stream().synchronize()   # resets are on the device
        n = 0
        for ids, rows in self.packed:
            t0 = time.perf_counter()
            start = self.ctx.tail(0)
            self.ctx.submit_packed(ids + np.uint32(start), rows)
            self.ctx.flush()
            self.ctx.sync()
            if latencies is not None:
                latencies.append(time.perf_counter() - t0)
            n += len(ids)
        return n


def per_input_bench(args, torch, dist, world, rank, peaks, peak_src, flush_buf, make, workload, extra_l2,
                    baselines, e2e_fn, oracle_fn):
    """One input per flush, each with a persistent launch of its own (the
    line's value); beside it the same flushes published to a resident kernel,
    then the baselines."""
    W = args.window or 32
    seed = 1 + rank
    arm = make("window", W, seed, False)
    lat = []
    if dist:
        dist.barrier()
    with ClockSampler(torch.cuda.current_device()) as clk:
        res = time_arm(arm, args.steps, args.warmup, flush_buf, lat)
    clocks = clk.summary()
    ms_step = statistics.mean(res["ms"])
    max_ms = max_over_ranks(ms_step, dist, "cuda")
    tps = res["tasks"] / args.steps
    lus = np.sort(np.array(lat)) * 1e6
    st = res["stats"]
    launches = st["launches"]
    avg_launch_s = (st["kernel_ms"] / 1e3) / max(1, launches)
    bpl = st["device_seg_bytes"] / max(1, launches)
    achieved = bpl / avg_launch_s / 1e9 if avg_launch_s > 0 else 0.0
    peak = float(peaks.get("hbm_gbs", 6400.0))
    e2e = e2e_fn(arm)
    arm.ctx.close()
    line = {"metric": METRIC, "value": whole_job_rate(world, tps, max_ms / 1e3), "unit": "tasks/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": max_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload, "window": W, "lookahead": effective_lookahead(W, 0, args.lookahead),
                       "inputs_per_step": len(lat) // args.steps,
                       "tasks_per_step": tps, "cta_slots": st.get("cta_slots"),
                       "mode": "window scheduler, one flush and one persistent launch per input",
                       "l2": "flushed between timed steps (512 MiB write)" + extra_l2,
                       "parallelism": f"replicas x{world}" if world > 1 else "one GPU"},
            "input_latency_us": {"p50": float(lus[len(lus) // 2]), "p99": float(lus[int(0.99 * (len(lus) - 1))])},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "kernel": "acs_persistent_kernel", "peak_source": peak_src,
                         "algorithmic_bytes_per_launch": bpl, "avg_launch_us": avg_launch_s * 1e6},
            "gpu_launches": int(launches), "clocks": clocks, "e2e": e2e}
    k = max(1, min(args.steps, 3))
    # the same inputs published to a resident kernel (no launch per input); its
    # publication path (copy engine, completion seen by the host, device
    # mirror) costs tens of microseconds per input
    flush_ce = copy_engine_flush(torch, flush_buf)
    ra = make("window", W, seed, True)
    rlat = []
    rr = time_arm(ra, k, 1, flush_ce, rlat)
    ra.ctx.close()
    rms = statistics.mean(rr["ms"])
    rl = np.sort(np.array(rlat)) * 1e6
    line["resident_per_input"] = {"tasks_per_s": (rr["tasks"] / k) / (rms / 1e3), "ms_per_step": rms,
                                  "input_latency_us": {"p50": float(rl[len(rl) // 2]),
                                                       "p99": float(rl[int(0.99 * (len(rl) - 1))])}}
    if not args.no_baselines:
        baselines(line, ms_step, k, W, seed)
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = oracle_fn(arm)
    elif rank == 0:
        line["cpu_baseline"] = None
    return line


def bench_dnn(args, torch, dist, world, rank, peaks, peak_src, flush_buf):
    def make(mode, W, seed, resident):
        return DNNInputs(torch, mode, W, args.cta_slots, seed, per_b=getattr(args, "dnn_per_b", 100),
                         resident=resident)

    def baselines(line, ms_step, k, W, seed):
        for mode in ("inorder", "graph", "sw"):
            b = make(mode, W, seed, False)
            r = time_arm(b, k, 1, flush_buf)
            ms = statistics.mean(r["ms"])
            entry = {"tasks_per_s": (r["tasks"] / k) / (ms / 1e3), "ms_per_step": ms,
                     "kernel_ms_per_step": r["stats"]["kernel_ms"] / k}
            if mode == "graph":
                entry["host_build_instantiate_ms_per_step"] = (r["stats"]["graph_build_ms"]
                                                               + r["stats"]["graph_instantiate_ms"]) / k
                line["graph_with_build"] = entry
                line["graph_launch"] = {"tasks_per_s": (r["tasks"] / k) / (entry["kernel_ms_per_step"] / 1e3),
                                        "device_ms_per_step": entry["kernel_ms_per_step"]}
                line["speedup_vs_graph_with_build"] = ms / ms_step
                line["speedup_vs_graph_launch_only"] = entry["kernel_ms_per_step"] / ms_step
            elif mode == "sw":
                line["sw_host_scheduler"] = entry
                line["speedup_vs_sw_host_scheduler"] = ms / ms_step
            else:
                line["inorder"] = entry
                line["speedup_vs_inorder"] = ms / ms_step
            b.ctx.close()

    def e2e(arm):
        # each input's activations in from pinned memory, its output h back
        pin_in = [{k: torch.from_numpy(st.buffers[k].view(np.uint8).copy()).pin_memory() for k in ("h", "t", "u")}
                  for st in arm.streams]
        pin_out = [torch.empty(b.t["h"].numel(), dtype=torch.uint8).pin_memory() for b in arm.bufs]
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.current_stream().synchronize()
        ev0.record()
        h2d = d2h = n = 0
        for (ids, rows), b, pi, po in zip(arm.packed, arm.bufs, pin_in, pin_out):
            for k, v in pi.items():
                b.t[k].copy_(v, non_blocking=True)
                h2d += v.numel()
            if arm.resident:
                torch.cuda.current_stream().synchronize()
            arm.ctx.submit_packed(ids + np.uint32(arm.ctx.tail(0)), rows)
            arm.ctx.flush()
            arm.ctx.sync()
            po.copy_(b.t["h"], non_blocking=True)
            d2h += po.numel()
            n += len(ids)
        ev1.record()
        torch.cuda.current_stream().synchronize()
        e_ms = ev0.elapsed_time(ev1)
        return {"value": n / (e_ms / 1e3), "unit": "tasks/s", "ms_per_step": e_ms,
                "h2d_bytes_per_step": int(h2d + 320 * n), "d2h_bytes_per_step": int(d2h)}

    def oracle(arm):
        from oracle import execute
        t0 = time.perf_counter()
        n = k = 0
        while k < len(arm.streams) and time.perf_counter() - t0 < 10.0:
            st = arm.streams[k]
            execute.run_inorder(st.buffers, st.tasks)
            n += len(st.tasks)
            k += 1
        dt = time.perf_counter() - t0
        return {"value": n / dt, "unit": "tasks/s", "cores": 1, "kind": "oracle",
                "sample": f"first {k} inputs of the step ({n} tasks), single-threaded numpy, {dt:.1f} s"}

    return per_input_bench(args, torch, dist, world, rank, peaks, peak_src, flush_buf, make,
                           WORKLOAD_DNN.format(per_b=getattr(args, "dnn_per_b", 100)), "", baselines, e2e, oracle)


class StaticInputs:
    """The static randomly wired network: one task graph, 100 inputs per
    step. The window scheduler and the in-order / software baselines run
    every input as its own flush; the CUDA graph is built for the first input
    and replayed for every later one (inputs change only the data). resident:
    the scheduler kernel stays on the device, each input is copied in from
    pinned host memory and then published."""

    def __init__(self, torch, mode, window, cta_slots, seed=1, n_inputs=100, resident=False):
        import streamgen as sg
        from paper_2401_12377_b300 import harness
        self.torch, self.mode, self.resident = torch, mode, resident
        self.stream = sg.random_wire_stream(seed, window=window)
        self.bufs = harness.DeviceBuffers(self.stream.buffers)
        rng = np.random.default_rng(seed + 17)
        host_in = rng.uniform(-1, 1, (n_inputs, 256)).astype(np.float32)
        self.inputs = torch.from_numpy(host_in).pin_memory() if resident else torch.from_numpy(host_in).cuda()
        self.ids, self.rows = harness.pack_tasks(self.stream.tasks, self.bufs)
        torch.cuda.current_stream().synchronize()
        self.ctx = harness.Context(window, mode=mode, timing=True, capacity=1 << 12, cta_slots=cta_slots,
                                   resident=resident)
        self.x0 = self.bufs.t["x"][:1024].view(torch.float32)
        self.built = False

    def reset_device(self):
        pass

    def run_once(self, latencies=None):
        n = 0
        for i in range(self.inputs.shape[0]):
            t0 = time.perf_counter()
            self.x0.copy_(self.inputs[i], non_blocking=True)
            if self.resident:
                self.torch.cuda.current_stream().synchronize()   # the input is on the device
            if self.mode == "graph" and self.built:
                self.ctx.replay()
            else:
                self.ctx.submit_packed(self.ids + np.uint32(self.ctx.tail(0)), self.rows)
                self.ctx.flush()
                self.built = True
            self.ctx.sync()
            if latencies is not None:
                latencies.append(time.perf_counter() - t0)
            n += len(self.ids)
        return n


def bench_static(args, torch, dist, world, rank, peaks, peak_src, flush_buf):
    def make(mode, W, seed, resident):
        return StaticInputs(torch, mode, W, args.cta_slots, seed, resident=resident)

    def baselines(line, ms_step, k, W, seed):
        for mode in ("inorder", "graph", "sw"):
            b = make(mode, W, seed, False)
            r = time_arm(b, k, 1, flush_buf)
            ms = statistics.mean(r["ms"])
            entry = {"tasks_per_s": (r["tasks"] / k) / (ms / 1e3), "ms_per_step": ms,
                     "kernel_ms_per_step": r["stats"]["kernel_ms"] / k}
            if mode == "graph":
                entry["note"] = "graph built once (first warm-up input), replayed for every input"
                line["graph_replay"] = entry
                line["speedup_vs_graph_replay"] = ms / ms_step
            elif mode == "sw":
                line["sw_host_scheduler"] = entry
                line["speedup_vs_sw_host_scheduler"] = ms / ms_step
            else:
                line["inorder"] = entry
                line["speedup_vs_inorder"] = ms / ms_step
            b.ctx.close()

    def e2e(arm):
        # each input in from pinned memory, the stage output back
        pin_in = arm.inputs if arm.resident else arm.inputs.cpu().pin_memory()
        pin_out = torch.empty(256, dtype=torch.float32).pin_memory()
        xout = arm.bufs.t["x"].view(torch.float32)[-256:]
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.current_stream().synchronize()
        ev0.record()
        n = 0
        for i in range(pin_in.shape[0]):
            arm.x0.copy_(pin_in[i], non_blocking=True)
            if arm.resident:
                torch.cuda.current_stream().synchronize()
            arm.ctx.submit_packed(arm.ids + np.uint32(arm.ctx.tail(0)), arm.rows)
            arm.ctx.flush()
            arm.ctx.sync()
            pin_out.copy_(xout, non_blocking=True)
            n += len(arm.ids)
        ev1.record()
        torch.cuda.current_stream().synchronize()
        e_ms = ev0.elapsed_time(ev1)
        return {"value": n / (e_ms / 1e3), "unit": "tasks/s", "ms_per_step": e_ms,
                "h2d_bytes_per_step": int(arm.inputs.numel() * 4 + 320 * n),
                "d2h_bytes_per_step": int(1024 * arm.inputs.shape[0])}

    def oracle(arm):
        from oracle import execute
        t0 = time.perf_counter()
        n = k = 0
        while time.perf_counter() - t0 < 10.0 and k < 200:
            execute.run_inorder(arm.stream.buffers, arm.stream.tasks)
            n += len(arm.stream.tasks)
            k += 1
        dt = time.perf_counter() - t0
        return {"value": n / dt, "unit": "tasks/s", "cores": 1, "kind": "oracle",
                "sample": f"{k} inputs ({n} tasks), single-threaded numpy, {dt:.1f} s"}

    return per_input_bench(args, torch, dist, world, rank, peaks, peak_src, flush_buf, make, WORKLOAD_STATIC,
                           "; 24 MB of weights per input", baselines, e2e, oracle)


class _ArenaAddr:
    """pack_task's view of named buffers placed at fixed device addresses."""

    def __init__(self, base):
        self.base = base

    def ptr(self, ref) -> int:
        return self.base[ref.buf] + ref.off * 4


class TinyStreams:
    """The tiny elementwise workload: streams of 64 axpy / scale / add tasks
    over 16 buffers of 4096 floats (window 8), seeds 0 .. n - 1, each its own
    flush and persistent launch, run back to back. All streams' buffers sit in
    one device arena (n x 256 KiB: 250 MiB for 1000 streams, larger than L2)."""

    N_BUF, N_ELEM = 16, 4096

    def __init__(self, torch, mode, n=1000, window=8, cta_slots=0):
        import streamgen as sg
        from paper_2401_12377_b300 import harness
        self.torch = torch
        self.streams = [sg.elementwise_stream(seed) for seed in range(n)]
        per = self.N_BUF * self.N_ELEM
        host = np.concatenate([st.buffers[f"b{i}"] for st in self.streams for i in range(self.N_BUF)])
        self.host_pinned = torch.from_numpy(host).pin_memory()
        self.arena = self.host_pinned.cuda()
        self.pristine = self.arena.clone()
        base = self.arena.data_ptr()
        self.packed = []
        for s, st in enumerate(self.streams):
            at = _ArenaAddr({f"b{i}": base + (s * per + i * self.N_ELEM) * 4 for i in range(self.N_BUF)})
            self.packed.append(harness.pack_tasks(st.tasks, at))
        torch.cuda.current_stream().synchronize()
        self.ctx = harness.Context(window, mode=mode, timing=True, capacity=1 << 12, cta_slots=cta_slots)
        self.n_tasks = sum(len(st.tasks) for st in self.streams)

    def reset_device(self):
        self.arena.copy_(self.pristine, non_blocking=True)

    def run_once(self, latencies=None, e2e_out=None):
        n = 0
        per = self.N_BUF * self.N_ELEM
        for s, (ids, rows) in enumerate(self.packed):
            t0 = time.perf_counter()
            if e2e_out is not None:      # this stream's buffers in from pinned host memory
                self.arena[s * per:(s + 1) * per].copy_(self.host_pinned[s * per:(s + 1) * per], non_blocking=True)
            self.ctx.submit_packed(ids + np.uint32(self.ctx.tail(0)), rows)
            self.ctx.flush()
            self.ctx.sync()
            if e2e_out is not None:      # and its buffers back
                e2e_out[s * per:(s + 1) * per].copy_(self.arena[s * per:(s + 1) * per], non_blocking=True)
            if latencies is not None:
                latencies.append(time.perf_counter() - t0)
            n += len(ids)
        return n


def bench_tiny(args, torch, dist, world, rank, peaks, peak_src, flush_buf, n_streams=1000):
    """The tiny elementwise workload (1000 streams, each its own launch) with
    its in-order and CUDA-graph baselines, end-to-end arm and CPU oracle."""
    W = 8
    arm = TinyStreams(torch, "window", n_streams, W, args.cta_slots)
    lat = []
    res = time_arm(arm, args.steps, args.warmup, flush_buf, lat)
    ms_step = statistics.mean(res["ms"])
    max_ms = max_over_ranks(ms_step, dist, "cuda")
    tps = res["tasks"] / args.steps
    st = res["stats"]
    launches = st["launches"]
    avg_launch_s = (st["kernel_ms"] / 1e3) / max(1, launches)
    bpl = st["device_seg_bytes"] / max(1, launches)
    achieved = bpl / avg_launch_s / 1e9 if avg_launch_s > 0 else 0.0
    peak = float(peaks.get("hbm_gbs", 6400.0))
    lus = np.sort(np.array(lat)) * 1e6
    line = {"value": whole_job_rate(world, tps, max_ms / 1e3), "unit": "tasks/s", "ms_per_step": max_ms,
            "steps": args.steps, "warmup": args.warmup,
            "config": {"workload": f"tiny elementwise streams: {n_streams} streams (seeds 0..{n_streams - 1}) of 64 "
                                   "FP32 axpy/scale/add tasks over 16 buffers x 4096 floats, 1-4 CTAs per task, "
                                   "window 8, one flush and one launch per stream, back to back",
                       "window": W, "lookahead": effective_lookahead(W, 0, args.lookahead),
                       "streams_per_step": n_streams, "tasks_per_step": tps,
                       "cta_slots": st.get("cta_slots"),
                       "l2": "inputs (250 MiB arena) larger than L2, and flushed between timed steps"},
            "stream_latency_us": {"p50": float(lus[len(lus) // 2]), "p99": float(lus[int(0.99 * (len(lus) - 1))])},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "kernel": "acs_persistent_kernel", "peak_source": peak_src,
                         "algorithmic_bytes_per_launch": bpl, "avg_launch_us": avg_launch_s * 1e6},
            "gpu_launches_per_step": launches / args.steps}
    # end to end: each stream's buffers in from pinned memory and back out
    out = torch.empty_like(arm.host_pinned).pin_memory()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.current_stream().synchronize()
    ev0.record()
    n = arm.run_once(e2e_out=out)
    ev1.record()
    torch.cuda.current_stream().synchronize()
    e_ms = ev0.elapsed_time(ev1)
    line["e2e"] = {"value": n / (e_ms / 1e3), "unit": "tasks/s", "ms_per_step": e_ms,
                   "h2d_bytes_per_step": int(arm.host_pinned.numel() * 4 + 320 * n),
                   "d2h_bytes_per_step": int(out.numel() * 4)}
    arm.ctx.close()
    k = max(1, min(args.steps, 3))
    if not args.no_baselines:
        for mode in ("inorder", "graph"):
            b = TinyStreams(torch, mode, n_streams, W, args.cta_slots)
            r = time_arm(b, k, 1, flush_buf)
            ms = statistics.mean(r["ms"])
            kms = r["stats"]["kernel_ms"] / k
            if mode == "graph":
                line["graph_with_build"] = {"tasks_per_s": (r["tasks"] / k) / (ms / 1e3), "ms_per_step": ms,
                                            "host_build_instantiate_ms_per_step":
                                                (r["stats"]["graph_build_ms"] + r["stats"]["graph_instantiate_ms"]) / k}
                line["graph_launch"] = {"tasks_per_s": (r["tasks"] / k) / (kms / 1e3), "device_ms_per_step": kms}
                line["speedup_vs_graph_with_build"] = ms / ms_step
                line["speedup_vs_graph_launch_only"] = kms / ms_step
            else:
                line["inorder"] = {"tasks_per_s": (r["tasks"] / k) / (ms / 1e3), "ms_per_step": ms}
                line["speedup_vs_inorder"] = ms / ms_step
            b.ctx.close()
            del b
    if rank == 0 and world == 1 and not args.no_cpu:
        from oracle import execute
        t0 = time.perf_counter()
        n = i = 0
        while i < len(arm.streams) and time.perf_counter() - t0 < 5.0:
            stm = arm.streams[i]
            execute.run_inorder(stm.buffers, stm.tasks)
            n += len(stm.tasks)
            i += 1
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": n / dt, "unit": "tasks/s", "cores": 1, "kind": "oracle",
                                "sample": f"the first {i} streams ({n} tasks), single-threaded numpy, {dt:.1f} s"}
    else:
        line["cpu_baseline"] = None
    return line


def bench_batched(args, torch, dist, world, rank, peaks, peak_src, flush_buf):
    """64 independent streams of uneven length in one persistent launch, window
    and CTA slots from the autotuner; lockstep host-driven baselines."""
    import streamgen as sg
    from paper_2401_12377_b300 import autotune, harness, shard
    # one batch for the whole job; with several ranks each runs its share of
    # the streams (longest first to the least-loaded rank), no data collective
    seed = 1
    all_specs = sg.batched_specs(seed)
    part = shard.partition_by_size([sp.target for sp in all_specs], world, rank)
    specs = [all_specs[i] for i in part]
    S = len(specs)
    cap = 1 << 13
    wl = harness.BatchedWorkload(specs, None)
    tuned = None
    if args.window or args.cta_slots or args.no_tune:
        W, slots = args.window or 32, args.cta_slots
    else:
        def make_run(ctx):
            wl.bind(ctx)

            def run():
                wl.reset()
                return wl.run()
            return run
        t0 = time.perf_counter()
        tuned = autotune.tune(f"{WORKLOAD_BATCHED}|seed={seed}|part={rank}/{world}", make_run, n_streams=S,
                              repeats=5, capacity=cap)
        tuned["tune_s"] = time.perf_counter() - t0
        W, slots = tuned["window"], tuned["cta_slots"]
    # the kernel alone: one flush and one launch per pass (roofline from its launches)
    ctx1 = harness.Context(W, n_streams=S, cta_slots=slots, timing=True, capacity=cap)
    wl.bind(ctx1)
    res1 = time_arm(BatchArm(torch, wl, ctx1), max(1, min(args.steps, 3)), 1, flush_buf)
    ctx1.close()
    # the DAG's critical path: one traced single-flush pass, outside the timed
    # regions; the pass is bounded by its longest stream chain
    ctx_t = harness.Context(W, n_streams=S, cta_slots=slots, capacity=cap, log=True, trace=True)
    wl.bind(ctx_t)
    wl.reset()
    wl.run()
    cps = [critical_path(ctx_t, i, 0, ctx_t.tail(i)) for i in range(S)]
    ctx_t.close()
    cp_i = max(range(S), key=lambda i: cps[i][0])
    # the method: a resident kernel, each stream published as soon as it is
    # submitted (longest first); a pass ends when every stream is idle. CUDA
    # events on this stream bracket each pass (the pass is host-synchronous).
    # (pinned copies for the resets first: the resident kernel holds every SM,
    # so resets go host to device, and there is no L2-flush kernel: the
    # inputs, 384 MB of gated-MLP weights, are larger than L2)
    wl.host_written()
    wl.host_inputs()
    wl.result_buffers()
    ctx = harness.Context(W, n_streams=S, cta_slots=slots, timing=True, capacity=cap, resident=True)
    wl.bind(ctx)
    arm = BatchArm(torch, wl, ctx)
    latencies = []
    if dist:
        dist.barrier()
    with ClockSampler(torch.cuda.current_device()) as clk:
        res = time_arm(arm, args.steps, args.warmup, None, latencies)
    clocks = clk.summary()
    ms_step = statistics.mean(res["ms"])
    tasks_per_step = res["tasks"] / args.steps
    max_ms = max_over_ranks(ms_step, dist, "cuda")
    job_tasks_per_step = shard.gather_sum(dist, tasks_per_step)
    st = res1["stats"]
    launches = st["launches"]
    avg_launch_s = (st["kernel_ms"] / 1e3) / max(1, launches)
    bytes_per_launch = st["device_seg_bytes"] / max(1, launches)
    achieved = bytes_per_launch / avg_launch_s / 1e9 if avg_launch_s > 0 else 0.0
    peak = float(peaks.get("hbm_gbs", 6400.0))
    line = {"metric": METRIC, "value": job_tasks_per_step / (max_ms / 1e3), "unit": "tasks/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": max_ms,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "critical_path": {"us": cps[cp_i][0], "tasks_on_chain": cps[cp_i][1], "stream": cp_i,
                              "kernel_us_per_pass": avg_launch_s * 1e6,
                              "note": "the longest of the 64 streams' chains (logged window DAG, tasks "
                                      "weighted by their body times in a traced pass): the makespan with "
                                      "no scheduling overhead"},
            "config": {"workload": WORKLOAD_BATCHED, "streams": S, "window": W,
                       "lookahead": effective_lookahead(W, 0, args.lookahead, S), "tasks_per_step": tasks_per_step,
                       "cta_slots": st.get("cta_slots"), "grid": st.get("grid"),
                       "stream_lengths": [sp.target for sp in specs],
                       "mode": "window scheduler, one resident persistent launch for all streams; each "
                               "stream published as soon as it is submitted",
                       "l2": "not flushed between passes: inputs larger than L2 (384 MB of gated-MLP weights)",
                       "parallelism": (f"one batch split over {world} GPUs by size ({S} of {len(all_specs)} "
                                       f"streams on rank 0)") if world > 1 else "one GPU"},
            "autotune": None if tuned is None else {
                "window": W, "cta_slots": slots, "tune_s": tuned.get("tune_s"), "cached": tuned.get("cached", False),
                "table": [(r["window"], r["cta_slots"], round(r["ms"], 4)) for r in tuned.get("table", [])]},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "acs_persistent_kernel",
                         "peak_source": peak_src, "algorithmic_bytes_per_launch": bytes_per_launch,
                         "launches_from": "single-flush arm (one launch per pass, CUDA events around it)",
                         "avg_launch_us": avg_launch_s * 1e6,
                         "note": "bytes named by the tasks' read+write segments per launch / mean launch time"},
            "sched_cycles_per_task": st["sched_cycles"] / max(1, st["sched_inserts"]),
            "gpu_launches": 1, "gpu_launches_note": "one resident persistent launch runs through the timed region",
            "pass_ms": [round(x, 3) for x in res["ms"]],
            "single_flush": {"ms_per_step": statistics.mean(res1["ms"]), "pass_ms": [round(x, 3) for x in res1["ms"]],
                             "tasks_per_s": (res1["tasks"] / max(1, min(args.steps, 3))) / (statistics.mean(res1["ms"]) / 1e3),
                             "kernel_ms_per_step": avg_launch_s * 1e3,
                             "note": "all streams submitted, then one flush and one launch per pass"},
            "clocks": clocks}

    # end to end: every stream's buffers in from pinned host memory, results out
    reps = max(1, min(args.steps, 3))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # (the pinned buffers exist already: pinning while the kernel runs is slow)
    torch.cuda.current_stream().synchronize()
    tasks = h2d = d2h = 0
    ev0.record()
    for _ in range(reps):
        h2d += wl.upload_host()
        tasks += wl.run()
        d2h += wl.download_results()
    ev1.record()
    torch.cuda.current_stream().synchronize()
    e_ms = ev0.elapsed_time(ev1) / reps
    desc = 320 * (tasks // reps)
    line["e2e"] = {"value": (tasks / reps) / (e_ms / 1e3), "unit": "tasks/s", "ms_per_step": e_ms,
                   "h2d_bytes_per_step": int(h2d // reps + desc), "d2h_bytes_per_step": int(d2h // reps)}
    ctx.close()
    if not args.no_baselines:
        steps_b = max(1, min(args.steps, 3))
        for mode, key in (("window", "window_host_driven"), ("inorder", "inorder"), ("graph", "graph"),
                          ("sw", "sw_host_scheduler")):
            c2 = harness.Context(W, mode=mode, n_streams=S, cta_slots=slots, timing=True, capacity=cap)
            hd = harness.BatchedHostDriven(specs, c2)
            r = time_arm(BatchArm(torch, hd, c2), steps_b, 1, flush_buf)
            ms = statistics.mean(r["ms"])
            tps = r["tasks"] / steps_b
            entry = {"tasks_per_s": tps / (ms / 1e3), "ms_per_step": ms, "flushes_per_step": hd.rounds,
                     "kernel_ms_per_step": r["stats"]["kernel_ms"] / steps_b,
                     "launches_per_step": r["stats"]["launches"] / steps_b}
            if mode == "graph":
                entry["host_build_instantiate_ms_per_step"] = (r["stats"]["graph_build_ms"]
                                                               + r["stats"]["graph_instantiate_ms"]) / steps_b
                line["graph_launch"] = {"tasks_per_s": tps / (entry["kernel_ms_per_step"] / 1e3),
                                        "device_ms_per_step": entry["kernel_ms_per_step"],
                                        "note": "graph launch device time only, build and round trips excluded"}
                line["speedup_vs_graph_with_build"] = ms / ms_step
                line["speedup_vs_graph_launch_only"] = entry["kernel_ms_per_step"] / ms_step
                key = "graph_with_build"
            elif mode == "inorder":
                line["speedup_vs_inorder"] = ms / ms_step
            elif mode == "sw":
                line["speedup_vs_sw_host_scheduler"] = ms / ms_step
            line[key] = entry
            c2.close()
            del hd

    if rank == 0 and world == 1 and not args.no_cpu:
        execute_tasks, n_streams, dt = oracle_batch(seed, limit_s=10.0)
        line["cpu_baseline"] = {"value": execute_tasks / dt, "unit": "tasks/s", "cores": 1, "kind": "oracle",
                                "sample": f"first {n_streams} streams of the batch ({execute_tasks} tasks), "
                                          f"single-threaded numpy + C bodies, {dt:.1f} s"}
    elif rank == 0:
        line["cpu_baseline"] = None
    return line


def bench_serving(args, torch, dist, world, rank, peaks, peak_src):
    """Open-loop serving: requests arrive as a Poisson process (args.rate per
    second, args.steps seconds of arrivals after args.warmup x 100 warm-up
    requests) and are served by one resident kernel with args.slots stream
    slots and a 20 GB budget. Host clock throughout: latency is completion seen
    by the host minus arrival; every request's inputs go host to device and its
    results device to host inside the run."""
    import streamgen as sg
    from paper_2401_12377_b300 import harness, serving, shard
    # one arrival process for the whole job; with several ranks, request i is
    # served by rank i mod world (each rank sees a Poisson process of rate / world)
    seed = 1
    t_prep = time.perf_counter()
    specs = sg.serving_catalogue(seed)
    cat = serving.Catalogue(specs)
    t_prep = time.perf_counter() - t_prep
    W = args.window or 32
    n_req = int(round(args.rate * args.steps))
    arrivals, kinds = sg.poisson_arrivals(seed, n_req, args.rate, len(specs))
    mine = shard.partition_round_robin(n_req, world, rank)
    arrivals, kinds = arrivals[mine], kinds[mine]
    wa, wk = sg.poisson_arrivals(seed + 1000, max(1, 100 * args.warmup), args.rate / world, len(specs))
    ctx = harness.Context(W, n_streams=args.slots, resident=True, timing=True, capacity=1 << 13)
    srv = serving.Server(cat, ctx, budget_bytes=20 << 30, readback=True)
    srv.run(wa, wk)
    if dist:
        dist.barrier()
    with ClockSampler(torch.cuda.current_device()) as clk:
        r = srv.run(arrivals, kinds)
    clocks = clk.summary()
    ctx.stop()
    st = ctx.stats()
    ctx.close()
    # every rank's per-request logs gathered on rank 0 (the only collective)
    lat = np.sort(shard.gather_values(dist, r["latency_s"], rank, world)) * 1e3
    q = np.sort(shard.gather_values(dist, r["queue_s"], rank, world)) * 1e3
    tasks = int(shard.gather_sum(dist, float(r["tasks"].sum())))
    span = max_over_ranks(r["span_s"], dist, "cuda")
    value = tasks / span
    pct = lambda a, p: float(a[min(len(a) - 1, int(p * len(a)))])
    mean_len = float(np.mean([specs[int(k)].target for k in kinds]))
    kernel_s = st["kernel_ms"] / 1e3
    # where the tail comes from: queueing (admission waits) or service, per
    # request kind and length
    lat_ms, q_ms = r["latency_s"] * 1e3, r["queue_s"] * 1e3
    svc_ms = lat_ms - q_ms
    kind_of = np.array([specs[int(k)].kind for k in kinds])
    length = np.array([specs[int(k)].target for k in kinds])

    def dist_of(a):
        a = np.sort(a)
        return {"n": int(len(a)), "p50": pct(a, 0.5), "p99": pct(a, 0.99)} if len(a) else None

    slow = lat_ms >= np.quantile(lat_ms, 0.99) if len(lat_ms) else np.zeros(0, bool)
    breakdown = {
        "service_ms": dist_of(svc_ms),
        "by_kind": {k: {"latency_ms": dist_of(lat_ms[kind_of == k]), "service_ms": dist_of(svc_ms[kind_of == k]),
                        "queue_ms": dist_of(q_ms[kind_of == k])} for k in ("rl", "dnn")},
        "by_length": {f"{lo}-{hi}": {"latency_ms": dist_of(lat_ms[(length >= lo) & (length < hi)]),
                                     "service_ms": dist_of(svc_ms[(length >= lo) & (length < hi)])}
                      for lo, hi in ((100, 300), (300, 1000), (1000, 2500), (2500, 5001))},
        "slowest_1pct": {"n": int(slow.sum()), "rl_share": float(np.mean(kind_of[slow] == "rl")) if slow.any() else None,
                         "mean_tasks": float(length[slow].mean()) if slow.any() else None,
                         "mean_queue_ms": float(q_ms[slow].mean()) if slow.any() else None,
                         "mean_service_ms": float(svc_ms[slow].mean()) if slow.any() else None}}
    line = {"metric": METRIC, "value": value, "unit": "tasks/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * span / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD_SERVING, "requests": n_req, "rate_per_s": args.rate,
                       "step": "one second of arrivals", "slots": args.slots, "window": W,
                       "lookahead": effective_lookahead(W, 0, args.lookahead, args.slots), "budget_gb": 20,
                       "catalogue_types": len(specs), "mean_request_tasks": mean_len,
                       "timing": "host clock (perf_counter) from first arrival to last completion",
                       "l2": "not flushed: a continuous open-loop run over > 126 MB of request data",
                       "parallelism": (f"one arrival process split over {world} GPUs round-robin, latency logs "
                                       f"gathered on rank 0") if world > 1 else "one GPU"},
            "latency_ms": {"p50": pct(lat, 0.5), "p99": pct(lat, 0.99), "mean": float(lat.mean()),
                           "max": float(lat[-1])},
            "queue_wait_ms": {"p50": pct(q, 0.5), "p99": pct(q, 0.99)},
            "latency_breakdown": breakdown,
            "offered_tasks_per_s": args.rate * mean_len,
            "mean_in_flight": r["mean_in_flight"], "peak_device_bytes": r["peak_bytes"],
            "requests_per_s": n_req / span,
            "resident_kernel_s": kernel_s, "catalogue_prep_s": t_prep,
            "roofline": {"bound": "hbm", "achieved": st["device_seg_bytes"] / kernel_s / 1e9 if kernel_s else 0.0,
                         "peak": float(peaks.get("hbm_gbs", 6400.0)), "unit": "GB/s",
                         "frac": (st["device_seg_bytes"] / kernel_s / 1e9 if kernel_s else 0.0)
                         / float(peaks.get("hbm_gbs", 6400.0)),
                         "traffic": None, "kernel": "acs_persistent_kernel", "peak_source": peak_src,
                         "note": "segment bytes of all tasks over the resident launch's whole life "
                                 "(warm-up, timed run and idle gaps included): a utilisation figure"},
            "gpu_launches": int(st["launches"]),
            "e2e": {"value": value, "unit": "tasks/s", "h2d_bytes_per_step": int(r["h2d_bytes"] / args.steps),
                    "d2h_bytes_per_step": int(r["d2h_bytes"] / args.steps),
                    "note": "the serving loop is end to end: inputs uploaded and results read back per request"},
            "clocks": clocks}
    if rank == 0 and world == 1 and not args.no_cpu:
        t, nr, dt = oracle_serving(seed, n_req, args.rate, limit_s=10.0)
        line["cpu_baseline"] = {"value": t / dt, "unit": "tasks/s", "cores": 1, "kind": "oracle",
                                "sample": f"first {nr} requests in arrival order ({t} tasks), "
                                          f"single-threaded numpy + C bodies, {dt:.1f} s"}
    elif rank == 0:
        line["cpu_baseline"] = None
    return line


SUB_KEYS = ("value", "unit", "ms_per_step", "steps", "warmup", "config", "stream_latency_us", "input_latency_us",
            "latency_ms", "queue_wait_ms", "latency_breakdown", "offered_tasks_per_s", "requests_per_s",
            "mean_in_flight", "roofline", "critical_path", "cpu_baseline", "e2e", "speedup_vs_inorder",
            "speedup_vs_graph_with_build", "speedup_vs_graph_launch_only", "speedup_vs_sw_host_scheduler",
            "inorder", "graph_with_build", "graph_launch", "sw_host_scheduler", "single_flush", "pass_ms", "autotune",
            "resident_per_input", "gpu_launches", "gpu_launches_per_step", "clocks")


def other_configs(args, torch, dist, world, rank, peaks, peak_src, flush_buf):
    """Compact runs of the tiny, dynamic-DNN, batched and serving workloads,
    each timed on its own (3 warm-up + 3 timed steps; dnn 25 inputs per batch
    size; serving --serving-seconds of arrivals), with its own baselines,
    roofline, end-to-end arm and CPU oracle sample."""
    import argparse as _ap
    out = {}
    base = dict(vars(args), window=0, cta_slots=0, no_tune=False, steps=3, warmup=3)
    t0 = time.perf_counter()
    out["tiny"] = bench_tiny(_ap.Namespace(**base), torch, dist, world, rank, peaks, peak_src, flush_buf)
    out["tiny"]["bench_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    d = bench_dnn(_ap.Namespace(**dict(base, dnn_per_b=25)), torch, dist, world, rank, peaks, peak_src, flush_buf)
    out["dnn"] = {k: d[k] for k in SUB_KEYS if k in d}
    out["dnn"]["bench_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    b = bench_batched(_ap.Namespace(**base), torch, dist, world, rank, peaks, peak_src, flush_buf)
    out["batched"] = {k: b[k] for k in SUB_KEYS if k in b}
    out["batched"]["bench_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    sv = bench_serving(_ap.Namespace(**dict(base, steps=args.serving_seconds, warmup=1)), torch, dist, world,
                       rank, peaks, peak_src)
    out["serving"] = {k: sv[k] for k in SUB_KEYS if k in sv}
    out["serving"]["bench_s"] = time.perf_counter() - t0
    return out


def main():
    args = parse()
    if args.lookahead is not None:
        from paper_2401_12377_b300 import harness
        harness.DEFAULT_LOOKAHEAD = args.lookahead
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    world, rank, local = ranks()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2401_12377_b300 import build
    build.build()
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else open(os.devnull) as f:
        try:
            peaks = json.load(f)
            peak_src = "measured"
        except json.JSONDecodeError:
            peaks, peak_src = {"hbm_gbs": 6400.0}, "fallback"

    # one non-default stream for all of this process's device work: torch
    # copies (state resets, L2 flush, read-backs) and the library's launches
    torch.cuda.set_stream(torch.cuda.Stream())
    flush_buf = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    seed = 1 + rank
    if args.workload in ("dnn", "static", "batched", "serving"):
        if args.workload == "batched":
            line = bench_batched(args, torch, dist, world, rank, peaks, peak_src, flush_buf)
        elif args.workload == "dnn":
            line = bench_dnn(args, torch, dist, world, rank, peaks, peak_src, flush_buf)
        elif args.workload == "static":
            line = bench_static(args, torch, dist, world, rank, peaks, peak_src, flush_buf)
        else:
            line = bench_serving(args, torch, dist, world, rank, peaks, peak_src)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    args.window = args.window or 32

    # ---- the method: window scheduler with device-side emission (one launch per run) ----
    acs_arm = RLBench("window", seed, args.window, args.cta_slots, emit=True)
    latencies = []
    if dist:
        dist.barrier()
    with ClockSampler(torch.cuda.current_device()) as clk:
        res = time_arm(acs_arm, args.steps, args.warmup, flush_buf, latencies)
    clocks = clk.summary()
    ms_step = statistics.mean(res["ms"])
    tasks_per_step = res["tasks"] / args.steps
    max_ms = max_over_ranks(ms_step, dist, "cuda")
    value = whole_job_rate(world, tasks_per_step, max_ms / 1e3)
    st = res["stats"]
    launches = st["launches"]
    kernel_ms = st["kernel_ms"]
    avg_launch_s = (kernel_ms / 1e3) / max(1, launches)
    bytes_per_launch = st["device_seg_bytes"] / max(1, launches)
    achieved = bytes_per_launch / avg_launch_s / 1e9 if avg_launch_s > 0 else 0.0
    peak = float(peaks.get("hbm_gbs", 6400.0))
    lat_us = sorted(1e6 * x for x in latencies)

    line = {"metric": METRIC, "value": value, "unit": "tasks/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": max_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "window": args.window, "tasks_per_step": tasks_per_step,
                       "lookahead": effective_lookahead(args.window, 0, args.lookahead),
                       "mode": "window scheduler, device-side emission: one flush and one launch per run",
                       "flushes_per_step": 1, "cta_slots": st.get("cta_slots"),
                       "grid": st.get("grid"), "l2": "flushed between timed steps (512 MiB write)",
                       "warm_up": f"at least {args.warmup} steps and {HOST_WARM_S} s of steps (every arm)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single stream"},
            "run_latency_us": {"p50": lat_us[len(lat_us) // 2] if lat_us else None,
                               "p99": lat_us[min(len(lat_us) - 1, int(0.99 * len(lat_us)))] if lat_us else None},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": TRAFFIC_RLSIM["bytes_per_launch"]
                         if kernel_sources_sha1() == TRAFFIC_RLSIM["sources_sha1"] else None,
                         "kernel": "acs_persistent_kernel", "peak_source": peak_src,
                         "algorithmic_bytes_per_launch": bytes_per_launch,
                         "avg_launch_us": avg_launch_s * 1e6,
                         "note": "bytes named by the tasks' read+write segments per launch / mean "
                                 "launch time (CUDA events around each cooperative launch)"},
            "sched_cycles_per_task": st["sched_cycles"] / max(1, st["sched_inserts"]),
            "gpu_launches": int(launches),
            "clocks": clocks}

    # ---- the DAG's critical path (a traced run outside the timed region) ----------------------
    # Nearly every conflict of this stream is W or more positions apart (a
    # step's broadphase and integrate tasks sit beyond the window from its
    # solves), so the chain is taken over the full DAG of the host-driven form
    # of the stream, whose every task the host knows
    ta = RLBench("window", seed, args.window, args.cta_slots, emit=False, traced=True)
    ta.reset_device()
    plans = ta.driver.run(record_plans=True)
    n_t = ta.ctx.tail(0)
    tr_t = ta.ctx.trace(0, 0, n_t).astype(np.int64)
    rows = np.concatenate([ta.driver.pack(p)[1] for p in plans])
    ta.ctx.close()
    cp_us, cp_n = critical_path_full(task_segments(rows), np.maximum(tr_t[:, 3] - tr_t[:, 2], 0) / 1e3)
    line["critical_path"] = {"us": cp_us, "tasks_on_chain": cp_n, "kernel_us_per_run": avg_launch_s * 1e6,
                             "note": "longest chain of the full dependency DAG of the stream's host-driven "
                                     "form (no emit tasks), tasks weighted by their body times in a traced "
                                     "run: the makespan with no scheduling overhead"}

    # ---- the window's bound: the same stream with device emission, traced -------------------
    # (the emit task of a step follows the step's tasks in the host-driven plans)
    kinds = []
    for i, pl in enumerate(plans):
        kinds += [0] * len(pl.kind) + ([1] if i < len(plans) - 1 else [])
    tw = RLBench("window", seed, args.window, args.cta_slots, emit=True, traced=True)
    for _ in range(2):
        tw.reset_device()
        n_w = tw.run_once()
    if n_w == len(kinds):
        emitter, last = [], -1
        for j, k in enumerate(kinds):
            emitter.append(last)
            if k:
                last = j
        wb = window_bound(tw.ctx, tw.ctx.tail(0) - n_w, n_w, args.window, emitter)
        line["window_bound"] = {
            "us": [wb["start"], wb["end"]], "kernel_us_per_run": avg_launch_s * 1e6,
            "frac": [wb["start"] / (avg_launch_s * 1e6), wb["end"] / (avg_launch_s * 1e6)],
            "note": "as-soon-as-possible schedule of the emitted stream with no scheduling overhead: a task "
                    "starts once its logged conflicting predecessors and every task window or more "
                    "positions back have ended, an emitted task once its emit task started (first value) "
                    "or ended (second); traced body times"}
    tw.ctx.close()

    # ---- baselines on the same box -----------------------------------------------------------
    if not args.no_baselines:
        host = RLBench("window", seed, args.window, args.cta_slots)
        step_lat = []
        r_h = time_arm(host, args.steps, max(1, args.warmup // 2), flush_buf, step_lat)
        ms_h = statistics.mean(r_h["ms"])
        tph = r_h["tasks"] / args.steps
        sl = sorted(1e6 * x for x in step_lat)
        line["window_host_driven"] = {
            "tasks_per_s": tph / (ms_h / 1e3), "ms_per_step": ms_h, "flushes_per_step": host.sim.p.steps + 1,
            "kernel_ms_per_step": r_h["stats"]["kernel_ms"] / args.steps,
            "sim_step_latency_us": {"p50": sl[len(sl) // 2], "p99": sl[min(len(sl) - 1, int(0.99 * len(sl)))]},
            "note": "same scheduler, host reads back island counts and submits each simulation step"}
        host.ctx.close()
        inorder = RLBench("inorder", seed, args.window, args.cta_slots)
        r_in = time_arm(inorder, args.steps, max(1, args.warmup // 2), flush_buf)
        ms_in = statistics.mean(r_in["ms"])
        graph = RLBench("graph", seed, args.window, args.cta_slots)
        r_g = time_arm(graph, args.steps, max(1, args.warmup // 2), flush_buf)
        ms_g = statistics.mean(r_g["ms"])
        g_launch_ms = r_g["stats"]["kernel_ms"] / args.steps
        g_build_ms = (r_g["stats"]["graph_build_ms"] + r_g["stats"]["graph_instantiate_ms"]) / args.steps
        tpi = r_in["tasks"] / args.steps
        line["inorder"] = {"tasks_per_s": tpi / (ms_in / 1e3), "ms_per_step": ms_in}
        line["graph_with_build"] = {"tasks_per_s": tpi / (ms_g / 1e3), "ms_per_step": ms_g,
                                    "host_build_instantiate_ms_per_step": g_build_ms}
        line["graph_launch"] = {"tasks_per_s": tpi / (g_launch_ms / 1e3),
                                "device_ms_per_step": g_launch_ms,
                                "note": "sum of graph launch device times only (build excluded, "
                                        "host round trips between graphs excluded)"}
        # per-run times compare the same simulation (the emitting stream has one
        # emit task per step on top of the ~15 000 tasks every arm runs)
        line["speedup_vs_inorder"] = ms_in / ms_step
        line["speedup_vs_graph_with_build"] = ms_g / ms_step
        line["speedup_vs_graph_launch_only"] = g_launch_ms / ms_step
        line["speedup_host_driven_window_vs_inorder"] = ms_in / ms_h
        line["acs_kernel_ms_per_step"] = kernel_ms / args.steps
        line["speedup_kernel_time_vs_graph_launch"] = g_launch_ms / (kernel_ms / args.steps)
        inorder.ctx.close()
        graph.ctx.close()
        swa = RLBench("sw", seed, args.window, args.cta_slots)
        r_sw = time_arm(swa, max(1, min(args.steps, 3)), 1, flush_buf)
        ms_sw = statistics.mean(r_sw["ms"])
        line["sw_host_scheduler"] = {"tasks_per_s": (r_sw["tasks"] / max(1, min(args.steps, 3))) / (ms_sw / 1e3),
                                     "ms_per_step": ms_sw, "threads": 8,
                                     "note": "the paper's software scheduler: host window, 8 threads x one "
                                             "CUDA stream, cudaStreamSynchronize per task"}
        line["speedup_vs_sw_host_scheduler"] = ms_sw / ms_step
        swa.ctx.close()

    # ---- window-size sensitivity: the ring dispatching ahead (the default), the plain ring
    # (lookahead 0) and free-slot (span 64) ------------------------------------------------------
    if args.window_study:
        study = []
        for span_mode in ("ring, dispatch ahead", "ring", "free-slot"):
            for W in (8, 16, 32, 64):
                if span_mode == "free-slot" and W == 64:
                    continue
                span = 64 if span_mode == "free-slot" else 0
                la = 0 if span_mode == "ring" else None
                arm = RLBench("window", seed, W, args.cta_slots, emit=True, span=span, lookahead=la)
                k_runs = max(1, min(args.steps, 3))
                with ClockSampler(torch.cuda.current_device()) as clk_row:   # clocks during each row too
                    r = time_arm(arm, k_runs, 1, flush_buf)
                ms = statistics.median(r["ms"])   # one host-side stall in a run cannot move it
                study.append({"window": W, "span": span or W, "lookahead": effective_lookahead(W, span, la),
                              "release": span_mode, "ms_per_run": ms,
                              "kernel_ms_per_run": r["stats"]["kernel_ms"] / max(1, r["stats"]["launches"]),
                              "clocks": clk_row.summary(),
                              "tasks_per_s": (r["tasks"] / max(1, min(args.steps, 3))) / (ms / 1e3)})
                arm.ctx.close()
        line["window_study"] = study

    # ---- end to end through the API with host buffers ---------------------------------------
    line["e2e"] = time_e2e(acs_arm, max(1, min(args.steps, 3)))
    acs_arm.ctx.close()

    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_oracle_rate()
    elif rank == 0:
        line["cpu_baseline"] = None

    # ---- the other workloads, compact, after the headline's timed region -------------------
    if not args.headline_only:
        line["configs"] = other_configs(args, torch, dist, world, rank, peaks, peak_src, flush_buf)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
