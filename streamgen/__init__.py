"""Seeded synthetic task streams: the inputs both sides of every check consume.

This module only *describes* work. It draws the random initial buffer contents,
chooses which task reads and writes which buffer range, and (for the rigid-body
stream) states which tasks a simulation step emits given the island counts that
the caller's own simulation produced. It holds no dependency detection, no
scheduling and no task-body arithmetic: the CPU oracle (``oracle/``) and the
CUDA path (``paper_2401_12377_b300``) each implement those on their own and both
read the streams built here.

A stream is a list of :class:`Task`. Array operands are :class:`Ref` triples
``(buffer name, element offset, element count)`` into named numpy buffers; the
consumer maps buffer names to its own storage (numpy arrays on the CPU, device
allocations on the GPU) and derives byte segments from the refs with its own
address-resolution code.

Workload shapes follow the paper's two workload classes (small kernels of a few
CTAs, Sec. II "Case Study 1/2"): the paper's own benchmarks (Brax physics
environments, InstaNAS / dynamic-routing DNNs on CIFAR10 / Cityscapes) are not
available, so these synthetic streams stand in for them by shape only.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, NamedTuple, Optional

import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """One output of the SplitMix64 generator (Steele, Lea, Flood; OOPSLA 2014)
    seeded with ``x``: a counter-based hash used for seeded per-task choices."""
    z = (x + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def mix(*keys: int) -> int:
    """Hash a tuple of small non-negative integers to 64 bits (chained SplitMix64)."""
    h = 0x2545F4914F6CDD1D
    for k in keys:
        h = splitmix64(h ^ (k & MASK64))
    return h


class Ref(NamedTuple):
    """A contiguous element range ``buf[off : off + n]`` of a named buffer."""
    buf: str
    off: int
    n: int


@dataclass
class Task:
    """One small kernel invocation in program order.

    ``op`` names the body; ``arrays`` maps operand roles to :class:`Ref`;
    ``scalars`` maps scalar roles to numpy scalars (float32 / uint32).
    ``ncta`` is the CTA count the task is launched with.
    """
    task_id: int
    op: str
    ncta: int
    arrays: Dict[str, Ref]
    scalars: Dict[str, object] = field(default_factory=dict)


@dataclass
class Stream:
    """A complete stream: initial buffers, tasks in program order, window size."""
    buffers: Dict[str, np.ndarray]
    tasks: List[Task]
    window: int
    name: str = ""


# ----------------------------------------------------------------------------
# Elementwise stream (16 buffers x 4096 floats, axpy / scale / add)
# ----------------------------------------------------------------------------

def elementwise_stream(seed: int, n_tasks: int = 64, n_buffers: int = 16,
                       n_elems: int = 4096, window: int = 8,
                       ranges: bool = False, max_ncta: int = 4) -> Stream:
    """Tiny synthetic stream of axpy / scale / add tasks.

    Each task picks its op uniformly, reads one (scale) or two (axpy, add)
    buffers and writes one buffer, all chosen uniformly (a written buffer may
    alias an input). ``a`` ~ U[0.5, 1.5), ``ncta`` ~ U{1..max_ncta}, buffer
    contents ~ U[-1, 1). With ``ranges`` every task instead works on one
    random sub-range ``[off, off + n)`` (same ``n`` for all its operands, any
    element alignment), which produces partial segment overlaps.
    """
    rng = np.random.default_rng(seed)
    bufs = {f"b{i}": rng.uniform(-1.0, 1.0, n_elems).astype(np.float32)
            for i in range(n_buffers)}
    tasks = []
    for t in range(n_tasks):
        op = ("axpy", "scale", "add")[int(rng.integers(0, 3))]
        ncta = int(rng.integers(1, max_ncta + 1))
        names = [f"b{int(i)}" for i in rng.integers(0, n_buffers, 3)]
        if ranges:
            # operands naming the same buffer share one offset: a task's own
            # reads and writes alias exactly or not at all (elementwise-safe)
            n = int(rng.integers(1, n_elems + 1))
            by_buf = {}
            offs = [by_buf.setdefault(nm, int(rng.integers(0, n_elems - n + 1))) for nm in names]
        else:
            n, offs = n_elems, [0, 0, 0]
        refs = [Ref(names[i], offs[i], n) for i in range(3)]
        a = np.float32(rng.uniform(0.5, 1.5))
        if op == "axpy":
            tasks.append(Task(t, op, ncta, {"x": refs[0], "y": refs[1]}, {"a": a}))
        elif op == "scale":
            tasks.append(Task(t, op, ncta, {"x": refs[0], "y": refs[1]}, {"a": a}))
        else:
            tasks.append(Task(t, op, ncta, {"x": refs[0], "y": refs[1], "z": refs[2]}))
    return Stream(bufs, tasks, window, f"elementwise(seed={seed},ranges={ranges})")


# ----------------------------------------------------------------------------
# Dynamic-DNN stream (gated residual MLP, hidden 256, 24 blocks)
# ----------------------------------------------------------------------------

GEMV_NCTA_CHOICES = (1, 2, 4, 8, 16, 32)


def dnn_gate(seed: int, sample: int, block: int) -> int:
    """Per-sample block gate (keep probability 1/2): 1 runs the block."""
    return int((mix(seed, 0xD5, sample, block) >> 17) & 1)


def dnn_weights(seed: int, sets: int = 24, hidden: int = 256):
    """(W, B): ``sets`` weight sets of the gated MLP, U[-1/16, 1/16), shaped as
    dnn_stream lays them out (flat float32)."""
    rng = np.random.default_rng(seed)
    W = rng.uniform(-1.0 / 16, 1.0 / 16, (sets, 2, hidden, hidden)).astype(np.float32)
    B = rng.uniform(-1.0 / 16, 1.0 / 16, (sets, 2, hidden)).astype(np.float32)
    return W.reshape(-1), B.reshape(-1)


def dnn_stream(seed: int, batch: int = 1, blocks: int = 24, hidden: int = 256,
               window: int = 32, task_id0: int = 0, weight_sets: int = 0, shared=None) -> Stream:
    """Gated residual MLP inference for ``batch`` samples, in block-major order.

    Block k of sample s runs iff ``dnn_gate(seed, s, k)``; a run block is four
    tasks: ``t_s = W1_k h_s`` (GEMV), ``t_s = relu(t_s + b1_k)``,
    ``u_s = W2_k t_s`` (GEMV), ``h_s = h_s + (u_s + b2_k)``. Weights and biases
    ~ U[-1/16, 1/16), inputs ~ U[-1, 1). Activations are per sample, so the
    samples' chains are independent; weights are shared read-only. GEMV tasks
    use 1..32 CTAs (seeded), the elementwise ones 1 CTA. With ``weight_sets``
    > 0 block k uses weight set k mod weight_sets (long streams, bounded memory).
    ``shared`` = (W, B) from dnn_weights (weight_sets of them) replaces the
    stream's own weights (many requests serving one model); the inputs then
    come from the seed alone.
    """
    rng = np.random.default_rng(seed)
    H = hidden
    nw = weight_sets if weight_sets > 0 else blocks
    if shared is None:
        W = rng.uniform(-1.0 / 16, 1.0 / 16, (nw, 2, H, H)).astype(np.float32)
        B = rng.uniform(-1.0 / 16, 1.0 / 16, (nw, 2, H)).astype(np.float32)
    else:
        W, B = shared
        assert W.size == nw * 2 * H * H and B.size == nw * 2 * H
    h = rng.uniform(-1.0, 1.0, (batch, H)).astype(np.float32)
    bufs = {"W": W.reshape(-1), "B": B.reshape(-1), "h": h.reshape(-1),
            "t": np.zeros(batch * H, np.float32), "u": np.zeros(batch * H, np.float32)}
    tasks = []
    tid = task_id0
    for k in range(blocks):
        for s in range(batch):
            if not dnn_gate(seed, s, k):
                continue
            kw = k % nw
            w1 = Ref("W", (kw * 2 + 0) * H * H, H * H)
            w2 = Ref("W", (kw * 2 + 1) * H * H, H * H)
            b1 = Ref("B", (kw * 2 + 0) * H, H)
            b2 = Ref("B", (kw * 2 + 1) * H, H)
            hs, ts, us = Ref("h", s * H, H), Ref("t", s * H, H), Ref("u", s * H, H)
            c1 = GEMV_NCTA_CHOICES[mix(seed, 0x61, s, k, 1) % len(GEMV_NCTA_CHOICES)]
            c2 = GEMV_NCTA_CHOICES[mix(seed, 0x61, s, k, 2) % len(GEMV_NCTA_CHOICES)]
            dims = {"m": np.uint32(H), "k": np.uint32(H)}
            tasks.append(Task(tid, "gemv", c1, {"W": w1, "x": hs, "y": ts}, dict(dims))); tid += 1
            tasks.append(Task(tid, "bias_relu", 1, {"t": ts, "b": b1})); tid += 1
            tasks.append(Task(tid, "gemv", c2, {"W": w2, "x": ts, "y": us}, dict(dims))); tid += 1
            tasks.append(Task(tid, "resid", 1, {"h": hs, "u": us, "b": b2})); tid += 1
    return Stream(bufs, tasks, window, f"dnn(seed={seed},batch={batch})")


def dnn_stream_unrolled(seed: int, batch: int = 1, blocks: int = 24, hidden: int = 256,
                        window: int = 32) -> Stream:
    """The computation of ``dnn_stream(seed, batch, blocks, hidden)`` with every
    intermediate kept, so that each task can be re-evaluated on its own inputs
    afterwards. Block k of sample s (when its gate runs it) is six tasks:
    ``p = W1_k h`` (GEMV into a fresh range), ``t = 1 * p`` (scale: a copy),
    ``t = relu(t + b1_k)``, ``u = W2_k t`` (GEMV, fresh), ``h' = 1 * h`` (copy
    into the next hidden-state slot) and ``h' = h' + (u + b2_k)``. Weights,
    biases, inputs, gates and GEMV CTA counts are those of ``dnn_stream``, and
    the copies are exact, so sample s's last hidden-state slot holds what
    ``dnn_stream`` leaves in its ``h``. Buffers: ``h`` [batch][blocks + 1][H]
    (slot 0 the input), ``p``, ``t``, ``u`` [batch][blocks][H]."""
    rng = np.random.default_rng(seed)
    H = hidden
    W = rng.uniform(-1.0 / 16, 1.0 / 16, (blocks, 2, H, H)).astype(np.float32)
    B = rng.uniform(-1.0 / 16, 1.0 / 16, (blocks, 2, H)).astype(np.float32)
    h0 = rng.uniform(-1.0, 1.0, (batch, H)).astype(np.float32)
    h = np.zeros((batch, blocks + 1, H), np.float32)
    h[:, 0] = h0
    z = np.zeros(batch * blocks * H, np.float32)
    bufs = {"W": W.reshape(-1), "B": B.reshape(-1), "h": h.reshape(-1), "p": z, "t": z.copy(), "u": z.copy()}
    one = np.float32(1.0)
    dims = {"m": np.uint32(H), "k": np.uint32(H)}
    cur = [0] * batch
    tasks: List[Task] = []

    def add(op, ncta, arrays, scalars=None):
        tasks.append(Task(len(tasks), op, ncta, arrays, dict(scalars or {})))

    for k in range(blocks):
        for s in range(batch):
            if not dnn_gate(seed, s, k):
                continue
            w1 = Ref("W", (k * 2 + 0) * H * H, H * H)
            w2 = Ref("W", (k * 2 + 1) * H * H, H * H)
            b1 = Ref("B", (k * 2 + 0) * H, H)
            b2 = Ref("B", (k * 2 + 1) * H, H)
            hs = Ref("h", (s * (blocks + 1) + cur[s]) * H, H)
            hn = Ref("h", (s * (blocks + 1) + k + 1) * H, H)
            ps, ts, us = (Ref(n, (s * blocks + k) * H, H) for n in ("p", "t", "u"))
            c1 = GEMV_NCTA_CHOICES[mix(seed, 0x61, s, k, 1) % len(GEMV_NCTA_CHOICES)]
            c2 = GEMV_NCTA_CHOICES[mix(seed, 0x61, s, k, 2) % len(GEMV_NCTA_CHOICES)]
            add("gemv", c1, {"W": w1, "x": hs, "y": ps}, dims)
            add("scale", 1, {"x": ps, "y": ts}, {"a": one})
            add("bias_relu", 1, {"t": ts, "b": b1})
            add("gemv", c2, {"W": w2, "x": ts, "y": us}, dims)
            add("scale", 1, {"x": hs, "y": hn}, {"a": one})
            add("resid", 1, {"h": hn, "u": us, "b": b2})
            cur[s] = k + 1
    st = Stream(bufs, tasks, window, f"dnn_unrolled(seed={seed},batch={batch})")
    st.last_slot = list(cur)
    return st


# ----------------------------------------------------------------------------
# Static irregular DAG (randomly wired network of small GEMVs)
# ----------------------------------------------------------------------------

def small_world_dag(rng, n: int, k: int = 4, p: float = 0.75):
    """Edges (u, v), u < v, of a Watts-Strogatz small-world graph (ring
    lattice, each node joined to its k nearest neighbours, each edge rewired
    with probability p to a uniform random node) oriented from the lower to
    the higher node index, which makes it acyclic."""
    edges = set()
    for u in range(n):
        for d in range(1, k // 2 + 1):
            v = (u + d) % n
            if rng.random() < p:
                w = int(rng.integers(0, n))
                while w == u or (min(u, w), max(u, w)) in edges:
                    w = int(rng.integers(0, n))
                v = w
            a, b = min(u, v), max(u, v)
            if a != b:
                edges.add((a, b))
    return sorted(edges)


def random_wire_stream(seed: int, n_nodes: int = 32, stages: int = 3, k: int = 4, p: float = 0.75,
                       hidden: int = 256, window: int = 32, x: Optional[np.ndarray] = None) -> Stream:
    """A static, randomly wired network (the shape of the paper's RandomWire
    and NAS-cell workloads: an irregular DAG of many small kernels, batch 1).
    Each stage is a small-world DAG of ``n_nodes`` nodes; node v aggregates
    the outputs of its predecessors (or the stage input when it has none)
    into h_v (one ``scale`` by 1 then one ``axpy`` by 1 per further input),
    then y_v = relu(W_v h_v + b_v) (GEMV with 1..8 CTAs, then bias+ReLU). The
    stage output, the next stage's input, sums the outputs of nodes without
    successors. The task graph is the same for every input ``x``."""
    rng = np.random.default_rng(seed)
    H = hidden
    N = n_nodes * stages
    Wt = rng.uniform(-1.0 / 16, 1.0 / 16, (N, H, H)).astype(np.float32)
    Bt = rng.uniform(-1.0 / 16, 1.0 / 16, (N, H)).astype(np.float32)
    xs = np.zeros((stages + 1) * H, np.float32)
    xs[:H] = rng.uniform(-1.0, 1.0, H).astype(np.float32)   # drawn always: the wiring below
    if x is not None:                                         # must not depend on the input
        xs[:H] = x
    bufs = {"W": Wt.reshape(-1), "B": Bt.reshape(-1), "x": xs,
            "h": np.zeros(N * H, np.float32), "y": np.zeros(N * H, np.float32)}
    one = np.float32(1.0)
    dims = {"m": np.uint32(H), "k": np.uint32(H)}
    tasks: List[Task] = []

    def add(op, ncta, arrays, scalars=None):
        tasks.append(Task(len(tasks), op, ncta, arrays, dict(scalars or {})))

    for st in range(stages):
        edges = small_world_dag(rng, n_nodes, k, p)
        preds = {v: [] for v in range(n_nodes)}
        succ = {v: 0 for v in range(n_nodes)}
        for u, v in edges:
            preds[v].append(u)
            succ[u] += 1
        xin = Ref("x", st * H, H)
        for v in range(n_nodes):
            g = st * n_nodes + v
            ins = [Ref("y", (st * n_nodes + u) * H, H) for u in preds[v]] or [xin]
            hv = Ref("h", g * H, H)
            add("scale", 1, {"x": ins[0], "y": hv}, {"a": one})
            for r in ins[1:]:
                add("axpy", 1, {"x": r, "y": hv}, {"a": one})
            ncta = (1, 2, 4, 8)[mix(seed, 0x77, g) % 4]
            add("gemv", ncta, {"W": Ref("W", g * H * H, H * H), "x": hv, "y": Ref("y", g * H, H)}, dims)
            add("bias_relu", 1, {"t": Ref("y", g * H, H), "b": Ref("B", g * H, H)})
        sinks = [v for v in range(n_nodes) if succ[v] == 0]
        xout = Ref("x", (st + 1) * H, H)
        add("scale", 1, {"x": Ref("y", (st * n_nodes + sinks[0]) * H, H), "y": xout}, {"a": one})
        for v in sinks[1:]:
            add("axpy", 1, {"x": Ref("y", (st * n_nodes + v) * H, H), "y": xout}, {"a": one})
    return Stream(bufs, tasks, window, f"random_wire(seed={seed})")


# ----------------------------------------------------------------------------
# Rigid-body RL-simulation stream (E envs x S spheres; input-dependent DAG)
# ----------------------------------------------------------------------------

RL_SPHERES = 32                 # spheres per environment (fixed by the record layout)
RL_REC_BYTES = 1088             # bytes of one environment's contact record
RL_PAIRS = RL_SPHERES * (RL_SPHERES - 1) // 2


@dataclass
class RLParams:
    n_env: int = 256
    steps: int = 50
    chunk: int = 8              # environments per broadphase / integrate task
    box: float = 0.9            # cubic box edge L (about 300 tasks per step)
    dt: float = 1.0 / 240.0
    gravity: float = -9.81
    beta: float = 0.2           # Baumgarte position-error feedback
    slop: float = 0.001
    max_solve_ncta: int = 16
    max_chunk_ncta: int = 4


class RLSim:
    """Task emission for the rigid-sphere stream.

    Per step t the program order is: one ``rl_solve`` task for every
    environment whose contact record reports at least one island, in
    environment order (``ncta = clamp(islands, 1, 16)``); then one
    ``rl_integrate`` task per chunk of environments; then (except after the
    last step) one ``rl_broadphase`` task per chunk for step t+1. The stream
    starts with the broadphase tasks of step 0. Because the solve tasks exist
    only where contacts were found, the DAG depends on the simulated state.

    The caller runs each emitted batch with its own implementation, reads the
    per-environment island counts (buffer ``nisl``) that its broadphase wrote,
    and passes them to :meth:`step_batch`.
    """

    def __init__(self, seed: int, params: Optional[RLParams] = None):
        self.seed = seed
        self.p = params or RLParams()
        if self.p.n_env % self.p.chunk:
            raise ValueError("n_env must be a multiple of chunk")
        self.next_id = 0

    # -- initial state -------------------------------------------------------
    def buffers(self, emit: bool = False) -> Dict[str, np.ndarray]:
        """Initial state; with ``emit`` also the emit tasks' 4-byte token."""
        b = self._buffers()
        if emit:
            b["token"] = np.zeros(1, np.uint32)
        return b

    def _buffers(self) -> Dict[str, np.ndarray]:
        p, S = self.p, RL_SPHERES
        rng = np.random.default_rng(self.seed)
        radius = rng.uniform(0.05, 0.1, (p.n_env, S)).astype(np.float32)
        invmass = rng.uniform(0.5, 2.0, (p.n_env, S)).astype(np.float32)
        u = rng.uniform(0.0, 1.0, (p.n_env, S, 3))
        lo = radius[..., None].astype(np.float64)
        pos = (lo + u * (p.box - 2.0 * lo)).astype(np.float32)
        vel = rng.uniform(-0.5, 0.5, (p.n_env, S, 3)).astype(np.float32)
        prop = np.stack([radius, invmass], axis=-1).astype(np.float32)
        return {"pos": pos.reshape(-1), "vel": vel.reshape(-1), "prop": prop.reshape(-1),
                "cont": np.zeros(p.n_env * RL_REC_BYTES, np.uint8),
                "nisl": np.zeros(p.n_env, np.uint32)}

    @property
    def window(self) -> int:
        return 32

    # -- helpers -----------------------------------------------------------------
    def _chunk_ncta(self, kind: int, step: int, c: int) -> int:
        return 1 + mix(self.seed, 0x71, kind, step, c) % self.p.max_chunk_ncta

    def _refs_env(self, e0: int, ne: int):
        S = RL_SPHERES
        return (Ref("pos", e0 * S * 3, ne * S * 3), Ref("vel", e0 * S * 3, ne * S * 3),
                Ref("prop", e0 * S * 2, ne * S * 2), Ref("cont", e0 * RL_REC_BYTES, ne * RL_REC_BYTES),
                Ref("nisl", e0, ne))

    # -- emission plans ----------------------------------------------------------
    # A plan lists the tasks of one batch in program order as three arrays:
    # kind (0 broadphase of a chunk, 1 solve of an env, 2 integrate of a chunk),
    # index (chunk or env) and ncta, plus the step whose scalars they use.
    KIND_BROADPHASE, KIND_SOLVE, KIND_INTEGRATE = 0, 1, 2

    def _chunks(self) -> np.ndarray:
        return np.arange(self.p.n_env // self.p.chunk, dtype=np.uint32)

    def _chunk_nctas(self, kind: int, step: int) -> np.ndarray:
        return np.array([self._chunk_ncta(kind, step, int(c)) for c in self._chunks()], np.uint16)

    def first_plan(self) -> "RLPlan":
        ch = self._chunks()
        return self._ids(RLPlan(np.zeros(len(ch), np.uint8), ch, self._chunk_nctas(0, 0), 0))

    def step_plan(self, step: int, nisl: np.ndarray) -> "RLPlan":
        """Solve + integrate of ``step`` and broadphase of ``step + 1``."""
        p = self.p
        nisl = np.asarray(nisl).reshape(-1).astype(np.int64)
        if nisl.shape[0] != p.n_env:
            raise ValueError("nisl must hold one count per environment")
        envs = np.nonzero(nisl > 0)[0].astype(np.uint32)
        solve_ncta = np.clip(nisl[envs], 1, p.max_solve_ncta).astype(np.uint16)
        ch = self._chunks()
        kinds = [np.full(len(envs), 1, np.uint8), np.full(len(ch), 2, np.uint8)]
        index = [envs, ch]
        ncta = [solve_ncta, self._chunk_nctas(1, step)]
        if step + 1 < p.steps:
            kinds.append(np.zeros(len(ch), np.uint8))
            index.append(ch)
            ncta.append(self._chunk_nctas(0, step + 1))
        return self._ids(RLPlan(np.concatenate(kinds), np.concatenate(index), np.concatenate(ncta), step))

    def _ids(self, plan: "RLPlan") -> "RLPlan":
        plan.ids = np.arange(self.next_id, self.next_id + len(plan.kind), dtype=np.uint32)
        self.next_id += len(plan.kind)
        return plan

    def scalars(self) -> Dict[str, Dict[str, object]]:
        """Scalar arguments of each task kind (the same every step)."""
        p, f32 = self.p, np.float32
        dt = f32(p.dt)
        return {"rl_broadphase": {"nenv": np.uint32(p.chunk)},
                "rl_solve": {"beta_dt": f32(f32(p.beta) / dt), "slop": f32(p.slop)},
                "rl_integrate": {"nenv": np.uint32(p.chunk), "dt": dt, "gdt": f32(f32(p.gravity) * dt),
                                 "box": f32(p.box)}}

    def tasks(self, plan: "RLPlan") -> List[Task]:
        """The plan as streamgen tasks."""
        p, sc, out = self.p, self.scalars(), []
        for tid, kind, idx, nc in zip(plan.ids, plan.kind, plan.index, plan.ncta):
            idx = int(idx)
            if kind == 1:
                pos, vel, prop, cont, _ = self._refs_env(idx, 1)
                out.append(Task(int(tid), "rl_solve", int(nc),
                                {"pos": pos, "vel": vel, "prop": prop, "cont": cont}, dict(sc["rl_solve"])))
            else:
                pos, vel, prop, cont, nisl = self._refs_env(idx * p.chunk, p.chunk)
                if kind == 0:
                    out.append(Task(int(tid), "rl_broadphase", int(nc),
                                    {"pos": pos, "prop": prop, "cont": cont, "nisl": nisl},
                                    dict(sc["rl_broadphase"])))
                else:
                    out.append(Task(int(tid), "rl_integrate", int(nc), {"pos": pos, "vel": vel, "prop": prop},
                                    dict(sc["rl_integrate"])))
        return out

    # -- device-side emission ------------------------------------------------------
    # In the emitting variant of the stream an ``rl_emit`` task follows each
    # broadphase batch: it reads the island counts and appends the next batch
    # (the same tasks ``step_plan`` lists) followed by the next emit task.
    # Program order: bp(0), emit(0), [solves(0), int(0), bp(1), emit(1)], ...,
    # [solves(T-1), int(T-1)].

    def ncta_table(self) -> np.ndarray:
        """CTA counts of chunk tasks: entry ((t * 2 + k) * n_chunks + c) is the
        broadphase (k = 0) or integrate (k = 1) CTA count of chunk c, step t."""
        nch = self.p.n_env // self.p.chunk
        tab = np.zeros((self.p.steps + 1, 2, nch), np.uint8)
        for t in range(self.p.steps + 1):
            for k in range(2):
                for c in range(nch):
                    tab[t, k, c] = self._chunk_ncta(k, t, c)
        return tab.reshape(-1)

    def emit_task(self, step: int) -> Task:
        """The emit task that follows the broadphase of ``step``."""
        t = Task(self.next_id, "rl_emit", 1,
                 {"nisl": Ref("nisl", 0, self.p.n_env), "token": Ref("token", 0, 1)},
                 {"step": np.uint32(step)})
        self.next_id += 1
        return t

    # -- batches ---------------------------------------------------------------------
    def first_batch(self) -> List[Task]:
        """Broadphase of step 0."""
        return self.tasks(self.first_plan())

    def step_batch(self, step: int, nisl: np.ndarray) -> List[Task]:
        """Solve + integrate of ``step`` and broadphase of ``step + 1``."""
        return self.tasks(self.step_plan(step, nisl))


@dataclass
class RLPlan:
    kind: np.ndarray
    index: np.ndarray
    ncta: np.ndarray
    step: int
    ids: Optional[np.ndarray] = None


# ----------------------------------------------------------------------------
# Sleep stream (scheduler micro-benchmarks: known body time, chosen DAG shape)
# ----------------------------------------------------------------------------

def sleep_chain_stream(n_tasks: int, sleep_ns: int, width: int, window: int = 32,
                       ncta: int = 1) -> Stream:
    """``width`` independent chains interleaved round-robin; each task sleeps
    ``sleep_ns`` and then sets ``y[0] = y[0] * 0.5 + tag`` on its chain's
    buffer (so tasks of one chain conflict and chains are independent)."""
    bufs = {f"c{i}": np.zeros(16, np.float32) for i in range(width)}
    tasks = [Task(t, "sleep", ncta, {"y": Ref(f"c{t % width}", 0, 1)},
                  {"ns": np.uint32(sleep_ns), "tag": np.float32(t % 7 + 1)})
             for t in range(n_tasks)]
    return Stream(bufs, tasks, window, f"sleep(n={n_tasks},w={width})")


# ----------------------------------------------------------------------------
# Batched streams (many independent streams of uneven length)
# ----------------------------------------------------------------------------

def loguniform_lengths(seed: int, n: int, lo: int = 100, hi: int = 5000) -> List[int]:
    rng = np.random.default_rng(seed)
    return [int(round(math.exp(x))) for x in rng.uniform(math.log(lo), math.log(hi), n)]


@dataclass
class BatchSpec:
    """One stream of a batch: ``kind`` 'rl' (an emitting rigid-sphere run) or
    'dnn' (gated residual MLP inference), sized to about ``target`` tasks by
    whole simulation steps or whole blocks."""
    kind: str
    seed: int
    target: int
    rl: Optional[RLParams] = None
    dnn_batch: int = 1
    dnn_blocks: int = 24


RL_BATCH_ENVS = 64          # environments of an RL stream in a batch (~75 tasks per step)


def batched_specs(seed: int, n_streams: int = 64, lo: int = 100, hi: int = 5000) -> List[BatchSpec]:
    """Independent streams of uneven length (log-uniform in [lo, hi] tasks),
    alternating rigid-sphere and dynamic-DNN kinds."""
    out = []
    for i, L in enumerate(loguniform_lengths(seed, n_streams, lo, hi)):
        sseed = mix(seed, 0xB7, i) & 0xFFFFFFFF
        if i % 2 == 0:
            per_step = RL_BATCH_ENVS + 2 * (RL_BATCH_ENVS // 8) + 1
            steps = max(1, int(round(L / per_step)))
            out.append(BatchSpec("rl", sseed, L, rl=RLParams(n_env=RL_BATCH_ENVS, steps=steps)))
        else:
            b = 1 + (i // 2) % 8
            blocks = max(1, int(round(L / (2 * b))))      # ~4 tasks per sample for half the blocks
            out.append(BatchSpec("dnn", sseed, L, dnn_batch=b, dnn_blocks=blocks))
    return out


# ----------------------------------------------------------------------------
# Serving: Poisson arrivals of requests drawn from a catalogue of streams
# ----------------------------------------------------------------------------

DNN_SERVE_BATCHES = (1, 2, 4, 8)
DNN_SERVE_WEIGHT_SETS = 24


def serving_catalogue(seed: int, n_types: int = 256, lo: int = 100, hi: int = 5000) -> List[BatchSpec]:
    """Request types: half rigid-sphere runs (64 environments, device-side
    emission), half gated-MLP inferences (batch in {1, 2, 4, 8}, the 24 shared
    weight sets of one model), each of a length log-uniform in [lo, hi]
    tasks, kinds interleaved."""
    out = []
    for i, L in enumerate(loguniform_lengths(mix(seed, 0x5E) & 0xFFFFFFFF, n_types, lo, hi)):
        sseed = mix(seed, 0x5F, i) & 0xFFFFFFFF
        if i % 2 == 0:
            per_step = RL_BATCH_ENVS + 2 * (RL_BATCH_ENVS // 8) + 1
            steps = max(1, int(round(L / per_step)))
            out.append(BatchSpec("rl", sseed, L, rl=RLParams(n_env=RL_BATCH_ENVS, steps=steps)))
        else:
            b = DNN_SERVE_BATCHES[mix(seed, 0x60, i) % len(DNN_SERVE_BATCHES)]
            blocks = max(1, int(round(L / (2 * b))))
            out.append(BatchSpec("dnn", sseed, L, dnn_batch=b, dnn_blocks=blocks))
    return out


def poisson_arrivals(seed: int, n: int, rate: float, n_types: int):
    """(arrival times in s, catalogue index) of n requests: exponential gaps of
    mean 1/rate, request types uniform over the catalogue."""
    rng = np.random.default_rng(mix(seed, 0x61) & 0xFFFFFFFF)
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    kinds = rng.integers(0, n_types, n)
    return t, kinds
