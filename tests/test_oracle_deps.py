"""Pins for the dependency oracle (Alg. 1 overlap test, DAG E, window DAG D_W,
legality check) against the paper's printed example, closed forms, hand-written
expected edges and an independently written buffer tracker. CPU only."""
import itertools
import os
import random

import numpy as np
import pytest

import streamgen as sg
from oracle import addresses, deps, execute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --- Alg. 1 overlap test ------------------------------------------------------

@pytest.mark.parametrize("a,b,want", [
    ((0, 4), (4, 4), False),          # adjacent: end1 == start2
    ((4, 4), (0, 4), False),
    ((0, 5), (4, 4), True),           # one shared byte
    ((7, 1), (0, 8), True),           # contained single byte
    ((0, 8), (2, 2), True),           # containment
    ((0, 0), (0, 8), False),          # zero size never overlaps
    ((3, 0), (0, 8), False),
    ((0, 8), (3, 0), False),
    (deps.WHOLE_MEMORY, (123456, 1), True),   # indirect access: all memory
    (deps.WHOLE_MEMORY, ((1 << 64) - 1, 1), True),
    ((100, 10), (50, 50), False),     # [100,110) vs [50,100)
    ((100, 10), (50, 51), True),
])
def test_overlap_truth_table(a, b, want):
    assert deps.overlap(a, b) == want
    assert deps.overlap(b, a) == want


# --- the paper's get_addresses worked example (Sec. IV-A) -------------------

def test_getaddress_matmul_golden():
    with open(os.path.join(GOLDEN, "getaddress_matmul.txt")) as f:
        rows = [ln for ln in f if ln.strip() and not ln.startswith("#")]
    assert rows
    for ln in rows:
        head, rd, wr = [p.split() for p in ln.split("|")]
        m, n, k, elt, i1, i2, out = map(int, head)
        reads, writes = addresses.matmul_segments(i1, i2, out, m, n, k, elt)
        assert reads == [tuple(map(int, s.split(":"))) for s in rd]
        assert writes == [tuple(map(int, s.split(":"))) for s in wr]


def test_gemv_roles_follow_matmul_example():
    # The GEMV task is the k = 1 case of the example: W (m x n) and x (n) read, y (m) written.
    bufs = {"W": np.zeros(6, np.float32), "x": np.zeros(3, np.float32), "y": np.zeros(2, np.float32)}
    t = sg.Task(0, "gemv", 1, {"W": sg.Ref("W", 0, 6), "x": sg.Ref("x", 0, 3), "y": sg.Ref("y", 0, 2)},
                {"m": 2, "k": 3})
    lay = addresses.Layout(bufs)
    reads, writes = addresses.task_segments(t, lay)
    want_r, want_w = addresses.matmul_segments(lay.base["W"], lay.base["x"], lay.base["y"], 2, 3, 1, 4)
    assert reads == want_r and writes == want_w


# --- hand-made streams with hand-written edges --------------------------------

def _seg(buf, lo=0, n=4):
    return ((buf + 1) << 20) + lo, n


HANDMADE = {
    # name: (stream of (reads, writes) over buffers 0..3, expected E)
    "raw_chain": ([([], [_seg(0)]), ([_seg(0)], [_seg(1)]), ([_seg(1)], [_seg(2)])],
                  {(0, 1), (1, 2)}),
    "war_only": ([([_seg(0)], []), ([], [_seg(0)])], {(0, 1)}),
    "waw_only": ([([], [_seg(0)]), ([], [_seg(0)])], {(0, 1)}),
    "read_read": ([([_seg(0)], [_seg(1)]), ([_seg(0)], [_seg(2)])], set()),
    "inplace_axpy": ([([_seg(0), _seg(1)], [_seg(1)]), ([_seg(0), _seg(1)], [_seg(1)]),
                      ([_seg(2), _seg(3)], [_seg(3)])], {(0, 1)}),
    "fan_out": ([([], [_seg(0)]), ([_seg(0)], [_seg(1)]), ([_seg(0)], [_seg(2)]),
                 ([_seg(0)], [_seg(3)])], {(0, 1), (0, 2), (0, 3)}),
    "wildcard": ([([], [_seg(0)]), ([deps.WHOLE_MEMORY], [_seg(3)]), ([_seg(2)], [_seg(2)]),
                  ([], [deps.WHOLE_MEMORY])], {(0, 1), (1, 2), (1, 3), (2, 3), (0, 3)}),
    "zero_size": ([([], [_seg(0, 0, 0)]), ([_seg(0)], [_seg(0, 0, 0)])], set()),
    "partial_ranges": ([([], [_seg(0, 0, 8)]), ([_seg(0, 8, 8)], [_seg(1)]),
                        ([_seg(0, 7, 2)], [_seg(2)])], {(0, 2)}),
}


@pytest.mark.parametrize("name", sorted(HANDMADE))
def test_handmade_streams(name):
    stream, want = HANDMADE[name]
    assert deps.full_dag(stream) == want


def test_literal_alg1_misses_raw():
    # Alg. 1 as printed tests only the new kernel's writes; a pure RAW pair
    # (writer then reader) is then missed, which is why the reading adds RAW.
    w, r = ([], [_seg(0)]), ([_seg(0)], [_seg(1)])
    literal = any(deps.overlap(s, t) for s in r[1] for t in w[0] + w[1])
    assert not literal
    assert deps.full_dag([w, r]) == {(0, 1)}


# --- exhaustive comparison against an independent buffer tracker -------------

def tracker_dag(stream_sets):
    """Independent formulation over whole one-element buffers: task j depends on
    every earlier writer of a buffer it touches and on every earlier reader of a
    buffer it writes."""
    writers, readers = {}, {}
    E = set()
    for j, (rs, ws) in enumerate(stream_sets):
        for b in set(rs) | set(ws):
            E |= {(i, j) for i in writers.get(b, ())}
        for b in ws:
            E |= {(i, j) for i in readers.get(b, ())}
        for b in rs:
            readers.setdefault(b, []).append(j)
        for b in ws:
            writers.setdefault(b, []).append(j)
    return E


SUBSETS = [frozenset(c) for r in range(4) for c in itertools.combinations(range(3), r)]
PATTERNS = [(r, w) for r in SUBSETS for w in SUBSETS]      # 64 R/W patterns per task


def _as_segments(stream_sets):
    return [([_seg(b) for b in sorted(r)], [_seg(b) for b in sorted(w)]) for r, w in stream_sets]


def test_exhaustive_pairs():
    for p in PATTERNS:
        for q in PATTERNS:
            st = [p, q]
            assert deps.full_dag(_as_segments(st)) == tracker_dag(st)


def test_exhaustive_triples():
    for st in itertools.product(PATTERNS, repeat=3):
        assert deps.full_dag(_as_segments(st)) == tracker_dag(st), st


def test_random_quads():
    rng = random.Random(7)
    for _ in range(20000):
        st = [rng.choice(PATTERNS) for _ in range(4)]
        assert deps.full_dag(_as_segments(st)) == tracker_dag(st), st


# --- closed-form special cases -------------------------------------------------

def test_all_writers_of_one_buffer_form_a_chain_in_E():
    n = 9
    st = [([], [_seg(0)]) for _ in range(n)]
    E = deps.full_dag(st)
    assert E == {(i, j) for j in range(n) for i in range(j)}
    assert deps.dag_stats(E, n)["depth"] == n


def test_disjoint_tasks_have_no_edges():
    st = [([_seg(2 * i)], [_seg(2 * i + 1)]) for i in range(8)]
    assert deps.full_dag(st) == set()


def test_window_dag_limits():
    s = sg.elementwise_stream(3, n_tasks=40)
    E = deps.full_dag(addresses.stream_segments(s.tasks, s.buffers))
    assert deps.window_dag(E, 40) == E            # W >= n: D_W = E
    assert deps.window_dag(E, 1) == set()          # W = 1: no candidates
    for W in (2, 8, 33):
        D = deps.window_dag(E, W)
        assert D <= E and all(j - i <= W - 1 for i, j in D)
        assert all((i, j) in D for i, j in E if j - i < W)


def test_edges_from_masks_roundtrip():
    s = sg.elementwise_stream(5, n_tasks=64)
    E = deps.full_dag(addresses.stream_segments(s.tasks, s.buffers))
    for W in (1, 2, 8, 32, 64):
        D = deps.window_dag(E, W)
        masks = [0] * 64
        for i, j in D:
            masks[j] |= 1 << (i % W)
        assert deps.edges_from_masks(masks, W) == D


# --- legality checker ------------------------------------------------------------

def test_legality_accepts_in_order_and_rejects_planted_violation():
    E = {(0, 1), (1, 2), (0, 2)}
    start, retire = [0, 2, 4], [1, 3, 5]
    assert deps.check_legal(E, start, retire) == []
    bad_start = [0, 2, 2]                    # task 2 starts with task 1 still running
    out = deps.check_legal(E, bad_start, [1, 3, 5])
    assert out and "edge (1,2)" in out[0]


# --- the window reading: a CPU simulation of ring-window issue -------------------

def _simulate_ring_window(n, E, W, rng):
    """Issue tasks under the ring-window reading: task j may enter once task
    j - W retired (in-order release), and may start once its D_W upstream tasks
    retired. Completion order is random. Returns (start, retire) tickets."""
    D = deps.window_dag(E, W)
    ups = {j: {i for i, jj in D if jj == j} for j in range(n)}
    ticket = 0
    start, retire = [None] * n, [None] * n
    entered, running, done = 0, set(), set()
    while len(done) < n:
        while entered < n and (entered < W or all(k in done for k in range(entered - W + 1))):
            entered += 1
        ready = [j for j in range(entered) if start[j] is None and ups[j] <= done]
        for j in ready:
            start[j] = ticket; ticket += 1
            running.add(j)
        j = rng.choice(sorted(running))
        running.discard(j)
        retire[j] = ticket; ticket += 1
        done.add(j)
    return start, retire


@pytest.mark.parametrize("seed", range(5))
def test_ring_window_issue_is_legal_and_schedule_independent(seed):
    s = sg.elementwise_stream(seed, n_tasks=48, ranges=bool(seed % 2))
    E = deps.full_dag(addresses.stream_segments(s.tasks, s.buffers))
    ref = execute.run_inorder(s.buffers, s.tasks)
    rng = random.Random(seed)
    for W in (1, 2, 8, 32):
        start, retire = _simulate_ring_window(len(s.tasks), E, W, rng)
        assert deps.check_legal(E, start, retire) == []
        order = sorted(range(len(s.tasks)), key=lambda j: start[j])
        out = execute.run_inorder(s.buffers, s.tasks, order)
        for k in ref:
            assert np.array_equal(ref[k], out[k])


def test_window_dag_direct_equals_window_of_E():
    for seed in range(4):
        s = sg.elementwise_stream(seed, n_tasks=70, ranges=True)
        segs = addresses.stream_segments(s.tasks, s.buffers)
        E = deps.full_dag(segs)
        for W in (1, 2, 8, 33):
            assert deps.window_dag_direct(segs, W) == deps.window_dag(E, W)


def test_release_order_check_accepts_ring_issue_and_rejects_a_violation():
    s = sg.elementwise_stream(8, n_tasks=48)
    E = deps.full_dag(addresses.stream_segments(s.tasks, s.buffers))
    start, retire = _simulate_ring_window(len(s.tasks), E, 8, random.Random(0))
    assert deps.check_release_order(start, retire, 8) == []
    bad = list(start)
    bad[20] = -1                                # starts before anything retired
    assert deps.check_release_order(bad, retire, 8)


def test_serving_arrivals_and_catalogue():
    """The serving workload's inputs: exponential gaps of mean 1/rate, request
    kinds half and half, lengths within [lo, hi]."""
    t, k = sg.poisson_arrivals(1, 20000, 2000.0, 256)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert (gaps > 0).all() and abs(gaps.mean() - 1 / 2000.0) < 0.03 / 2000.0
    assert abs(np.std(gaps) / gaps.mean() - 1.0) < 0.05          # exponential: cv = 1
    assert k.min() >= 0 and k.max() < 256
    cat = sg.serving_catalogue(1, n_types=256)
    assert sum(c.kind == "rl" for c in cat) == 128
    assert all(100 <= c.target <= 5000 for c in cat)
    assert {c.dnn_batch for c in cat if c.kind == "dnn"} == {1, 2, 4, 8}


def test_random_wire_inputs():
    """The static randomly wired network: edges point from lower to higher
    node index (acyclic), every node aggregates at least one input, the task
    structure does not depend on the input vector, and the DAG's critical
    path is far shorter than the stream (irregular parallelism)."""
    rng = np.random.default_rng(3)
    edges = sg.small_world_dag(rng, 32, 4, 0.75)
    assert all(u < v for u, v in edges) and len(set(edges)) == len(edges)
    assert 40 <= len(edges) <= 64
    a = sg.random_wire_stream(1)
    b = sg.random_wire_stream(1, x=np.ones(256, np.float32))
    assert [(t.op, t.ncta, t.arrays) for t in a.tasks] == [(t.op, t.ncta, t.arrays) for t in b.tasks]
    E = deps.full_dag(addresses.stream_segments(a.tasks, a.buffers))
    depth = [1] * len(a.tasks)
    for i, j in sorted(E, key=lambda e: e[1]):
        depth[j] = max(depth[j], depth[i] + 1)
    assert max(depth) * 3 < len(a.tasks)
