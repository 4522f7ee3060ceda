"""bench.py on the CPU: the reference arm's one JSON line with the keys the
benchmark contract requires (the default workload and a per-input one), and
the critical-path bound computed from a logged DAG."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
REQUIRED = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
            "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"}


@pytest.mark.parametrize("workload", ["rlsim", "static"])
def test_reference_arm_json_line(workload):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", workload,
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=300,
                       env=dict(os.environ, RANK="0", WORLD_SIZE="1"))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert REQUIRED <= set(line)
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "tasks/s"
    assert line["higher_is_better"] is True and line["n_gpus"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["config"]["workload"]


class _FakeCtx:
    """Stands in for a traced context: logged masks (bit = predecessor's slot,
    seq mod span) and trace rows for a hand-made DAG."""

    def __init__(self, span, first, edges, body_us):
        self.span, self.first = span, first
        n = len(body_us)
        self.masks = np.zeros(n, np.uint64)
        for i, j in edges:
            self.masks[j] |= np.uint64(1 << ((first + i) % span))
        self.tr = np.zeros((n, 5), np.uint64)
        self.tr[:, 2] = 1000
        self.tr[:, 3] = 1000 + (np.array(body_us) * 1000).astype(np.uint64)

    def log(self, stream, first, n):
        assert first == self.first and n == len(self.masks)
        return self.masks, None, None

    def trace(self, stream, first, n):
        return self.tr


@pytest.mark.parametrize("first", [0, 6, 13])
def test_critical_path_of_a_logged_dag(first):
    import bench
    # 0->1->3->5, 2->3->5, 4->5 with bodies 1, 2, 5, 1, 1, 1 us: the longest
    # chain is 2 -> 3 -> 5 (7 us, 3 tasks)
    ctx = _FakeCtx(4, first, [(0, 1), (1, 3), (2, 3), (3, 5), (4, 5)], [1, 2, 5, 1, 1, 1])
    us, k = bench.critical_path(ctx, 0, first, 6)
    assert abs(us - 7.0) < 1e-9 and k == 3
    # no edges: the longest single body
    ctx = _FakeCtx(4, first, [], [1, 2, 5, 1, 1, 1])
    assert bench.critical_path(ctx, 0, first, 6) == (5.0, 1)


@pytest.mark.parametrize("first", [0, 5])
def test_window_bound_of_a_logged_stream(first):
    import bench
    # no conflicts, window 2: task j waits for every task j - 2 or further back
    # to end; bodies 1, 2, 3, 4 us give ends 1, 2, 4, 6
    ctx = _FakeCtx(8, first, [], [1, 2, 3, 4])
    assert bench.window_bound(ctx, first, 4, 2, [-1] * 4) == {"start": 6.0, "end": 6.0}
    # a wide window: the chain 0 -> 1 -> 2 (1 + 2 + 3 us) binds, task 3 runs beside it
    ctx = _FakeCtx(8, first, [(0, 1), (1, 2)], [1, 2, 3, 1])
    assert bench.window_bound(ctx, first, 4, 8, [-1] * 4) == {"start": 6.0, "end": 6.0}
    # tasks 1 and 2 appended by the emit task 0 (2 us): released at its start
    # they end at 1 us and the emit binds (2 us); at its end, 2 + 1 us
    ctx = _FakeCtx(8, first, [], [2, 1, 1])
    assert bench.window_bound(ctx, first, 3, 8, [-1, 0, 0]) == {"start": 2.0, "end": 3.0}


@pytest.mark.parametrize("seed", range(6))
def test_full_dag_critical_path_against_brute_force(seed):
    """bench.critical_path_full (per-byte last writer / readers) against the
    longest path over the oracle's all-pairs DAG E, on random small streams
    with read-write ranges, zero-size segments and distant conflicts."""
    import bench
    from oracle import deps
    rng = np.random.default_rng(seed)
    base = 1 << 30
    segs, body = [], []
    for _ in range(120):
        def one():
            return (base + int(rng.integers(0, 4096)) * 4 * (1 + seed % 2), int(rng.integers(0, 65)) * 4)
        rd = [one() for _ in range(int(rng.integers(0, 4)))]
        wr = [one() for _ in range(int(rng.integers(0 if rd else 1, 3)))]
        if wr and rng.random() < 0.3:
            rd.append(wr[0])                        # a read-modify-write range
        segs.append((rd, wr))
        body.append(float(rng.integers(1, 50)))
    E = deps.full_dag(segs)
    preds = {}
    for i, j in E:
        preds.setdefault(j, []).append(i)
    fin = []
    for j in range(len(segs)):
        fin.append(body[j] + max((fin[i] for i in preds.get(j, [])), default=0.0))
    us, k = bench.critical_path_full(segs, body)
    assert abs(us - max(fin)) < 1e-9
    assert 1 <= k <= len(segs)
