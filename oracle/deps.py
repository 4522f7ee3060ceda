"""Brute-force dependency oracle (test infrastructure only).

Follows the dependency check of Alg. 1 (Sec. IV-B, "The window module") and the
state semantics of Sec. III-C ("Tracking kernel state at runtime"):

* Overlap of two byte segments ``[start, start + size)`` is the test printed in
  Alg. 1: ``start1 < end2 and end1 > start2`` with ``end = start + size``.
  Python integers are unbounded, so nothing overflows; the "whole memory"
  segment for indirect access (Sec. IV-A) is ``(0, 2**64)``.
* Alg. 1 compares only the *new* kernel's write segments with the window
  kernel's read and write segments, which leaves out read-after-write. Reading
  used here (Sec. III-C states dependencies follow from read/write overlap in
  general): task j depends on an earlier task i iff a write segment of j
  overlaps any segment of i, or a read segment of j overlaps a write segment of
  i. Read/read never conflicts; a task never depends on itself.
* E is the full DAG over all pairs i < j. D_W keeps the edges of E whose
  distance is at most W - 1: with a ring of W slots released in program order,
  exactly tasks j-W+1 .. j-1 share the window with task j when it is inserted
  (the HW window has N slots and N-1 upstream entries, Sec. IV-C), and every
  farther edge is satisfied because task j cannot enter before task j-W
  retired.

Pinned by: the overlap truth table, hand-made streams with hand-written edges,
an exhaustive comparison against an independent last-writer/readers tracker on
all tiny streams, and closed-form special cases (see tests/test_oracle_deps.py).
"""
from __future__ import annotations

from typing import Dict, Iterable, List, Sequence, Set, Tuple

WHOLE_MEMORY = (0, 1 << 64)

Segment = Tuple[int, int]          # (start byte, size in bytes)


def overlap(a: Segment, b: Segment) -> bool:
    """Alg. 1's test on half-open byte ranges.

    A zero-size segment holds no byte and never overlaps (Alg. 1's strict test
    alone would report an empty range lying strictly inside another one)."""
    if a[1] == 0 or b[1] == 0:
        return False
    s1, e1 = a[0], a[0] + a[1]
    s2, e2 = b[0], b[0] + b[1]
    return s1 < e2 and e1 > s2


def conflict(reads_i: Sequence[Segment], writes_i: Sequence[Segment],
             reads_j: Sequence[Segment], writes_j: Sequence[Segment]) -> bool:
    """True iff later task j must wait for earlier task i (RAW, WAR or WAW)."""
    for s in writes_j:                       # WAW and WAR
        for t in list(reads_i) + list(writes_i):
            if overlap(s, t):
                return True
    for s in reads_j:                        # RAW
        for t in writes_i:
            if overlap(s, t):
                return True
    return False


def full_dag(segs: Sequence[Tuple[Sequence[Segment], Sequence[Segment]]]) -> Set[Tuple[int, int]]:
    """E = {(i, j) : i < j and conflict(i, j)} over a stream of (reads, writes)."""
    E = set()
    n = len(segs)
    for j in range(n):
        rj, wj = segs[j]
        for i in range(j):
            ri, wi = segs[i]
            if conflict(ri, wi, rj, wj):
                E.add((i, j))
    return E


def window_dag(E: Iterable[Tuple[int, int]], window: int) -> Set[Tuple[int, int]]:
    """D_W = {(i, j) in E : j - i <= W - 1}."""
    if window < 1:
        raise ValueError("window must be >= 1")
    return {(i, j) for (i, j) in E if j - i <= window - 1}


def window_dag_direct(segs, window: int) -> Set[Tuple[int, int]]:
    """D_W built directly: the same conflict test, only over pairs at distance
    at most W - 1 (for streams too long for the all-pairs E)."""
    if window < 1:
        raise ValueError("window must be >= 1")
    D = set()
    for j in range(len(segs)):
        rj, wj = segs[j]
        for i in range(max(0, j - window + 1), j):
            ri, wi = segs[i]
            if conflict(ri, wi, rj, wj):
                D.add((i, j))
    return D


def check_release_order(start: Sequence[int], retire: Sequence[int], window: int) -> List[str]:
    """Every task j starts after all tasks i <= j - W retired. With legality on
    D_W this implies legality on all of E: every edge of E longer than W - 1 is
    covered (the ring-window reading of Sec. IV-C's bounded window)."""
    bad = []
    run_max = -1
    for j in range(len(start)):
        i = j - window
        if i >= 0:
            run_max = max(run_max, retire[i])
            if not run_max < start[j]:
                bad.append(f"task {j}: starts at {start[j]} before task <= {i} retired ({run_max})")
    return bad


def check_legal(E: Iterable[Tuple[int, int]], start: Sequence[int], retire: Sequence[int]) -> List[str]:
    """Launch-legality of a ticketed execution log.

    ``start[j]`` is the smallest ticket any CTA of task j drew when it began,
    ``retire[i]`` the ticket drawn when task i's last CTA finished (tickets are
    drawn from one counter). Legal iff every task started before it retired and
    every conflicting predecessor retired before its dependent started. Returns
    the list of violations (empty when legal).
    """
    bad = []
    for j in range(len(start)):
        if not start[j] < retire[j]:
            bad.append(f"task {j}: start {start[j]} not before retire {retire[j]}")
    for (i, j) in sorted(E):
        if not retire[i] < start[j]:
            bad.append(f"edge ({i},{j}): retire {retire[i]} not before start {start[j]}")
    return bad


def edges_from_masks(masks: Sequence[int], window: int) -> Set[Tuple[int, int]]:
    """Decode per-task upstream-candidate masks of a ring window into edges.

    Bit b of task j's mask names the slot b of the W-slot ring; the task in that
    slot is the unique i in [j-W+1, j-1] with i mod W == b.
    """
    E = set()
    for j, m in enumerate(masks):
        b = 0
        while m:
            if m & 1:
                i = j - ((j - b) % window)
                if i == j or i < 0:
                    raise ValueError(f"task {j}: mask names its own or a missing slot {b}")
                E.add((i, j))
            m >>= 1
            b += 1
    return E


def dag_stats(E: Set[Tuple[int, int]], n: int) -> Dict[str, float]:
    """Depth (longest chain, in tasks) and average width n / depth of a DAG."""
    depth = [1] * n
    for (i, j) in sorted(E, key=lambda e: e[1]):
        depth[j] = max(depth[j], depth[i] + 1)
    d = max(depth) if n else 0
    return {"tasks": n, "edges": len(E), "depth": d, "width": (n / d) if d else 0.0}
