"""CPU oracle for ACS (arXiv 2401.12377) -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct CPU code that states what the GPU path must
compute:

* ``deps``      -- the segment-overlap test of Alg. 1 (Sec. IV-B), extended to
                   read-after-write, as a brute-force all-pairs builder of the
                   full dependency DAG E and of the window DAG D_W, plus the
                   launch-legality check (no task starts before a conflicting
                   predecessor retired).
* ``addresses`` -- read/write segment resolution from a task's operands
                   (the ``get_addresses`` wrapper of Sec. IV-A).
* ``execute``   -- an in-order executor of the task bodies: the memory state the
                   method must reproduce, since correct out-of-order issue is
                   schedule-independent.
* ``rlsim.c``   -- the rigid-sphere task bodies in plain C (fp32, no
                   contraction), loaded through ctypes.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package. It shares no code with ``paper_2401_12377_b300`` and
never imports it; the two meet only in the seeded inputs of ``streamgen``.

Parity status per function is stated in each module header.
"""
