"""Host-side checks on the CPU (no device). The serving loop's admission policy: oldest first,
a free stream slot and the device budget both required, and no request
overtakes the head of the queue."""
import collections

from paper_2401_12377_b300.serving import admit_fifo


def _q(xs):
    return collections.deque(xs)


def test_admits_in_arrival_order_while_slots_and_budget_last():
    need = {0: 4, 1: 3, 2: 2, 3: 1}.__getitem__
    waiting, free = _q([0, 1, 2, 3]), _q([7, 5, 6])
    out = admit_fifo(waiting, free, 0, 100, need)
    assert out == [(0, 7), (1, 5), (2, 6)]          # slots run out first
    assert list(waiting) == [3] and not free


def test_budget_blocks_the_head_and_everything_behind_it():
    need = {0: 6, 1: 5, 2: 1}.__getitem__
    waiting, free = _q([0, 1, 2]), _q([0, 1, 2])
    out = admit_fifo(waiting, free, 0, 10, need)
    assert out == [(0, 0)]                          # 6 + 5 > 10: request 1 waits, 2 does not overtake
    assert list(waiting) == [1, 2] and list(free) == [1, 2]
    # bytes already in use count against the budget
    assert admit_fifo(_q([2]), _q([0]), 10, 10, need) == []
    assert admit_fifo(_q([2]), _q([0]), 9, 10, need) == [(2, 0)]


def test_nothing_waiting_or_no_slot():
    assert admit_fifo(_q([]), _q([0]), 0, 10, lambda r: 1) == []
    w = _q([0])
    assert admit_fifo(w, _q([]), 0, 10, lambda r: 1) == [] and list(w) == [0]


def test_emit_driver_rejects_a_zero_cta_count():
    """A device emitter takes its chunk CTA counts from the table as they are,
    so the host driver refuses a table with a 0 before anything reaches the
    device."""
    import numpy as np
    import pytest
    import streamgen as sg
    from paper_2401_12377_b300 import harness

    class Sim(sg.RLSim):
        def ncta_table(self):
            t = super().ncta_table()
            t[3] = 0
            return t

    with pytest.raises(ValueError, match="ncta_table"):
        harness.RLEmitDriver(Sim(1, sg.RLParams(n_env=16, steps=2)), bufs=None, ctx=None)
