"""acs_run_noalloc, the entry point for callers that cannot allocate (code
inside a framework that owns the device memory budget, or a path that cannot
absorb an allocator's latency or failure): it must give exactly what the
regular entry points (acs_init / acs_submit_ops / acs_flush / acs_sync) give,
on consecutive calls that share its fixed scratch array. Collected last on
purpose."""
import numpy as np
import pytest
import torch

import streamgen as sg

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2401_12377_b300 import build
    build.build()
    from paper_2401_12377_b300 import acs, harness


def _noalloc_run(stream, window):
    bufs = harness.DeviceBuffers(stream.buffers)
    ids, packed = harness.pack_tasks(stream.tasks, bufs)
    torch.cuda.synchronize()
    rc = acs.acs_run_noalloc(window, ids, packed, torch.cuda.current_stream().cuda_stream)
    assert rc == acs.ACS_OK, acs.acs_strerror(rc)
    return bufs.download()


@pytest.mark.parametrize("make,window", [
    (lambda: sg.elementwise_stream(17, n_tasks=64, ranges=True), 8),
    (lambda: sg.dnn_stream(23, batch=4, blocks=8), 32),
])
def test_noalloc_matches_the_regular_path_on_two_calls_in_a_row(make, window):
    s = make()
    ref, _, _ = harness.run_stream(s, window=window)        # acs_init .. acs_sync
    for call in range(2):                                    # the scratch keeps the last call's contents
        out = _noalloc_run(s, window)
        for k in ref:
            # same kernels and the same fixed reduction order: bit-identical
            assert np.array_equal(out[k].view(np.uint8), ref[k].view(np.uint8)), (call, k)


def test_noalloc_rejects_more_tasks_than_its_scratch_holds():
    n = acs.ACS_NOALLOC_MAX_TASKS + 1 if hasattr(acs, "ACS_NOALLOC_MAX_TASKS") else 4097
    ids = np.arange(n, dtype=np.uint32)
    packed = np.zeros(n, acs.ARGS_DTYPE)
    packed["ncta"] = 1
    assert acs.acs_run_noalloc(8, ids, packed) == acs.ACS_ERR_INVALID
    assert acs.acs_run_noalloc(0, ids[:1], packed[:1]) == acs.ACS_ERR_INVALID


def test_noalloc_at_its_limits_matches_the_oracle():
    """The largest call the scratch array takes: ACS_NOALLOC_MAX_TASKS tasks,
    window 64, every task 256 CTAs, so the work ring carries as many units as
    can ever be in flight. Outputs must equal the oracle's in-order run bit for
    bit (elementwise bodies round each operation once, like the oracle)."""
    from oracle import execute
    s = sg.elementwise_stream(5, n_tasks=acs.ACS_NOALLOC_MAX_TASKS, n_buffers=64, window=64)
    for t in s.tasks:
        t.ncta = acs.ACS_MAX_NCTA
    ref = execute.run_inorder(s.buffers, s.tasks)
    for call in range(2):
        out = _noalloc_run(s, 64)
        for k in ref:
            assert np.array_equal(out[k].view(np.uint8), ref[k].view(np.uint8)), (call, k)
