"""The C ABI library loads and exports every entry point include/acs.h
declares; host-only entry points behave as documented. CPU only."""
import ctypes as C
import os
import re

import pytest

from paper_2401_12377_b300 import acs, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return acs.load()


def _declared():
    txt = open(os.path.join(ROOT, "include", "acs.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(acs_\w+)\s*\(", txt, flags=re.M)))


def test_header_declares_the_documented_api():
    names = _declared()
    for n in ["acs_init", "acs_submit", "acs_submit_stream", "acs_submit_ops", "acs_flush", "acs_sync",
              "acs_get_log", "acs_get_stats", "acs_get_addresses", "acs_destroy", "acs_strerror"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(acs.EXPORTS)


def test_struct_sizes_match_the_header(lib):
    assert C.sizeof(acs.acs_segment) == 16
    assert C.sizeof(acs.acs_args) == 56
    cfg = acs.acs_config_default()
    assert cfg.n_streams == 1 and cfg.capacity == 8192 and cfg.timeout_ns == 5_000_000_000 and cfg.device == -1


def test_strerror_covers_codes(lib):
    for code in range(0, -8, -1):
        assert acs.acs_strerror(code) != "unknown status"
    assert acs.acs_strerror(-99) == "unknown status"


def _args(op, fields, ncta=1):
    from paper_2401_12377_b300.harness import _args_row
    row = _args_row(op, ncta, fields)
    a = acs.acs_args()
    C.memmove(C.byref(a), row.tobytes(), C.sizeof(a))
    return a


def test_get_addresses_gemv_follows_the_matmul_example(lib):
    # Sec. IV-A example: a product reads m*n and n*k elements, writes m*k (here k = 1 column)
    r, w = acs.acs_get_addresses(_args("gemv", {"W": 4096, "x": 8192, "y": 16384, "m": 3, "k": 5}))
    assert r == [(4096, 3 * 5 * 4), (8192, 5 * 4)] and w == [(16384, 3 * 4)]


@pytest.mark.parametrize("op,fields,reads,writes", [
    ("axpy", {"x": 100, "y": 200, "n": 10, "a": 2.0}, [(100, 40), (200, 40)], [(200, 40)]),
    ("scale", {"x": 100, "y": 200, "n": 10, "a": 2.0}, [(100, 40)], [(200, 40)]),
    ("add", {"x": 1, "y": 2, "z": 3, "n": 4}, [(1, 16), (2, 16)], [(3, 16)]),
    ("bias_relu", {"t": 8, "b": 16, "n": 2}, [(8, 8), (16, 8)], [(8, 8)]),
    ("resid", {"h": 8, "u": 16, "b": 24, "n": 2}, [(8, 8), (16, 8), (24, 8)], [(8, 8)]),
    ("rl_broadphase", {"pos": 0, "prop": 1, "cont": 2, "nisl": 3, "nenv": 2},
     [(0, 2 * 32 * 12), (1, 2 * 32 * 8)], [(2, 2 * 1088), (3, 8)]),
    ("rl_solve", {"pos": 0, "prop": 1, "cont": 2, "vel": 3}, [(0, 384), (1, 256), (2, 1088), (3, 384)], [(3, 384)]),
    ("rl_integrate", {"pos": 0, "vel": 1, "prop": 2, "nenv": 1}, [(0, 384), (1, 384), (2, 256)], [(0, 384), (1, 384)]),
    ("sleep", {"y": 64, "ns": 5, "tag": 1.0}, [], [(64, 4)]),
])
def test_get_addresses_per_op(lib, op, fields, reads, writes):
    assert acs.acs_get_addresses(_args(op, fields)) == (reads, writes)


def test_get_addresses_rejects_unknown_op(lib):
    a = acs.acs_args()
    a.op = 77
    r = (acs.acs_segment * 16)()
    w = (acs.acs_segment * 16)()
    n1, n2 = C.c_uint32(), C.c_uint32()
    assert lib.acs_get_addresses(C.byref(a), r, C.byref(n1), w, C.byref(n2)) == acs.ACS_ERR_INVALID


def test_init_argument_checks_need_no_device(lib):
    h = C.c_void_p()
    assert lib.acs_init(C.byref(h), 0, None) == acs.ACS_ERR_INVALID
    assert lib.acs_init(C.byref(h), 65, None) == acs.ACS_ERR_INVALID
    cfg = acs.acs_config_default()
    cfg.n_streams = 257
    assert lib.acs_init(C.byref(h), 8, C.byref(cfg)) == acs.ACS_ERR_INVALID
    cfg = acs.acs_config_default()
    cfg.reserved[0] = 1
    assert lib.acs_init(C.byref(h), 8, C.byref(cfg)) == acs.ACS_ERR_INVALID


def test_init_without_a_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    assert lib.acs_init(C.byref(h), 8, None) == acs.ACS_ERR_DEVICE
    assert lib.acs_flush(None) == acs.ACS_ERR_INVALID
    lib.acs_destroy(None)
