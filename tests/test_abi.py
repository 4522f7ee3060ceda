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


def test_lookahead_checks_need_no_device(lib):
    h = C.c_void_p()
    cfg = acs.acs_config_default()
    assert cfg.lookahead == acs.LOOKAHEAD_AUTO          # dispatch ahead by default
    for window, ahead, span, mode in [(32, 33, 0, 0),   # window + lookahead above 64
                                      (64, 1, 0, 0),
                                      (8, 4, 16, 0),    # not with a free-slot span
                                      (8, 4, 0, 1)]:    # window mode only
        cfg = acs.acs_config_default()
        cfg.lookahead, cfg.span, cfg.mode = ahead, span, mode
        assert lib.acs_init(C.byref(h), window, C.byref(cfg)) == acs.ACS_ERR_INVALID, (window, ahead, span, mode)


def test_init_without_a_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    assert lib.acs_init(C.byref(h), 8, None) == acs.ACS_ERR_DEVICE
    assert lib.acs_flush(None) == acs.ACS_ERR_INVALID
    assert lib.acs_abort(None) == acs.ACS_ERR_INVALID
    lib.acs_destroy(None)


def _noalloc_rows(specs):
    """Packed rows for acs_run_noalloc: (op, ncta, fields) per task."""
    import numpy as np
    from paper_2401_12377_b300.harness import _args_row
    return np.concatenate([_args_row(op, ncta, f) for op, ncta, f in specs])


_AXPY = {"x": 4096, "y": 8192, "n": 16, "a": 2.0}
_EMIT = {"cfg": 4096, "nisl": 8192, "token": 12288, "ncta_table": 16384, "n_env": 8, "step": 0, "steps": 2,
         "chunk": 4}


@pytest.mark.parametrize("case,expect", [
    ("ids_equal", acs.ACS_ERR_ORDER),
    ("ids_decrease", acs.ACS_ERR_ORDER),
    ("unknown_op", acs.ACS_ERR_INVALID),
    ("ncta_0", acs.ACS_ERR_INVALID),
    ("ncta_257", acs.ACS_ERR_INVALID),
    ("reserved", acs.ACS_ERR_INVALID),
    ("emit_task", acs.ACS_ERR_INVALID),
    ("segment_overflow", acs.ACS_ERR_INVALID),
])
def test_noalloc_refuses_bad_tasks_on_the_host(lib, case, expect):
    """acs_run_noalloc checks every task before it touches the device, so each
    refusal below comes back on a machine without a GPU as on one with a GPU."""
    import numpy as np
    ids = np.array([1, 2, 3], np.uint32)
    specs = [("axpy", 1, _AXPY)] * 3
    if case == "ids_equal":
        ids = np.array([1, 2, 2], np.uint32)
    elif case == "ids_decrease":
        ids = np.array([5, 4, 6], np.uint32)
    elif case == "ncta_0":
        specs = [("axpy", 1, _AXPY), ("axpy", 0, _AXPY), ("axpy", 1, _AXPY)]
    elif case == "ncta_257":
        specs = [("axpy", 1, _AXPY), ("axpy", 1, _AXPY), ("axpy", 257 % 65536, _AXPY)]
    elif case == "emit_task":
        specs = [("axpy", 1, _AXPY), ("rl_emit", 1, _EMIT), ("axpy", 1, _AXPY)]
    elif case == "segment_overflow":   # a range whose end passes 2^64
        specs = [("axpy", 1, _AXPY), ("axpy", 1, {"x": 2**64 - 8, "y": 8192, "n": 16, "a": 1.0}),
                 ("axpy", 1, _AXPY)]
    packed = _noalloc_rows(specs)
    if case == "unknown_op":
        packed["op"][1] = 77
    if case == "reserved":
        packed["reserved"][2] = 1
    assert acs.acs_run_noalloc(8, ids, packed) == expect


def test_noalloc_refuses_bad_window_and_size_on_the_host(lib):
    import numpy as np
    packed = _noalloc_rows([("axpy", 1, _AXPY)])
    ids = np.array([1], np.uint32)
    assert acs.acs_run_noalloc(0, ids, packed) == acs.ACS_ERR_INVALID
    assert acs.acs_run_noalloc(65, ids, packed) == acs.ACS_ERR_INVALID
    n = acs.ACS_NOALLOC_MAX_TASKS + 1
    big = np.repeat(packed, n)
    assert acs.acs_run_noalloc(8, np.arange(n, dtype=np.uint32), big) == acs.ACS_ERR_INVALID
    assert acs.acs_run_noalloc(8, ids[:0], packed[:0]) == acs.ACS_OK    # nothing to run


def test_noalloc_valid_tasks_without_a_gpu_fail_cleanly(lib):
    import numpy as np
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    packed = _noalloc_rows([("axpy", 1, _AXPY)] * 2)
    assert acs.acs_run_noalloc(8, np.array([1, 2], np.uint32), packed) == acs.ACS_ERR_DEVICE


def test_stream_rebase_checks_need_no_device(lib):
    """acs_stream_rebase refuses a missing context; the position-limit error has
    its own code and message, and the binding's limit is the header's."""
    assert lib.acs_stream_rebase(None, 0, 0) == acs.ACS_ERR_INVALID
    hdr = open(os.path.join(ROOT, "include", "acs.h")).read()
    assert re.search(r"#define ACS_ERR_RANGE\s+\(-8\)", hdr) and acs.ACS_ERR_RANGE == -8
    assert re.search(r"#define ACS_MAX_POSITION 0x80000000u", hdr) and acs.ACS_MAX_POSITION == 1 << 31
    assert b"2^31" in lib.acs_strerror(acs.ACS_ERR_RANGE)


def test_header_compiles_as_c99(tmp_path):
    """include/acs.h is a C header: it compiles on its own as C99 with every
    warning enabled (no C++-only constructs, no missing includes)."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    src = tmp_path / "use_acs.c"
    src.write_text('#include "acs.h"\n'
                   'int main(void) { acs_config cfg; acs_config_default(&cfg);\n'
                   '  return (int)cfg.lookahead == 0 ? ACS_ERR_RANGE : (int)(ACS_MAX_POSITION >> 31); }\n')
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-I", os.path.join(ROOT, "include"), "-c", str(src), "-o", str(tmp_path / "use_acs.o")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
