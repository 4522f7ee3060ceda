"""The solve body's reciprocal and division helpers (rcp_rn, div_from_rcp in
csrc/acs_bodies.cuh) against CUDA's IEEE reciprocal and quotient: a small
test program (tests/cuda/div_check.cu) includes the body header and compares
them bit for bit on the GPU; on the CPU it is only compiled."""
import json
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "cuda", "div_check.cu")


def _build(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "div_check")
    cmd = [nvcc, "-O3", "-std=c++17", "-fmad=false", "-gencode", "arch=compute_103a,code=sm_103a",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_2401_12377_b300", "csrc"),
           SRC, "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return exe


def test_div_check_program_builds(tmp_path):
    assert os.path.exists(_build(tmp_path))


@pytest.mark.gpu
def test_rcp_and_division_equal_ieee(tmp_path):
    exe = _build(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["cuda"] == "no error"
    assert out["rcp_values"] == (1 << 23) * 201 and out["rcp_mismatches"] == 0
    assert out["div_mismatches_solve"] == 0 and out["div_mismatches_normal"] == 0
    assert r.returncode == 0
