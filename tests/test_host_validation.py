"""Host-side test of the ghost-position validation in the level and adjoint
kernels: the shared helpers (ghost_slot_of, the source probe) are compiled by
nvcc as host code and run on the CPU with ghost tags planted in the tag buffer
that the plan does not hold.  No GPU is used: such a buffer is never given to
the GPU kernels in the tests."""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_foreign_ghost_tags_are_skipped(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "probe_validation")
    src = os.path.join(HERE, "host", "probe_validation.cu")
    subprocess.run([nvcc, "-std=c++17", "-O1", "--expt-relaxed-constexpr", "-o", exe, src], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("ok")
