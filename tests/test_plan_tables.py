"""Host logic of the batch plan (no GPU): the stream-K unit split, the partial
slot tables, per-pair block / tile / row / cell ranges, replayed on the CPU
exactly as the kernels walk them (tests/host/plan_tables.cpp)."""
import os
import shutil
import subprocess

import pytest

from paper_2103_15039_gb300 import _build

HERE = os.path.dirname(os.path.abspath(__file__))


def test_plan_tables_cover_every_unit_slot_and_range(tmp_path):
    gxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if gxx is None or not os.path.isdir(cuda_inc):
        pytest.skip("g++ or the CUDA headers are not available")
    lib = _build.build()
    exe = str(tmp_path / "plan_tables")
    cmd = [gxx, "-O1", "-std=c++17", "-I", _build.INCLUDE, "-I", _build.CSRC, "-I", cuda_inc,
           os.path.join(HERE, "host", "plan_tables.cpp"), "-L", os.path.dirname(lib), "-llsgcpd",
           f"-Wl,-rpath,{os.path.dirname(lib)}", "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "0 failures" in r.stdout
