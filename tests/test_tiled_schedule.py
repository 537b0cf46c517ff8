"""CPU check of the tiled fused form's item order and slot rings: the header
the kernel uses (csrc/tiled_schedule.h) is compiled with the host C++
compiler and every item of several queues (mixed 64x64 / 32x32, tiny grids,
single pairs, the mixed-resolution workload at full size) is decoded; the
program checks the decode is a bijection and that every wait is on an earlier
item (tests/tiled_schedule_check.cpp)."""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2303_05420_gb300", "csrc")


def test_tiled_schedule_order(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "tiled_schedule_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "tiled_schedule_check.cpp"), "-o",
                    exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip().endswith("ok")
