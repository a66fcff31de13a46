"""Host logic of the one-shot launch schedule: the work items of a launch
cover every (tile, level) exactly once, and the grouped list-scheduling
model matches an item-by-item simulation (tests/sched_check.cpp, compiled
against the library's internal header with the host compiler)."""
import os
import shutil
import subprocess

import pytest

from paper_2107_13500_gb300 import build

HERE = os.path.dirname(os.path.abspath(__file__))


def test_schedule_covers_every_tile_level_once(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(build.nvcc())), "include")
    exe = str(tmp_path / "sched_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", build.CSRC, "-I", build.INCLUDE, "-I", cuda_inc,
                    os.path.join(HERE, "sched_check.cpp"), "-o", exe], check=True, capture_output=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    cases, bad = (int(x) for x in out.stdout.split()[1::2])
    assert cases > 1000 and bad == 0
