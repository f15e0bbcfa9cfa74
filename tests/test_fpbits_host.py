"""The FP64 <-> FP32 conversions done with integer operations on bit patterns
(csrc/fpbits.cuh, used by the grid conversion kernels) must give exactly the hardware
conversions' results: compiled as plain C++ and checked on about 2.5e7 values."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bit_conversions_match_the_hardware_conversions(tmp_path):
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("no g++")
    exe = tmp_path / "fpbits_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2404_15249_gb300", "csrc"),
                    "-o", str(exe), os.path.join(ROOT, "tests", "fpbits_check.cpp")], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert " 0 mismatches" in r.stdout
