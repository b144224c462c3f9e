"""The refinement's power-of-two conversions between its FP64 vectors and the FP32 inner vectors: the integer
bit manipulation of csrc/qp_convert.cuh (host path, compiled here with g++) against the FP64 expressions it stands
for, bit for bit, on random bit patterns, ties, rounding carries, zeros, subnormals, infinities and NaN."""
import pathlib
import shutil
import subprocess

import pytest

ROOT = pathlib.Path(__file__).resolve().parent.parent


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_power_of_two_conversions_are_the_fp64_expressions(tmp_path):
    exe = tmp_path / "convert_check"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", str(ROOT / "paper_2404_06841_gb300" / "csrc"),
                    str(ROOT / "tests" / "native" / "convert_check.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("ok "), out.stdout
