"""Serving loop admission (host logic): least estimated work first within a window of the 8
oldest requests, budget fit, oversize requests only on an idle device, the oldest admitted
after 8 passes, and the properties of the device-memory estimate.  Compiles
tests/admission_check.cpp with the system C++ compiler."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_admission_policy(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path / "admission_check")
    subprocess.run([cxx, "-std=c++17", "-O1", "-o", exe, os.path.join(HERE, "admission_check.cpp")], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout
