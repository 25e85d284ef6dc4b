"""CPU checks of the request server's host-side core (arena allocator and
wave planner), compiled from its header with the host C++ compiler."""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1212_1095_gb300", "csrc")


def test_arena_and_wave_planner(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "sched_host_test")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I" + CSRC, os.path.join(HERE, "native", "sched_host_test.cpp"),
                    "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
