"""CPU checks of host-compiled internals.  The solve server's factor cache and HBM admission
(server_cache.h, host logic only): LRU eviction order, pinned entries kept, impossible
reservations refused without evicting, byte accounting.  The refinement's integer FP32-pair
split (pairsplit.h).  Each compiles a program under tests/cpp with the host compiler and runs
it."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("g++") is None, reason="no host C++ compiler")
def test_server_cache_logic(tmp_path):
    exe = str(tmp_path / "server_cache_check")
    src = os.path.join(ROOT, "tests", "cpp", "server_cache_check.cpp")
    inc = os.path.join(ROOT, "paper_2301_10762_gb300", "csrc")
    subprocess.run(["g++", "-std=c++17", "-O1", "-Wall", "-I", inc, src, "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr


@pytest.mark.skipif(shutil.which("g++") is None, reason="no host C++ compiler")
def test_integer_pair_split_equals_the_fp64_split(tmp_path):
    """The refinement's right-hand side is split into FP32 pairs by integer operations
    (pairsplit.h): bit for bit the FP64 definition hi = (float)v, lo = (float)(v - hi), on 2
    million values across the exponent range and at the rounding ties, and the widening back to
    FP64 equals (double)hi + (double)lo."""
    exe = str(tmp_path / "pairsplit_check")
    src = os.path.join(ROOT, "tests", "cpp", "pairsplit_check.cpp")
    inc = os.path.join(ROOT, "paper_2301_10762_gb300", "csrc")
    subprocess.run(["g++", "-std=c++17", "-O1", "-Wall", "-I", inc, src, "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
