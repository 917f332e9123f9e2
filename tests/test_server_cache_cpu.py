"""CPU checks of the solve server's factor cache and HBM admission (server_cache.h, host
logic only): LRU eviction order, pinned entries kept, impossible reservations refused
without evicting, byte accounting.  Compiles tests/cpp/server_cache_check.cpp with the host
compiler and runs it."""
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
