"""CPU checks of the setup worker pools (csrc/host_pool.cpp), compiled here
with g++ into a small harness (tests/host_pool_check.cpp): every member of a
team runs once and at the same time as the others (they meet at a barrier),
row ranges cover every row once, three concurrent callers each get a whole
team (two pools, then threads of their own), an exception of any member
reaches the caller after the others finish, and the pool keeps working after
it.  Run with 1, 4 and 16 as the thread cap (below 16 the 16-member teams
start threads of their own)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2503_21618_gb300", "csrc")


@pytest.fixture(scope="module")
def pool_check(tmp_path_factory):
    gxx = shutil.which(os.environ.get("CXX", "g++"))
    if gxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("pool") / "host_pool_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-I" + CSRC, os.path.join(ROOT, "tests", "host_pool_check.cpp"),
                    os.path.join(CSRC, "host_pool.cpp"), "-lpthread", "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("cap", ["1", "4", "16"])
def test_host_pool(pool_check, cap):
    env = dict(os.environ, SLRF_HOST_THREADS=cap)
    r = subprocess.run([pool_check], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "passed" in r.stdout
