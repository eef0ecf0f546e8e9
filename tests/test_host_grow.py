"""Buffer growth after a failed device allocation (host logic, no GPU).

Every capacity-tracked buffer set of the library grows through grow_set
(csrc/grow.h).  tests/grow_check.cpp drives it with a fake allocator that
fails on request and checks that a failed growth leaves the set empty
(capacity 0, null pointers, nothing leaked), so that the next call allocates
again instead of launching kernels on a stale capacity with null pointers.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_grow_set_recovers_from_failed_allocation(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "grow_check")
    subprocess.check_call([gxx, "-std=c++17", "-O1", "-Wall", "-o", exe, os.path.join(HERE, "grow_check.cpp")])
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "OK", out.stdout + out.stderr
