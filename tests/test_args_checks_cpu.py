"""Argument checks of the per-call XTS entry points and the lookup of
registered host ranges (the guard on every host pointer a kernel is given),
checked on the CPU through a small C++ harness built against the library's
own header (tests/args_check.cc).  The harness registers [0x1000, 0x2000),
[0x2000, 0x3000) (adjacent), [0x5000, 0x9000) and [0x10000, 0x11000), seen by
the device at +0x100000, +0x200000, +0x300000 and +0."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
OK, EFAULT, EINVAL = 0, -14, -22


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if not cxx or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers are not available")
    exe = str(tmp_path_factory.mktemp("args") / "args_check")
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I",
                    os.path.join(ROOT, "paper_1305_3345_gb300", "csrc"), "-I", cuda_inc,
                    os.path.join(HERE, "args_check.cc"), "-o", exe], check=True)
    return exe


def run(exe, lines):
    out = subprocess.run([exe], input="".join(l + "\n" for l in lines), capture_output=True, text=True,
                         check=True).stdout.split("\n")
    return out[:len(lines)]


def xts(exe, dir=0, len=8192, du=4096, sector=0, stealing=0):
    return int(run(exe, [f"x {dir} {len} {du} {sector} {stealing}"])[0])


def host(exe, p, n):
    rc, dev = run(exe, [f"h {p:x} {n}"])[0].split()
    return int(rc), int(dev, 16)


def test_xts_arguments(harness):
    assert xts(harness) == OK
    assert xts(harness, dir=1, du=512) == OK
    assert xts(harness, len=0) == OK                         # nothing to do
    assert xts(harness, dir=2) == EINVAL                     # direction
    assert xts(harness, du=0, len=0) == EINVAL               # no data unit
    assert xts(harness, du=8, len=16) == EINVAL              # units below one block
    assert xts(harness, len=4100) == EINVAL                  # length not a multiple of the unit
    assert xts(harness, du=100, len=400) == EINVAL           # partial blocks only with stealing
    assert xts(harness, du=100, len=400, stealing=1) == OK
    assert xts(harness, du=17, len=34, stealing=1) == OK     # the shortest unit that steals
    assert xts(harness, du=16 << 32, len=0) == EINVAL        # 2^32 blocks per unit
    assert xts(harness, du=(16 << 32) - 16, len=0) == OK
    # the 64-bit unit numbers of the request must not wrap
    assert xts(harness, sector=2**64 - 2) == OK               # units 2^64-2 and 2^64-1
    assert xts(harness, sector=2**64 - 1) == EINVAL
    assert xts(harness, sector=2**64 - 1, len=4096) == OK
    assert xts(harness, sector=2**64 - 1, len=0) == OK


def test_host_ranges(harness):
    assert host(harness, 0x1000, 0x1000) == (OK, 0x101000)             # a whole range
    assert host(harness, 0x1ff0, 16) == (OK, 0x101ff0)                 # its last block
    assert host(harness, 0x2000, 16) == (OK, 0x202000)                 # the adjacent range's first
    assert host(harness, 0x8000, 0x1000) == (OK, 0x308000)             # ends exactly at the range's end
    assert host(harness, 0x10800, 16) == (OK, 0x10800)                 # mapped at the same address
    assert host(harness, 0x1ff0, 32)[0] == EFAULT                      # spans two ranges, even adjacent ones
    assert host(harness, 0x8000, 0x1001)[0] == EFAULT                  # one byte past the end
    assert host(harness, 0x3000, 16)[0] == EFAULT                      # the gap after a range
    assert host(harness, 0x4ff0, 32)[0] == EFAULT                      # runs from the gap into a range
    assert host(harness, 0x800, 16)[0] == EFAULT                       # before the first range
    assert host(harness, 0x20000, 16)[0] == EFAULT                     # after the last
    assert host(harness, 0, 16)[0] == EFAULT                           # null
    assert host(harness, 0x5000, 2**64 - 0x1000)[0] == EFAULT          # a length that wraps
