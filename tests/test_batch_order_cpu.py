"""Run order of a batch (host logic of kgpu_submit and kgpu_submit_noalloc),
checked on the CPU through a small C++ harness built against the library's
own header (tests/order_check.cc).

The rule: requests run smallest first (fewest tiles; ties keep submission
order), except that every CBC-encryption request runs before the tail
reserve, the largest other requests holding the last `reserve` tiles.  The
checks are the properties that rule promises, on seeded random batches with
every mode, refused requests (no tiles) and reserves from none to all.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CBC_DEC, CBC_ENC = 1, 2


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    cuda_inc = next((p for p in ("/usr/local/cuda/include",) if os.path.exists(os.path.join(p, "cuda_runtime.h"))),
                    None)
    if not cxx or not cuda_inc:
        pytest.skip("g++ or the CUDA headers are not available")
    exe = str(tmp_path_factory.mktemp("order") / "order_check")
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I",
                    os.path.join(ROOT, "paper_1305_3345_gb300", "csrc"), "-I", cuda_inc,
                    os.path.join(HERE, "order_check.cc"), "-o", exe], check=True)
    return exe


def tiles_of(r):
    mode, nb, ub, tu, refused = r
    if refused:
        return 0
    units = nb // ub if mode in (CBC_DEC, CBC_ENC) else (nb + 31) // 32
    return (units + tu - 1) // tu


def run(exe, reserve, reqs):
    text = f"{reserve} {len(reqs)}\n" + "".join(" ".join(map(str, r)) + "\n" for r in reqs)
    out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout.split("\n")
    return [int(x) for x in out[0].split()], [int(x) for x in out[1].split()]


def draw(seed, n, big):
    """big: some requests of 1,024 tiles or more (the comparison sort);
    otherwise every count is small (the counting sort)."""
    rng = np.random.default_rng(seed)
    reqs = []
    for _ in range(n):
        mode = int(rng.choice([0, CBC_DEC, CBC_ENC, 3]))
        ub = 256
        nb = ub * int(rng.integers(1, 600 if big else 20))
        tu = 32 if mode == CBC_ENC else int(rng.choice([1, 2, 8, 64]))
        reqs.append((mode, nb, ub, tu, int(rng.integers(0, 20) == 0)))
    return reqs


@pytest.mark.parametrize("big", [False, True])
@pytest.mark.parametrize("seed", range(8))
def test_order_properties(harness, seed, big):
    reqs = draw(seed, 1 + seed * 53, big)
    assert (max(tiles_of(r) for r in reqs) >= 1024) == big or len(reqs) < 20
    t = [tiles_of(r) for r in reqs]
    enc = [r[0] == CBC_ENC for r in reqs]
    other_total = sum(x for x, e in zip(t, enc) if not e)
    for reserve in (0, 1, 7, other_total // 3, other_total, 10 ** 9):
        order, prefix = run(harness, reserve, reqs)
        assert sorted(order) == list(range(len(reqs)))
        assert prefix[0] == 0 and all(prefix[j + 1] - prefix[j] == t[order[j]] for j in range(len(reqs)))
        for kind in (True, False):   # each kind ascending by tiles, ties in submission order
            seq = [i for i in order if enc[i] == kind]
            assert seq == sorted(seq, key=lambda i: (t[i], i)), (reserve, kind)
        last_enc = max((j for j, i in enumerate(order) if enc[i]), default=-1)
        tail = sum(t[i] for i in order[last_enc + 1:])
        assert tail >= min(reserve, other_total), (reserve, tail)


@pytest.mark.parametrize("big", [False, True])
def test_order_extremes(harness, big):
    reqs = draw(99, 300, big)
    t = [tiles_of(r) for r in reqs]
    enc = [r[0] == CBC_ENC for r in reqs]
    order, _ = run(harness, 0, reqs)                 # no reserve: plain shortest first
    assert order == sorted(range(len(reqs)), key=lambda i: (t[i], i))
    order, _ = run(harness, 10 ** 12, reqs)          # everything reserved: all CBC encryption first
    assert order == sorted(range(len(reqs)), key=lambda i: (not enc[i], t[i], i))
