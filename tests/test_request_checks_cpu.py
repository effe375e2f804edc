"""Validation of batched and served requests (the host side of kgpu_submit,
kgpu_submit_noalloc and kgpu_serve_submit), checked on the CPU through a small
C++ harness built against the library's own header (tests/desc_check.cc).

Every refusal listed here is what keeps a malformed request from reaching a
kernel: nothing is launched for a request whose validation fails.  The harness
fakes the context: key handles 1 (XTS, live), 2 (single key, live) and 3 (XTS,
deleted); device allocations D1 and D2 of 1 MiB; one registered host range H of
1 MiB that the device sees at H + 0x1000000000.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

OK, ENOENT, EFAULT, EINVAL = 0, -2, -14, -22
XTS, CBC_DEC, CBC_ENC, ECB, COPY = 0, 1, 2, 3, 4
SRC_HOST, DST_HOST, IVS_HOST = 1, 2, 4
D1, D2, H = 0x10000000, 0x20000000, 0x70000000
MIB = 1 << 20
H_DEV = 0x1000000000
FIELDS = ("rc", "src", "dst", "ivs", "nblocks", "first_sector", "unit_blocks", "key", "mode", "dir", "flags",
          "tile_units")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if not cxx or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers are not available")
    exe = str(tmp_path_factory.mktemp("desc") / "desc_check")
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I",
                    os.path.join(ROOT, "paper_1305_3345_gb300", "csrc"), "-I", cuda_inc,
                    os.path.join(HERE, "desc_check.cc"), "-o", exe], check=True)
    return exe


def req(mode=XTS, dir=0, key=1, flags=0, src=D1, dst=D1 + 0x10000, len=4096, unit=4096, sector=0, ivs=0):
    return (mode, dir, key, flags, src, dst, len, unit, sector, ivs)


def run(exe, reqs, tile_chunks=32):
    text = f"{tile_chunks}\n" + "".join(
        f"{m} {d} {k} {f} {s:x} {t:x} {n} {u} {sec} {iv:x}\n" for m, d, k, f, s, t, n, u, sec, iv in reqs)
    out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout.split("\n")
    rows = []
    for line in out[:len(reqs)]:
        v = line.split()
        rows.append(dict(zip(FIELDS, [int(v[0])] + [int(x, 16) for x in v[1:4]] + [int(x) for x in v[4:]])))
    return rows


def test_valid_requests_give_their_descriptors(harness):
    cases = [
        req(sector=7),                                                        # XTS encryption
        req(dir=1, src=D1, dst=D1, len=8192, unit=512, sector=2**64 - 16),     # XTS decryption in place
        req(mode=CBC_DEC, key=2, dst=D2, len=8192, ivs=D2 + 0x10000),          # CBC decryption
        req(mode=CBC_ENC, key=2, dst=D2, len=8192, ivs=D2 + 0x10000),          # CBC encryption
        req(mode=ECB, dir=1, key=2, unit=0),                                    # ECB ignores unit_size
        req(mode=COPY, key=0, unit=256),                                        # the empty service: no key
        req(src=0, dst=0, len=0),                                               # an empty request
        req(flags=SRC_HOST, src=H + 0x100),                                     # host source
        req(flags=SRC_HOST | DST_HOST, src=H, dst=H),                           # host pages in place
        req(mode=CBC_DEC, key=2, flags=IVS_HOST, ivs=H + 0x200),                # host IVs
        req(mode=CBC_DEC, key=2, len=65536, unit=65536, ivs=D2),                # a page larger than a tile
    ]
    r = run(harness, cases)
    assert [x["rc"] for x in r] == [OK] * len(cases)
    x = r[0]
    assert (x["src"], x["dst"], x["ivs"]) == (D1, D1 + 0x10000, 0)
    assert (x["nblocks"], x["first_sector"], x["unit_blocks"]) == (256, 7, 256)
    assert (x["key"], x["mode"], x["dir"], x["flags"], x["tile_units"]) == (0, XTS, 0, 0, 32)
    assert (r[1]["src"], r[1]["dst"], r[1]["dir"], r[1]["unit_blocks"]) == (D1, D1, 1, 32)
    assert r[1]["first_sector"] == 2**64 - 16
    # CBC: the key is table slot 1; decryption runs the inverse direction;
    # decryption tiles hold tile_chunks x 32 blocks in whole pages, encryption
    # tiles 32 pages
    assert (r[2]["key"], r[2]["dir"], r[2]["ivs"], r[2]["tile_units"]) == (1, 1, D2 + 0x10000, 4)
    assert (r[3]["dir"], r[3]["tile_units"]) == (0, 32)
    assert (r[4]["unit_blocks"], r[4]["nblocks"], r[4]["dir"]) == (1, 256, 1)
    assert (r[5]["key"], r[5]["dir"], r[5]["tile_units"], r[5]["unit_blocks"]) == (0, 0, 1, 16)
    assert (r[6]["nblocks"], r[6]["src"]) == (0, 0)
    assert (r[7]["src"], r[7]["dst"], r[7]["flags"]) == (H + 0x100 + H_DEV, D1 + 0x10000, 1)
    assert (r[8]["src"], r[8]["dst"], r[8]["flags"]) == (H + H_DEV, H + H_DEV, 3)
    assert r[9]["ivs"] == H + 0x200 + H_DEV and r[9]["flags"] == 0  # host IVs are not a page flag
    assert r[10]["tile_units"] == 1
    # the tile size follows tile_chunks
    r = run(harness, [cases[0], cases[2], cases[3]], tile_chunks=128)
    assert [x["tile_units"] for x in r] == [128, 16, 32]


@pytest.mark.parametrize("case,rc", [
    (req(flags=8), EINVAL),                                   # unknown flag bit
    (req(mode=5), EINVAL),                                    # unknown mode
    (req(dir=2), EINVAL),                                     # XTS direction
    (req(mode=ECB, key=2, dir=2), EINVAL),                    # ECB direction
    (req(unit=0), EINVAL),                                    # no unit size
    (req(unit=100, len=400), EINVAL),                         # unit not a multiple of 16
    (req(len=4100), EINVAL),                                  # length not a multiple of the unit
    (req(len=0, unit=16 << 32), EINVAL),                      # unit of 2^32 blocks or more
    (req(len=8192, sector=2**64 - 1), EINVAL),                # 64-bit unit numbers would wrap
    (req(key=0), ENOENT),                                     # no key handle
    (req(key=4), ENOENT),                                     # beyond the table
    (req(key=3), ENOENT),                                     # deleted key
    (req(key=2), ENOENT),                                     # XTS with a single key
    (req(mode=CBC_DEC, key=1, ivs=D2), ENOENT),               # CBC with an XTS key
    (req(src=D1 + 8), EINVAL),                                # source not 16-byte aligned
    (req(dst=D1 + 0x10008), EINVAL),                          # destination not 16-byte aligned
    (req(dst=D1 + 0x800), EINVAL),                            # partial overlap
    (req(src=0x30000000), EFAULT),                            # source in no allocation
    (req(src=D1 + MIB - 4096, len=8192), EFAULT),             # source past its allocation's end
    (req(dst=0), EFAULT),                                     # no destination
    (req(mode=CBC_DEC, key=2, ivs=D2 + 8), EINVAL),           # IVs not 16-byte aligned
    (req(mode=CBC_DEC, key=2, ivs=0), EFAULT),                # no IVs
    (req(mode=CBC_DEC, key=2, ivs=0x30000000), EFAULT),       # IVs in no allocation
    (req(mode=CBC_ENC, key=2, dst=D2, len=65536, ivs=D2 + MIB - 16 * 15), EFAULT),  # 16 IVs, past the end
    (req(mode=CBC_ENC, key=2, dst=D2, ivs=D2 + 0x10), EINVAL),             # IVs inside the output
    (req(flags=SRC_HOST, src=D1), EFAULT),                    # host flag on an unregistered pointer
    (req(flags=SRC_HOST, src=H + MIB - 4096, len=8192), EFAULT),  # past the registered range
    (req(src=H), EFAULT),                                     # host pointer without the flag
    (req(mode=CBC_DEC, key=2, flags=IVS_HOST, ivs=D2), EFAULT),   # host IV flag on a device pointer
])
def test_refusals(harness, case, rc):
    assert run(harness, [case])[0]["rc"] == rc


def test_refusals_do_not_depend_on_order(harness):
    """A refused request leaves the next one's validation unchanged (the range
    cache is per call, and a refusal records nothing)."""
    good, bad = req(sector=3), req(src=0x30000000)
    r = run(harness, [bad, good, bad, good])
    assert [x["rc"] for x in r] == [EFAULT, OK, EFAULT, OK]
    assert r[1] == r[3]
