"""Whole-buffer parity at the bulk workload's full size.

The two page-granular encryption kernels whose output a symmetric bug could
hide from a round trip (XTS encryption with the closed-form tweak, and CBC
encryption run one chain per page) are compared byte for byte with the oracle
over the whole 1 GiB buffer, in the launch configuration the bench times:

- AES-256-XTS encryption, 262,144 data units of 4096 B numbered 0..262143
  (IEEE 1619 5.3.1), seed 2;
- AES-128-CBC encryption of 262,144 pages of 4096 B with per-page IVs
  (SP 800-38A 6.2), seed 2.

The other variants of that workload are compared whole as well: AES-256-XTS
decryption, the 512-byte-unit variant (2,097,152 units, AES-128) and AES-128-CBC
decryption (SP 800-38A 6.2), each on the 1 GiB buffer the bench uses.

The oracle runs on every host core (about 10-15 s per GiB on 16 cores).
"""
import numpy as np
import pytest

import oracle
import workloads as w

pytestmark = pytest.mark.gpu

GIB = 1 << 30
PAGE = 4096


def _first_bad_unit(got: np.ndarray, ref: np.ndarray, unit: int):
    bad = np.flatnonzero((got.reshape(-1, unit) != ref.reshape(-1, unit)).any(axis=1))
    return None if bad.size == 0 else (int(bad[0]), int(bad.size))


def test_xts256_encrypt_1gib_whole_buffer(ctx):
    import torch
    key = w.xts_key(2, 256)
    data = w.seeded_bytes(2, w.STREAM_DATA, GIB)
    src = torch.from_numpy(data).cuda()
    dst = torch.empty_like(src)
    kh = ctx.setkey(key, True)
    try:
        ctx.xts_crypt(kh, 0, src, dst, PAGE, 0)
        got = dst.cpu().numpy()
    finally:
        ctx.delkey(kh)
    del src, dst
    torch.cuda.empty_cache()
    ref = oracle.xts(key, 0, data, PAGE, 0)
    assert _first_bad_unit(got, ref, PAGE) is None, "first mismatching sector, count"


def test_cbc128_encrypt_pages_1gib_whole_buffer(ctx):
    import torch
    key = w.single_key(2, 128)
    npages = GIB // PAGE
    data = w.seeded_bytes(2, w.STREAM_DATA, GIB)
    ivs = w.page_ivs(2, npages)
    src = torch.from_numpy(data).cuda()
    iv_d = torch.from_numpy(ivs.reshape(-1).copy()).cuda()
    dst = torch.empty_like(src)
    kh = ctx.setkey(key, False)
    try:
        ctx.cbc_encrypt_pages(kh, src, dst, PAGE, iv_d)
        got = dst.cpu().numpy()
    finally:
        ctx.delkey(kh)
    del src, dst, iv_d
    torch.cuda.empty_cache()
    ref = oracle.cbc(key, 0, data, PAGE, ivs)
    assert _first_bad_unit(got, ref, PAGE) is None, "first mismatching page, count"


def test_xts256_decrypt_1gib_whole_buffer(ctx):
    import torch
    key = w.xts_key(2, 256)
    data = w.seeded_bytes(2, w.STREAM_DATA, GIB)   # taken as ciphertext
    src = torch.from_numpy(data).cuda()
    dst = torch.empty_like(src)
    kh = ctx.setkey(key, True)
    try:
        ctx.xts_crypt(kh, 1, src, dst, PAGE, 0)
        got = dst.cpu().numpy()
    finally:
        ctx.delkey(kh)
    del src, dst
    torch.cuda.empty_cache()
    ref = oracle.xts(key, 1, data, PAGE, 0)
    assert _first_bad_unit(got, ref, PAGE) is None, "first mismatching sector, count"


def test_xts128_encrypt_512b_units_1gib_whole_buffer(ctx):
    import torch
    key = w.xts_key(2, 128)
    data = w.seeded_bytes(2, w.STREAM_DATA, GIB)
    src = torch.from_numpy(data).cuda()
    dst = torch.empty_like(src)
    kh = ctx.setkey(key, True)
    try:
        ctx.xts_crypt(kh, 0, src, dst, 512, 0)
        got = dst.cpu().numpy()
    finally:
        ctx.delkey(kh)
    del src, dst
    torch.cuda.empty_cache()
    ref = oracle.xts(key, 0, data, 512, 0)
    assert _first_bad_unit(got, ref, 512) is None, "first mismatching unit, count"


def test_cbc128_decrypt_1gib_whole_buffer(ctx):
    import torch
    key = w.single_key(2, 128)
    npages = GIB // PAGE
    data = w.seeded_bytes(2, w.STREAM_DATA, GIB)   # taken as ciphertext
    ivs = w.page_ivs(2, npages)
    src = torch.from_numpy(data).cuda()
    iv_d = torch.from_numpy(ivs.reshape(-1).copy()).cuda()
    dst = torch.empty_like(src)
    kh = ctx.setkey(key, False)
    try:
        ctx.cbc_decrypt(kh, src, dst, PAGE, iv_d)
        got = dst.cpu().numpy()
    finally:
        ctx.delkey(kh)
    del src, dst, iv_d
    torch.cuda.empty_cache()
    ref = oracle.cbc(key, 1, data, PAGE, ivs)
    assert _first_bad_unit(got, ref, PAGE) is None, "first mismatching page, count"
