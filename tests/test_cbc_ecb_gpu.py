"""CBC (decrypt parallel per block, encrypt parallel per page) and ECB parity:
the CUDA path through the C ABI against the CPU oracle, bit-exact."""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
import workloads as w
from conftest import to_dev, to_np

pytestmark = pytest.mark.gpu


def run_cbc(ctx, key, enc, data, page, ivs, in_place=False):
    kh = ctx.setkey(key, False)
    try:
        src = to_dev(data)
        dst = src if in_place else src.new_empty(src.shape)
        iv = to_dev(np.ascontiguousarray(ivs).reshape(-1))
        if enc:
            ctx.cbc_encrypt_pages(kh, src, dst, page, iv)
        else:
            ctx.cbc_decrypt(kh, src, dst, page, iv)
        return to_np(dst)
    finally:
        ctx.delkey(kh)


def test_cbc_golden(ctx):
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_digests.json")))
    d = w.seeded_bytes(2, w.STREAM_DATA, 64 * 4096)
    ivs = w.page_ivs(2, 64)
    k = w.single_key(2, 128)
    assert hashlib.sha256(run_cbc(ctx, k, True, d, 4096, ivs).tobytes()).hexdigest() == gold["cbc128_enc"]
    assert hashlib.sha256(run_cbc(ctx, k, False, d, 4096, ivs).tobytes()).hexdigest() == gold["cbc128_dec"]


@pytest.mark.parametrize("bits", [128, 192, 256])
@pytest.mark.parametrize("page,npages", [(4096, 333), (512, 1025), (16, 700), (48, 517), (4112, 45)])
def test_cbc_vs_oracle(ctx, bits, page, npages):
    key = w.single_key(12, bits)
    data = w.seeded_bytes(12 + page, w.STREAM_DATA, page * npages)
    ivs = w.page_ivs(12 + page, npages)
    for enc in (True, False):
        ref = oracle.cbc(key, 0 if enc else 1, data, page, ivs)
        got = run_cbc(ctx, key, enc, data, page, ivs)
        assert np.array_equal(got, ref), (bits, page, npages, enc)


@pytest.mark.parametrize("page,npages", [
    (128, 1217 * 32 + 3),     # 1,218 groups of 32 pages: one wave of 9 warps per CTA, ragged last group
    (128, 8192 * 32 + 5),     # 8,193 groups: several waves, the warp count set by the tail, ragged last group
    (256, 100003),            # 3,126 groups, 16 blocks a page
])
def test_cbc_encrypt_launch_shapes(ctx, page, npages):
    """CBC encryption of many short pages: the staged kernel's warp count per
    CTA follows the number of 32-page groups (one wave, or waves sized to
    leave no small last wave), so these sizes cover each choice."""
    key = w.single_key(13, 128)
    data = w.seeded_bytes(13 + page, w.STREAM_DATA, page * npages)
    ivs = w.page_ivs(13 + page, npages)
    ref = oracle.cbc(key, 0, data, page, ivs)
    got = run_cbc(ctx, key, True, data, page, ivs)
    assert np.array_equal(got, ref), (page, npages)


@pytest.mark.parametrize("page", [128, 4096])
def test_cbc_encrypt_pages_at_16_byte_offsets(ctx, page):
    """Source and destination 16-byte aligned but not 128-byte aligned (the
    tensor-tile copies need 16), with enough 32-page groups for the tile
    kernel (12 per SM; 4-KiB pages: 240 MB) and a ragged last group; nothing
    is written outside the destination, and no bounded wait of the bulk
    kernels has run out in this process."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    key = w.single_key(14, 256)
    npages = 12 * sms * 32 + 7
    n = page * npages
    data = w.seeded_bytes(14 + page, w.STREAM_DATA, n)
    ivs = w.page_ivs(14 + page, npages)
    kh = ctx.setkey(key, False)
    try:
        sbuf = torch.zeros(n + 64, dtype=torch.uint8, device="cuda")
        dbuf = torch.zeros(n + 64, dtype=torch.uint8, device="cuda")
        src, dst = sbuf[16:16 + n], dbuf[48:48 + n]
        src.copy_(torch.from_numpy(data))
        iv = to_dev(np.ascontiguousarray(ivs).reshape(-1))
        ctx.cbc_encrypt_pages(kh, src, dst, page, iv)
        assert np.array_equal(to_np(dst), oracle.cbc(key, 0, data, page, ivs))
        assert not dbuf[:48].any() and not dbuf[48 + n:].any()   # nothing written outside
    finally:
        ctx.delkey(kh)
    assert ctx.bulk_wait_timeouts() == 0


def test_cbc_encrypt_in_place_in_tensor_tiles(ctx):
    """In-place CBC encryption with enough 32-page groups for the tensor-tile
    kernel (each chunk is stored back over itself before the next one is
    loaded), ragged last group."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    key = w.single_key(15, 128)
    npages = 12 * sms * 32 + 19
    data = w.seeded_bytes(15, w.STREAM_DATA, 128 * npages)
    ivs = w.page_ivs(15, npages)
    c = run_cbc(ctx, key, True, data, 128, ivs, in_place=True)
    assert np.array_equal(c, oracle.cbc(key, 0, data, 128, ivs))


def test_cbc_in_place(ctx):
    key = w.single_key(13, 128)
    data = w.seeded_bytes(13, w.STREAM_DATA, 4096 * 500)
    ivs = w.page_ivs(13, 500)
    c = run_cbc(ctx, key, True, data, 4096, ivs, in_place=True)
    assert np.array_equal(c, oracle.cbc(key, 0, data, 4096, ivs))
    p = run_cbc(ctx, key, False, c, 4096, ivs, in_place=True)
    assert np.array_equal(p, data)


def test_cbc_argument_errors(ctx):
    import torch
    import paper_1305_3345_gb300 as kg
    key = w.single_key(14, 128)
    kh = ctx.setkey(key, False)
    xk = ctx.setkey(w.xts_key(14, 128), True)
    buf = torch.zeros(3 * 4096, dtype=torch.uint8, device="cuda")
    ivs = torch.zeros(3 * 16, dtype=torch.uint8, device="cuda")
    L, h, s = kg.lib(), ctx.handle, torch.cuda.current_stream().cuda_stream
    p, ip = buf.data_ptr(), ivs.data_ptr()
    for fn in (L.kgpu_aes_cbc_decrypt, L.kgpu_aes_cbc_encrypt_pages):
        assert fn(h, kh, p, p, 3 * 4096, 4096, ip, s) == 0
        assert fn(h, kh, p, p, 3 * 4096, 4000, ip, s) == -22        # page % 16
        assert fn(h, kh, p, p, 2 * 4096 + 16, 4096, ip, s) == -22   # not whole pages
        assert fn(h, xk, p, p, 4096, 4096, ip, s) == -2             # XTS key
        assert fn(h, kh, p, p, 4096, 4096, ip + 8, s) == -22        # misaligned IVs
        assert fn(h, kh, p, p, 4096, 4096, 0, s) == -14             # no IVs
        assert fn(h, kh, p, p, 1 << 40, 4096, ip, s) == -14         # past the allocation
        assert fn(h, kh, ip, ip, 16, 16, ip, s) == -22              # IVs overwritten by output
    torch.cuda.synchronize()
    ctx.delkey(kh)
    ctx.delkey(xk)


def test_cbc_full_size_sampled(ctx):
    """1 GiB as 262,144 x 4096-B pages, AES-128, per-page IVs: sampled pages
    against the oracle; decrypt(encrypt(x)) == x over the whole buffer."""
    import torch
    key = w.single_key(2, 128)
    n = 1 << 30
    npages = n // 4096
    data = torch.from_numpy(w.seeded_bytes(2, w.STREAM_DATA, n)).cuda()
    ivs_np = w.page_ivs(2, npages)
    ivs = torch.from_numpy(ivs_np.reshape(-1).copy()).cuda()
    kh = ctx.setkey(key, False)
    enc = torch.empty_like(data)
    ctx.cbc_encrypt_pages(kh, data, enc, 4096, ivs)
    rng = np.random.default_rng(2)
    sample = np.unique(np.concatenate([[0, npages - 1], rng.integers(0, npages, 46)]))
    for pg in sample:
        pg = int(pg)
        src = data[pg * 4096:(pg + 1) * 4096].cpu().numpy()
        assert np.array_equal(enc[pg * 4096:(pg + 1) * 4096].cpu().numpy(),
                              oracle.cbc(key, 0, src, 4096, ivs_np[pg:pg + 1])), pg
    dec = torch.empty_like(data)
    ctx.cbc_decrypt(kh, enc, dec, 4096, ivs)
    for pg in sample[:16]:
        pg = int(pg)
        c = enc[pg * 4096:(pg + 1) * 4096].cpu().numpy()
        assert np.array_equal(dec[pg * 4096:(pg + 1) * 4096].cpu().numpy(),
                              oracle.cbc(key, 1, c, 4096, ivs_np[pg:pg + 1])), pg
    assert torch.equal(dec, data)
    ctx.delkey(kh)
    del data, enc, dec
    torch.cuda.empty_cache()


@pytest.mark.parametrize("bits", [128, 256])
@pytest.mark.parametrize("nblocks", [1, 31, 32, 33, 4097, 100003])
def test_ecb_vs_oracle(ctx, bits, nblocks):
    key = w.single_key(15, bits)
    data = w.seeded_bytes(15, w.STREAM_DATA, 16 * nblocks)
    kh = ctx.setkey(key, False)
    for dir in (0, 1):
        src = to_dev(data)
        dst = src.new_empty(src.shape)
        ctx.ecb_crypt(kh, dir, src, dst)
        assert np.array_equal(to_np(dst), oracle.ecb(key, dir, data)), (bits, nblocks, dir)
    ctx.delkey(kh)
