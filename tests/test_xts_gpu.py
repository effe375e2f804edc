"""XTS parity: the CUDA path (through the C ABI) against the CPU oracle, bit-exact.

Sizes span many warps' ranges and ragged tails; data-unit sizes cover the
closed-form tweak paths (du a multiple of 512 B, du < 512 B so several units
share a warp step, and du not a multiple of 512 B so units straddle steps).
"""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
import workloads as w
from conftest import to_dev, to_np

pytestmark = pytest.mark.gpu

ENC, DEC = 0, 1


def run_xts(ctx, key_bytes, dir, data, du, first):
    kh = ctx.setkey(key_bytes, True)
    try:
        src = to_dev(data)
        dst = src.new_empty(src.shape)
        ctx.xts_crypt(kh, dir, src, dst, du, first)
        return to_np(dst)
    finally:
        ctx.delkey(kh)


def test_config1_aes256_xts_1mib(ctx):
    """256 sectors x 4096 B, sectors 0..255: encrypt then decrypt, bit-exact."""
    key = w.xts_key(1, 256)
    data = w.seeded_bytes(1, w.STREAM_DATA, 1 << 20)
    ref = oracle.xts(key, ENC, data, 4096, 0)
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_digests.json")))
    c = run_xts(ctx, key, ENC, data, 4096, 0)
    assert np.array_equal(c, ref)
    assert hashlib.sha256(c.tobytes()).hexdigest() == gold["xts256_1mib"]
    p = run_xts(ctx, key, DEC, c, 4096, 0)
    assert np.array_equal(p, data)


@pytest.mark.parametrize("bits", [128, 256])
@pytest.mark.parametrize("du,units,first", [
    (4096, 301, 0),            # several warps, ragged split
    (512, 2049, 2**40 + 17),   # many units per warp batch, large sector numbers
    (16, 1537, 5),             # one block per unit: 32 units per warp step
    (48, 999, 2**63),          # 3 blocks per unit, units straddle warp steps
    (4112, 67, 1),             # 257 blocks per unit, not a multiple of 32
    (65536, 9, 100),           # 4096 blocks per unit (long closed-form start)
])
def test_xts_vs_oracle(ctx, bits, du, units, first):
    key = w.xts_key(3, bits)
    data = w.seeded_bytes(3 + du, w.STREAM_DATA, du * units)
    for dir in (ENC, DEC):
        ref = oracle.xts(key, dir, data, du, first)
        got = run_xts(ctx, key, dir, data, du, first)
        assert np.array_equal(got, ref), (bits, du, units, dir)


@pytest.mark.parametrize("bits", [128, 256])
@pytest.mark.parametrize("du,units,first", [
    (17, 301, 0),              # one full block + 1 byte: the stealing pair is the whole unit
    (31, 100, 5),              # 15-byte tail
    (100, 1000, 2**40 + 3),    # 4-byte aligned unit starts, more units than a CTA has warps
    (527, 257, 2**63 - 300),   # odd unit starts (byte accesses)
    (4100, 67, 11),            # 256 full blocks + 4 bytes
    (4097, 33, 1),             # 256 full blocks + 1 byte, byte-aligned starts
])
def test_xts_ciphertext_stealing_vs_oracle(ctx, bits, du, units, first):
    """Data units that are not a multiple of 16 bytes end with ciphertext
    stealing (IEEE 1619 5.3.2 / 5.4.2), bit-exact with the oracle both ways
    and in place."""
    import torch
    key = w.xts_key(8, bits)
    data = w.seeded_bytes(8 + du, w.STREAM_DATA, du * units)
    for dir in (ENC, DEC):
        ref = oracle.xts(key, dir, data, du, first)
        assert np.array_equal(run_xts(ctx, key, dir, data, du, first), ref), (bits, du, dir)
    kh = ctx.setkey(key, True)
    buf = to_dev(data)
    ctx.xts_crypt(kh, ENC, buf, buf, du, first)
    torch.cuda.synchronize()
    assert np.array_equal(to_np(buf), oracle.xts(key, ENC, data, du, first))
    ctx.delkey(kh)


def test_xts_tiny_and_single_unit(ctx):
    key = w.xts_key(4, 256)
    for du, units in ((16, 1), (4096, 1), (512, 1), (32, 3)):
        data = w.seeded_bytes(9, w.STREAM_DATA, du * units)
        assert np.array_equal(run_xts(ctx, key, ENC, data, du, 7), oracle.xts(key, ENC, data, du, 7))
    # the last data-unit number there is (LE128 of 2^64 - 1), and units just below it
    for du, units, first in ((4096, 1, 2**64 - 1), (512, 4, 2**64 - 4)):
        data = w.seeded_bytes(10, w.STREAM_DATA, du * units)
        for dir in (ENC, DEC):
            assert np.array_equal(run_xts(ctx, key, dir, data, du, first), oracle.xts(key, dir, data, du, first))


def test_xts_in_place(ctx):
    import torch
    key = w.xts_key(5, 256)
    data = w.seeded_bytes(5, w.STREAM_DATA, 4096 * 77)
    kh = ctx.setkey(key, True)
    buf = to_dev(data)
    ctx.xts_crypt(kh, ENC, buf, buf, 4096, 3)
    assert np.array_equal(to_np(buf), oracle.xts(key, ENC, data, 4096, 3))
    ctx.xts_crypt(kh, DEC, buf, buf, 4096, 3)
    torch.cuda.synchronize()
    assert np.array_equal(to_np(buf), data)
    ctx.delkey(kh)


def test_xts_on_side_stream(ctx):
    import torch
    key = w.xts_key(6, 128)
    data = w.seeded_bytes(6, w.STREAM_DATA, 512 * 300)
    kh = ctx.setkey(key, True)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        src = to_dev(data)
        dst = torch.empty_like(src)
        ctx.xts_crypt(kh, ENC, src, dst, 512, 0, stream=s)
    s.synchronize()
    assert np.array_equal(to_np(dst), oracle.xts(key, ENC, data, 512, 0))
    ctx.delkey(kh)


def test_xts_argument_errors(ctx):
    import torch
    import paper_1305_3345_gb300 as kg
    key = w.xts_key(7, 256)
    kh = ctx.setkey(key, True)
    single = ctx.setkey(key[:32], False)
    buf = torch.zeros(8192 + 64, dtype=torch.uint8, device="cuda")
    L = kg.lib()
    h = ctx.handle
    p = buf.data_ptr()
    s = torch.cuda.current_stream().cuda_stream
    assert L.kgpu_aes_xts_crypt(h, kh, 0, p, p, 8192, 4096, 0, s) == 0
    assert L.kgpu_aes_xts_crypt(h, kh, 0, p, p, 8000, 4096, 0, s) == -22     # not whole units
    assert L.kgpu_aes_xts_crypt(h, kh, 0, p, p, 8002, 4001, 0, s) == 0       # du % 16: ciphertext stealing
    assert L.kgpu_aes_xts_crypt(h, kh, 0, p, p, 8192, 4001, 0, s) == -22     # not whole units
    assert L.kgpu_aes_xts_crypt(h, kh, 0, p, p, 80, 8, 0, s) == -22          # unit shorter than a block
    assert L.kgpu_aes_xts_crypt(h, kh, 2, p, p, 8192, 4096, 0, s) == -22     # bad direction
    assert L.kgpu_aes_xts_crypt(h, kh, 0, p + 8, p + 8, 4096, 4096, 0, s) == -22   # misaligned
    assert L.kgpu_aes_xts_crypt(h, kh, 0, p, p + 16, 4096, 4096, 0, s) == -22  # partial overlap
    assert L.kgpu_aes_xts_crypt(h, single, 0, p, p, 4096, 4096, 0, s) == -2  # not an XTS key
    assert L.kgpu_aes_xts_crypt(h, 999, 0, p, p, 4096, 4096, 0, s) == -2     # unknown key
    assert L.kgpu_aes_xts_crypt(h, kh, 0, p, p, 0, 4096, 0, s) == 0          # empty: no-op
    # a range that runs past the end of the allocation is refused, not launched
    assert L.kgpu_aes_xts_crypt(h, kh, 0, p, p, 1 << 40, 4096, 0, s) == -14
    host = np.zeros(4096, np.uint8)
    assert L.kgpu_aes_xts_crypt(h, kh, 0, host.ctypes.data, p, 4096, 4096, 0, s) == -14  # host pointer
    assert L.kgpu_aes_xts_crypt(h, kh, 0, p, p, 4096, 4096, 2**64 - 1, s) == 0   # one unit, last number
    assert L.kgpu_aes_xts_crypt(h, kh, 0, p, p, 8192, 4096, 2**64 - 1, s) == -22  # unit numbers wrap
    # K1 == K2 is rejected, and XTS takes AES-128 or AES-256 keys only
    with pytest.raises(kg.KgpuError):
        ctx.setkey(key[:32] * 2, True)
    with pytest.raises(kg.KgpuError):
        ctx.setkey(key[:48], True)
    torch.cuda.synchronize()
    ctx.delkey(kh)
    ctx.delkey(single)


def test_xts_full_size_sampled(ctx):
    """1 GiB as 262,144 x 4096-B sectors (the bulk workload), in the bench's launch
    configuration: sampled sectors against the oracle, and the whole buffer
    round-trips."""
    import torch
    key = w.xts_key(2, 256)
    n = 1 << 30
    data = torch.from_numpy(w.seeded_bytes(2, w.STREAM_DATA, n)).cuda()
    kh = ctx.setkey(key, True)
    enc = torch.empty_like(data)
    ctx.xts_crypt(kh, ENC, data, enc, 4096, 0)
    rng = np.random.default_rng(0)
    sample = np.unique(np.concatenate([[0, 1, 262143], rng.integers(0, 262144, 61)]))
    encv = enc.view(262144, 4096)
    datv = data.view(262144, 4096)
    for s in sample:
        s = int(s)
        ref = oracle.xts(key, ENC, datv[s].cpu().numpy(), 4096, s)
        assert np.array_equal(encv[s].cpu().numpy(), ref), s
    dec = torch.empty_like(data)
    ctx.xts_crypt(kh, DEC, enc, dec, 4096, 0)
    assert torch.equal(dec, data)
    assert not torch.equal(enc[:4096], data[:4096])
    ctx.delkey(kh)
    del data, enc, dec
    torch.cuda.empty_cache()


def test_xts_512b_units_full_size_sampled(ctx):
    """The 512-B-sector variant of the bulk workload: 2,097,152 units."""
    import torch
    key = w.xts_key(2, 128)
    n = 1 << 30
    data = torch.from_numpy(w.seeded_bytes(2, w.STREAM_DATA, n)).cuda()
    kh = ctx.setkey(key, True)
    enc = torch.empty_like(data)
    ctx.xts_crypt(kh, ENC, data, enc, 512, 0)
    rng = np.random.default_rng(1)
    sample = np.unique(np.concatenate([[0, 2097151], rng.integers(0, 2097152, 62)]))
    encv = enc.view(-1, 512)
    datv = data.view(-1, 512)
    for s in sample:
        s = int(s)
        assert np.array_equal(encv[s].cpu().numpy(), oracle.xts(key, ENC, datv[s].cpu().numpy(), 512, s)), s
    ctx.xts_crypt(kh, DEC, enc, enc, 512, 0)
    assert torch.equal(enc, data)
    ctx.delkey(kh)
    del data, enc
    torch.cuda.empty_cache()
