"""Bitsliced XTS-AES encryption (the comparison variant of the table kernels)
against the CPU oracle, bit-exact (AES output is exact: zero tolerance).

Each thread of the bitsliced kernel enciphers 32 blocks as bit-planes and a
warp covers 1024 blocks, so the cases below put tails at every level: units
of one block (every block its own tweak), units that straddle a lane's
32-block steps, spans that end mid-warp, and sector numbers near the top of
the 64-bit range.
"""
import numpy as np
import pytest

import oracle
import workloads as w
from conftest import to_dev, to_np

pytestmark = pytest.mark.gpu


def run_bs(ctx, key_bytes, data, du, first):
    kh = ctx.setkey(key_bytes, True)
    try:
        src = to_dev(data)
        dst = src.new_empty(src.shape)
        ctx.xts_crypt_bitsliced(kh, 0, src, dst, du, first)
        return to_np(dst)
    finally:
        ctx.delkey(kh)


@pytest.mark.parametrize("bits", [128, 256])
@pytest.mark.parametrize("du,units,first", [
    (4096, 301, 0),            # spans of 4 units per warp, ragged last span
    (512, 2049, 2**40 + 17),   # one unit per lane step
    (16, 1537, 5),             # one block per unit: every block starts a unit
    (48, 999, 2**63),          # 3 blocks per unit: units straddle lane steps
    (4112, 67, 1),             # 257 blocks per unit, not a multiple of 32
    (65536, 9, 100),           # 4096 blocks per unit
    (4096, 1, 2**64 - 1),      # one unit, the last unit number
])
def test_bitsliced_xts_vs_oracle(ctx, bits, du, units, first):
    key = w.xts_key(40 + bits, bits)
    data = w.seeded_bytes(41 + du, w.STREAM_DATA, du * units)
    assert np.array_equal(run_bs(ctx, key, data, du, first), oracle.xts(key, 0, data, du, first)), (bits, du)


def test_bitsliced_equals_table_kernel_and_in_place(ctx):
    """64 MiB: the bitsliced and table kernels give identical bytes, and the
    bitsliced one works in place."""
    import torch
    key = w.xts_key(42, 256)
    data = w.seeded_bytes(42, w.STREAM_DATA, 64 << 20)
    kh = ctx.setkey(key, True)
    src = to_dev(data)
    a, b = torch.empty_like(src), torch.empty_like(src)
    ctx.xts_crypt(kh, 0, src, a, 4096, 77)
    ctx.xts_crypt_bitsliced(kh, 0, src, b, 4096, 77)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    ctx.xts_crypt_bitsliced(kh, 0, src, src, 4096, 77)
    torch.cuda.synchronize()
    assert torch.equal(src, a)
    ctx.delkey(kh)


def test_bitsliced_full_size_sampled(ctx):
    """1 GiB as 262,144 x 4096-B sectors (the bench's bulk workload):
    sampled sectors against the oracle."""
    import torch
    key = w.xts_key(2, 256)
    n = 1 << 30
    src = torch.empty(n, dtype=torch.uint8, device="cuda")
    src.copy_(torch.from_numpy(w.seeded_bytes(2, w.STREAM_DATA, n)))
    dst = torch.empty_like(src)
    kh = ctx.setkey(key, True)
    ctx.xts_crypt_bitsliced(kh, 0, src, dst, 4096, 0)
    torch.cuda.synchronize()
    rng = np.random.default_rng(43)
    for s in sorted(set(rng.integers(0, n // 4096, 24).tolist()) | {0, n // 4096 - 1}):
        plain = to_np(src[s * 4096:(s + 1) * 4096])
        got = to_np(dst[s * 4096:(s + 1) * 4096])
        assert np.array_equal(got, oracle.xts(key, 0, plain, 4096, s)), s
    ctx.delkey(kh)


def test_bitsliced_argument_errors(ctx):
    import torch
    import paper_1305_3345_gb300 as kg
    key = w.xts_key(44, 256)
    kh = ctx.setkey(key, True)
    buf = torch.zeros(8192, dtype=torch.uint8, device="cuda")
    L, h, p = kg.lib(), ctx.handle, buf.data_ptr()
    s = torch.cuda.current_stream().cuda_stream
    f = L.kgpu_aes_xts_crypt_bitsliced
    assert f(h, kh, 1, p, p, 8192, 4096, 0, s) == -22          # decryption is table-only
    assert f(h, kh, 0, p, p, 8000, 4096, 0, s) == -22          # not whole units
    assert f(h, kh, 0, p, p, 8002, 4001, 0, s) == -22          # partial blocks: table path only
    assert f(h, kh, 0, p, p + 16, 4096, 4096, 0, s) == -22     # partial overlap
    assert f(h, kh, 0, p, p, 1 << 40, 4096, 0, s) == -14       # past the allocation
    assert f(h, 999, 0, p, p, 4096, 4096, 0, s) == -2          # unknown key
    assert f(h, kh, 0, p, p, 0, 4096, 0, s) == 0               # empty: no-op
    torch.cuda.synchronize()
    assert not buf.any()                                       # nothing ran
    ctx.delkey(kh)
