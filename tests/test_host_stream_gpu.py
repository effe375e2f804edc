"""Host-resident pages streamed through the device (pinned and pageable),
chunked with copy/compute overlap: bit-exact against the oracle."""
import numpy as np
import pytest

import oracle
import workloads as w

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("chunk", [0, 65536, 1 << 20, 3 * 4096, 7 << 20])
def test_host_stream_pinned(ctx, chunk):
    import torch
    key = w.xts_key(16, 256)
    n = 4096 * 1000 + 4096 * 3
    data = w.seeded_bytes(16, w.STREAM_DATA, n)
    src = torch.from_numpy(data.copy()).pin_memory()
    dst = torch.empty(n, dtype=torch.uint8).pin_memory()
    kh = ctx.setkey(key, True)
    ctx.xts_crypt_host(kh, 0, src, dst, 4096, 11, chunk)
    assert np.array_equal(dst.numpy(), oracle.xts(key, 0, data, 4096, 11))
    ctx.xts_crypt_host(kh, 1, dst, dst, 4096, 11, chunk)   # in place
    assert np.array_equal(dst.numpy(), data)
    ctx.delkey(kh)


def test_host_stream_pageable_512(ctx):
    key = w.xts_key(17, 128)
    data = w.seeded_bytes(17, w.STREAM_DATA, 512 * 5000)
    out = np.empty_like(data)
    kh = ctx.setkey(key, True)
    ctx.xts_crypt_host(kh, 0, data, out, 512, 0, 1 << 18)
    assert np.array_equal(out, oracle.xts(key, 0, data, 512, 0))
    ctx.delkey(kh)


def test_host_stream_rejects_device_pointer(ctx):
    import torch
    import paper_1305_3345_gb300 as kg
    kh = ctx.setkey(w.xts_key(18, 128), True)
    d = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    assert kg.lib().kgpu_aes_xts_crypt_host(ctx.handle, kh, 0, d.data_ptr(), d.data_ptr(), 4096, 4096, 0, 0) == -14
    ctx.delkey(kh)


@pytest.mark.parametrize("bits,du", [(256, 4096), (128, 512)])
def test_host_call_on_registered_pages_in_place_over_the_link(ctx, bits, du):
    """Both buffers registered: the call runs the kernel on the host pages
    directly (no staging).  Out of place, in place and decryption must equal
    the oracle; with only one buffer registered the call takes the copy
    pipeline and gives the same bytes; unregistering afterwards succeeds."""
    import torch
    key = w.xts_key(19 + bits, bits)
    n = du * 3001
    data = w.seeded_bytes(19 + du, w.STREAM_DATA, n)
    src = torch.from_numpy(data.copy()).pin_memory()
    dst = torch.zeros(n, dtype=torch.uint8).pin_memory()
    other = torch.zeros(n, dtype=torch.uint8).pin_memory()
    kh = ctx.setkey(key, True)
    ref = oracle.xts(key, 0, data, du, 2**40 + 3)
    ctx.host_register(src)
    ctx.host_register(dst)
    try:
        ctx.xts_crypt_host(kh, 0, src, dst, du, 2**40 + 3, 0)
        assert np.array_equal(dst.numpy(), ref)
        ctx.xts_crypt_host(kh, 0, src, other, du, 2**40 + 3, 1 << 20)   # dst not registered: pipeline
        assert np.array_equal(other.numpy(), ref)
        ctx.xts_crypt_host(kh, 1, dst, dst, du, 2**40 + 3, 0)           # in place, registered
        assert np.array_equal(dst.numpy(), data)
    finally:
        ctx.host_unregister(src)
        ctx.host_unregister(dst)
    ctx.delkey(kh)

