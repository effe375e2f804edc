"""The empty service (KGPU_MODE_COPY): the paper's round-trip measurement of
its Non-Stop Kernel uses a service that does no work on a 4 KB input
(section 3.1).  Here that service copies its input through unchanged, so its
output must equal its input byte for byte -- through the batch kernel, the
serving ring and one plain launch per request, with the pages in device memory
and in registered pinned host memory -- and bytes outside the request must be
left alone.
"""
import numpy as np
import pytest

import oracle
import workloads as w

pytestmark = pytest.mark.gpu

# bytes per warp-tile: a 4 KiB request then runs on 1, 16, 32 and 64 warps
# (32, 512, 1024 and 2048 threads), plus an odd tile of 48 B
TILES = (4096, 256, 128, 64, 48)


def copy_requests(kg, src, dst, sizes, tiles, flags=0):
    n = len(sizes)
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    r = np.zeros(n, dtype=kg.request_dtype())
    r["mode"] = kg.MODE_COPY
    r["src"] = src.data_ptr() + offs
    r["dst"] = dst.data_ptr() + offs
    r["len"] = sizes
    r["unit_size"] = tiles
    r["flags"] = flags
    return r, offs


def draw(seed, n):
    """n requests: tile sizes from TILES, lengths 1..40 tiles (4 KiB mostly)."""
    u = w.u64(seed, 3, 2 * n).reshape(n, 2)
    tiles = np.array(TILES, dtype=np.int64)[u[:, 0] % len(TILES)]
    count = np.where(u[:, 1] % 3 == 0, 1 + (u[:, 1] >> 8) % 40, 4096 // tiles)
    count = np.maximum(count, 1)
    return tiles * count, tiles


@pytest.mark.parametrize("where", ["device", "host"])
def test_empty_service_batched_and_launched(ctx, where):
    import torch
    import paper_1305_3345_gb300 as kg
    sizes, tiles = draw(301, 200)
    total = int(sizes.sum())
    data = w.seeded_bytes(301, w.STREAM_DATA, total + 4096)
    if where == "host":
        src = torch.from_numpy(data.copy()).pin_memory()
        outs = [torch.full((total + 4096,), 0xA5, dtype=torch.uint8).pin_memory() for _ in range(2)]
        for t in [src] + outs:
            ctx.host_register(t)
        flags = kg.REQ_SRC_HOST | kg.REQ_DST_HOST
    else:
        src = torch.from_numpy(data.copy()).cuda()
        outs = [torch.full((total + 4096,), 0xA5, dtype=torch.uint8, device="cuda") for _ in range(2)]
        flags = 0
    try:
        r0, _ = copy_requests(kg, src, outs[0], sizes, tiles, flags)
        r1, _ = copy_requests(kg, src, outs[1], sizes, tiles, flags)
        assert ctx.poll(ctx.submit(r0), -1) == 0
        arr = (np.arange(len(r1)) * 20_000).astype(np.uint64)
        rc, _, _ = ctx.replay_launches(r1, arr, nstreams=4)
        assert rc == 0
        torch.cuda.synchronize()
        for o in outs:
            got = o.cpu().numpy()
            assert np.array_equal(got[:total], data[:total])
            assert (got[total:] == 0xA5).all()
    finally:
        if where == "host":
            for t in [src] + outs:
                ctx.host_unregister(t)


@pytest.mark.parametrize("where", ["device", "host"])
def test_empty_service_through_the_ring(ctx, where):
    """One request at a time (the round-trip measurement's pattern) and then a
    burst, through the serving ring."""
    import torch
    import paper_1305_3345_gb300 as kg
    sizes, tiles = draw(302, 300)
    total = int(sizes.sum())
    data = w.seeded_bytes(302, w.STREAM_DATA, total)
    if where == "host":
        src = torch.from_numpy(data.copy()).pin_memory()
        dst = torch.zeros(total, dtype=torch.uint8).pin_memory()
        for t in (src, dst):
            ctx.host_register(t)
        flags = kg.REQ_SRC_HOST | kg.REQ_DST_HOST
    else:
        src = torch.from_numpy(data.copy()).cuda()
        dst = torch.zeros(total, dtype=torch.uint8, device="cuda")
        flags = 0
    torch.cuda.synchronize()
    try:
        r, _ = copy_requests(kg, src, dst, sizes, tiles, flags)
        ctx.serve_start()
        try:
            arr = (np.arange(150) * 100_000).astype(np.uint64)
            rc, lat, _ = ctx.replay_serve(r[:150], arr)
            assert rc == 0 and (lat < 10**9).all()
            rc, _, _ = ctx.replay_serve(r[150:], np.zeros(150, np.uint64))
            assert rc == 0
        finally:
            ctx.serve_stop(10_000_000_000)
        assert np.array_equal(dst.cpu().numpy(), data)
    finally:
        if where == "host":
            for t in (src, dst):
                ctx.host_unregister(t)


def test_empty_service_beside_cipher_requests(ctx):
    """Copy requests interleaved with XTS requests of one key in a batch: the
    copies need no key and leave the warps' cached key schedules usable."""
    import torch
    import paper_1305_3345_gb300 as kg
    key = w.xts_key(303, 256)
    kh = ctx.setkey(key, True)
    n, size = 64, 8192
    data = w.seeded_bytes(303, w.STREAM_DATA, n * size)
    src = torch.from_numpy(data.copy()).cuda()
    dst = torch.zeros_like(src)
    r = np.zeros(n, dtype=kg.request_dtype())
    xts = np.arange(n) % 2 == 0
    r["mode"] = np.where(xts, kg.MODE_XTS, kg.MODE_COPY)
    r["key"] = np.where(xts, kh, 0)
    r["src"] = src.data_ptr() + size * np.arange(n)
    r["dst"] = dst.data_ptr() + size * np.arange(n)
    r["len"] = size
    r["unit_size"] = np.where(xts, 4096, 128)
    r["sector"] = 2 * np.arange(n)
    assert ctx.poll(ctx.submit(r), -1) == 0
    got = dst.cpu().numpy().reshape(n, size)
    ref = oracle.xts(key, 0, data, 4096, 0).reshape(n, size)
    dat = data.reshape(n, size)
    for i in range(n):
        assert np.array_equal(got[i], ref[i] if xts[i] else dat[i]), i
    ctx.delkey(kh)


def test_empty_service_refusals(ctx):
    import torch
    import paper_1305_3345_gb300 as kg
    src = torch.zeros(8192, dtype=torch.uint8, device="cuda")
    dst = torch.zeros_like(src)
    for unit, length in ((0, 4096), (24, 4096), (4096, 4000), (1024, 4096 + 512)):
        r, _ = copy_requests(kg, src, dst, np.array([length]), np.array([unit]))
        st = np.zeros(1, np.int32)
        with pytest.raises(kg.KgpuError) as e:
            ctx.submit(r, status=st)
        assert e.value.code == "EINVAL" and st[0] == -22
    # a length past the end of the allocation is refused, not launched (in
    # place, so the overlap check does not answer first)
    r, _ = copy_requests(kg, src, src, np.array([1 << 40]), np.array([4096]))
    with pytest.raises(kg.KgpuError) as e:
        ctx.submit(r)
    assert e.value.code == "EFAULT"
