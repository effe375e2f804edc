"""Requests over registered host memory: the batched and serving kernels read
input pages from page-locked host memory and write output pages back there
directly over the NVLink-C2C link, with no staging copies.

Every result must equal the oracle byte for byte (AES output is exact, so the
tolerance is zero), and equal what the same request gives over device memory.
The error cases check that no host pointer reaches the GPU unless it lies in a
registered range: those requests are refused on the host before any launch.
"""
import mmap

import numpy as np
import pytest

import oracle
import workloads as w

pytestmark = pytest.mark.gpu


def pinned(nbytes):
    import torch
    return torch.zeros(nbytes, dtype=torch.uint8, pin_memory=True)


class HostTraffic:
    """Seeded requests (XTS both ways, CBC decrypt/encrypt, ECB; AES-128/256;
    sizes log-uniform lo..hi in 4-KiB pages) whose input, output and IVs all
    live in pinned host memory."""

    def __init__(self, ctx, seed, n, lo, hi, nkeys):
        import torch
        self.ctx = ctx
        mix = w.request_mix(seed, n, lo, hi, nkeys)
        self.modes = np.where(w.uniform01(seed, 98, n) < 0.15, w.MODE_ECB, mix.modes)
        self.dirs, self.sizes, self.offsets, self.kidx = mix.dirs, mix.sizes, mix.offsets, mix.keys
        self.keys, self.key_bits = w.mix_key_material(seed, mix), mix.key_bits
        self.hx = [ctx.setkey(k[: 2 * b // 8], True) for k, b in zip(self.keys, self.key_bits)]
        self.hs = [ctx.setkey(k[: b // 8], False) for k, b in zip(self.keys, self.key_bits)]
        total = int(self.sizes.sum())
        self.data = w.seeded_bytes(seed, w.STREAM_DATA, total)
        self.src = pinned(total)
        self.src.copy_(torch.from_numpy(self.data))
        self.out = pinned(total)
        npages = self.sizes // 4096
        self.iv_off = np.concatenate([[0], np.cumsum(npages)[:-1]])
        self.ivs_np = w.page_ivs(seed, int(npages.sum()))
        self.ivs = pinned(self.ivs_np.size)
        self.ivs.copy_(torch.from_numpy(self.ivs_np.reshape(-1).copy()))
        self.sectors = (w.u64(seed, 7, n) % (1 << 40)).astype(np.uint64)
        self.buffers = (self.src, self.out, self.ivs)
        for b in self.buffers:
            ctx.host_register(b)

    def array(self, src=None, dst=None, ivs=None, flags=None):
        """Requests as a request_dtype() array; src/dst/ivs override the base
        addresses (e.g. a device copy) and flags the residency bits."""
        import paper_1305_3345_gb300 as kg
        n = len(self.sizes)
        r = np.zeros(n, dtype=kg.request_dtype())
        cbc = (self.modes == w.MODE_CBC_DEC) | (self.modes == w.MODE_CBC_ENC)
        r["mode"] = self.modes
        r["dir"] = np.where(cbc, 0, self.dirs)
        r["key"] = np.where(self.modes == w.MODE_XTS, np.array(self.hx)[self.kidx], np.array(self.hs)[self.kidx])
        r["src"] = (src if src is not None else self.src.data_ptr()) + self.offsets
        r["dst"] = (dst if dst is not None else self.out.data_ptr()) + self.offsets
        r["len"] = self.sizes
        r["unit_size"] = 4096
        r["sector"] = self.sectors
        r["ivs"] = np.where(cbc, (ivs if ivs is not None else self.ivs.data_ptr()) + 16 * self.iv_off, 0)
        if flags is None:
            import paper_1305_3345_gb300 as kg
            flags = kg.REQ_SRC_HOST | kg.REQ_DST_HOST | kg.REQ_IVS_HOST
        r["flags"] = np.where(cbc, flags, flags & ~4)
        return r

    def expected(self, i):
        m, k = int(self.modes[i]), int(self.kidx[i])
        bits = int(self.key_bits[k])
        a, b = int(self.offsets[i]), int(self.offsets[i] + self.sizes[i])
        x = self.data[a:b]
        if m == w.MODE_XTS:
            return oracle.xts(self.keys[k][: 2 * bits // 8], int(self.dirs[i]), x, 4096, int(self.sectors[i]))
        if m == w.MODE_ECB:
            return oracle.ecb(self.keys[k][: bits // 8], int(self.dirs[i]), x)
        p0 = int(self.iv_off[i])
        return oracle.cbc(self.keys[k][: bits // 8], 0 if m == w.MODE_CBC_ENC else 1, x, 4096,
                          self.ivs_np[p0:p0 + int(self.sizes[i]) // 4096])

    def span(self, buf, i):
        a, b = int(self.offsets[i]), int(self.offsets[i] + self.sizes[i])
        return buf[a:b].cpu().numpy()

    def close(self):
        for b in self.buffers:
            self.ctx.host_unregister(b)
        for h in self.hx + self.hs:
            self.ctx.delkey(h)


def run_batch(ctx, reqs):
    st = np.full(len(reqs), 7, np.int32)
    t = ctx.submit(reqs, status=st)
    assert ctx.poll(t, -1, st) == 0
    assert not st.any()


def test_batch_over_host_pages_vs_oracle_and_device(ctx):
    import torch
    t = HostTraffic(ctx, seed=301, n=48, lo=4096, hi=256 << 10, nkeys=8)
    try:
        run_batch(ctx, t.array())
        for i in range(len(t.sizes)):
            assert np.array_equal(t.span(t.out, i), t.expected(i)), (i, int(t.modes[i]))
        # the same requests over device copies of the buffers give the same bytes
        dsrc, divs = t.src.cuda(), t.ivs.cuda()
        dout = torch.zeros_like(dsrc)
        run_batch(ctx, t.array(dsrc.data_ptr(), dout.data_ptr(), divs.data_ptr(), flags=0))
        torch.cuda.synchronize()
        assert torch.equal(dout.cpu(), t.out)
    finally:
        t.close()


def test_mixed_residency_and_in_place(ctx):
    """Host -> device, device -> host, and in place in host memory."""
    import torch
    import paper_1305_3345_gb300 as kg
    t = HostTraffic(ctx, seed=302, n=24, lo=4096, hi=128 << 10, nkeys=4)
    try:
        divs = t.ivs.cuda()
        dout = torch.zeros(t.src.numel(), dtype=torch.uint8, device="cuda")
        run_batch(ctx, t.array(dst=dout.data_ptr(), ivs=divs.data_ptr(), flags=kg.REQ_SRC_HOST))
        torch.cuda.synchronize()
        dsrc = t.src.cuda()
        run_batch(ctx, t.array(src=dsrc.data_ptr(), flags=kg.REQ_DST_HOST | kg.REQ_IVS_HOST))
        for i in range(len(t.sizes)):
            e = t.expected(i)
            a, b = int(t.offsets[i]), int(t.offsets[i] + t.sizes[i])
            assert np.array_equal(dout[a:b].cpu().numpy(), e), ("to device", i)
            assert np.array_equal(t.span(t.out, i), e), ("to host", i)
        # in place: src == dst, both host
        run_batch(ctx, t.array(dst=t.src.data_ptr()))
        for i in range(len(t.sizes)):
            assert np.array_equal(t.span(t.src, i), t.expected(i)), ("in place", i)
    finally:
        t.close()


def test_library_pins_pageable_memory(ctx):
    """KGPU_HOSTREG_PIN: the library page-locks an ordinary (mmap) buffer, the
    kernels work on it in place, and unregistering unpins it so that it can be
    registered again."""
    import paper_1305_3345_gb300 as kg
    nbytes = 64 * 4096
    m = mmap.mmap(-1, nbytes)
    buf = np.frombuffer(m, dtype=np.uint8)
    data = w.seeded_bytes(303, w.STREAM_DATA, nbytes)
    buf[:] = data
    key = w.xts_key(303, 256)
    kh = ctx.setkey(key, True)
    try:
        for rep in range(2):
            ctx.host_register(buf, flags=kg.HOSTREG_PIN)
            r = np.zeros(1, dtype=kg.request_dtype())
            r["mode"], r["dir"], r["key"] = w.MODE_XTS, rep, kh
            r["src"] = r["dst"] = buf.ctypes.data
            r["len"], r["unit_size"], r["sector"] = nbytes, 4096, 500
            r["flags"] = kg.REQ_SRC_HOST | kg.REQ_DST_HOST
            run_batch(ctx, r)
            ctx.host_unregister(buf)
            want = oracle.xts(key, 0, data, 4096, 500) if rep == 0 else data
            assert np.array_equal(buf, want), rep
    finally:
        ctx.delkey(kh)
        del buf
        m.close()


def test_serving_over_host_pages(ctx):
    """The serving ring with every buffer in registered host memory."""
    t = HostTraffic(ctx, seed=304, n=40, lo=4096, hi=256 << 10, nkeys=8)
    reqs = t.array()
    try:
        ctx.serve_start()
        try:
            tickets = [ctx.serve_submit(reqs[i]) for i in range(len(reqs))]
            for tk in tickets:
                rc, st, _ = ctx.serve_poll(tk, 10_000_000_000)
                assert rc == 0 and st == 0
        finally:
            assert ctx.serve_stop(5_000_000_000) == 0
        for i in range(len(t.sizes)):
            assert np.array_equal(t.span(t.out, i), t.expected(i)), (i, int(t.modes[i]))
    finally:
        t.close()


def test_host_request_errors_are_refused_before_launch(ctx):
    import torch
    import paper_1305_3345_gb300 as kg
    L, h = kg.lib(), ctx.handle
    reg = pinned(16 * 4096)
    other = pinned(4 * 4096)         # pinned, but never registered
    dev = torch.zeros(16 * 4096, dtype=torch.uint8, device="cuda")
    kh = ctx.setkey(w.xts_key(305, 256), True)
    ctx.host_register(reg)
    try:
        def req(src, dst, ln, flags):
            r = np.zeros(1, dtype=kg.request_dtype())
            r["mode"], r["dir"], r["key"] = w.MODE_XTS, 0, kh
            r["src"], r["dst"], r["len"], r["unit_size"], r["flags"] = src, dst, ln, 4096, flags
            return r

        HH = kg.REQ_SRC_HOST | kg.REQ_DST_HOST
        base = reg.data_ptr()
        cases = [
            (req(base, base, 4096, 0x8), "EINVAL"),                               # unknown flag bit
            (req(other.data_ptr(), base, 4096, HH), "EFAULT"),                    # unregistered host range
            (req(base + 15 * 4096, base, 2 * 4096, HH), "EFAULT"),                # runs past the range's end
            (req(dev.data_ptr(), base, 4096, HH), "EFAULT"),                      # device pointer flagged host
            (req(base, dev.data_ptr(), 4096, 0), "EFAULT"),                       # host pointer not flagged
            (req(base, base + 4096, 2 * 4096, HH), "EINVAL"),                     # partial overlap
        ]
        for r, code in cases:
            with pytest.raises(kg.KgpuError) as e:
                ctx.submit(r)
            assert e.value.code == code, (code, e.value.code)
        # registration errors
        assert L.kgpu_host_register(h, reg.data_ptr() + 4096, 4096, 1) == -22      # overlaps a registered range
        assert L.kgpu_host_register(h, reg.data_ptr(), 4096, 9) == -22             # unknown flag
        assert L.kgpu_host_register(h, None, 4096, 1) == -22
        pageable = np.zeros(8 * 4096, np.uint8)
        assert L.kgpu_host_register(h, pageable.ctypes.data, pageable.nbytes, 1) == -14  # not pinned
        assert L.kgpu_host_register(h, dev.data_ptr(), 4096, 1) == -14                   # device memory
        assert L.kgpu_host_unregister(h, reg.data_ptr() + 4096) == -2                    # not a range start
        assert L.kgpu_host_unregister(h, other.data_ptr()) == -2
        torch.cuda.synchronize()
        assert not dev.any() and not reg.any()   # nothing ran
    finally:
        ctx.host_unregister(reg)
        ctx.delkey(kh)


@pytest.mark.parametrize("threads", [512, 1024])
@pytest.mark.parametrize("page,npages", [(4096, 45), (512, 1025), (4112, 33), (48, 70), (128, 31)])
def test_cbc_encrypt_of_host_pages(ctx, threads, page, npages):
    """CBC encryption over host pages: pages of a multiple of 8 blocks go
    through the staged (whole-line) copies, the others through direct loads;
    ragged page counts leave part of the last 32-page tile empty."""
    import torch
    import paper_1305_3345_gb300 as kg
    seed = 306 + page + npages
    data = w.seeded_bytes(seed, w.STREAM_DATA, page * npages)
    ivs_np = w.page_ivs(seed, npages)
    key = w.single_key(seed, 128)
    src, dst = pinned(data.size), pinned(data.size)
    src.copy_(torch.from_numpy(data))
    ivs = pinned(ivs_np.size)
    ivs.copy_(torch.from_numpy(ivs_np.reshape(-1).copy()))
    kh = ctx.setkey(key, False)
    before = ctx.get_tuning()
    for b in (src, dst, ivs):
        ctx.host_register(b)
    try:
        ctx.set_tuning(threads=threads, tile_chunks=32)
        r = np.zeros(1, dtype=kg.request_dtype())
        r["mode"], r["key"] = w.MODE_CBC_ENC, kh
        r["src"], r["dst"], r["ivs"] = src.data_ptr(), dst.data_ptr(), ivs.data_ptr()
        r["len"], r["unit_size"] = data.size, page
        r["flags"] = kg.REQ_SRC_HOST | kg.REQ_DST_HOST | kg.REQ_IVS_HOST
        run_batch(ctx, r)
        assert np.array_equal(dst.numpy(), oracle.cbc(key, 0, data, page, ivs_np))
    finally:
        ctx.set_tuning(threads=before["threads"], tile_chunks=before["tile_chunks"], ctas=before["ctas"])
        for b in (src, dst, ivs):
            ctx.host_unregister(b)
        ctx.delkey(kh)


@pytest.mark.parametrize("bits", [128, 192, 256])
@pytest.mark.parametrize("page,npages", [(4096, 45), (512, 1025), (128, 31), (4112, 33), (1024, 9)])
def test_cbc_encrypt_of_host_pages_through_the_ring(ctx, bits, page, npages):
    """CBC encryption of host pages through the serving ring while it keeps up:
    pages of a multiple of 8 blocks run four lanes to a page through the
    warp's scratch (8 pages a tile, whole-line copies, the next chunk fetched
    while the current one is enciphered), the others one lane per page; one
    request alone, then the same request in place."""
    import torch
    import paper_1305_3345_gb300 as kg
    seed = 900 + page + npages + bits
    data = w.seeded_bytes(seed, w.STREAM_DATA, page * npages)
    ivs_np = w.page_ivs(seed, npages)
    key = w.single_key(seed, bits)
    src, dst = pinned(data.size), pinned(data.size)
    src.copy_(torch.from_numpy(data))
    ivs = pinned(ivs_np.size)
    ivs.copy_(torch.from_numpy(ivs_np.reshape(-1).copy()))
    kh = ctx.setkey(key, False)
    for b in (src, dst, ivs):
        ctx.host_register(b)
    ref = oracle.cbc(key, 0, data, page, ivs_np)
    try:
        ctx.serve_start()
        try:
            for out in (dst, src):
                r = np.zeros(1, dtype=kg.request_dtype())
                r["mode"], r["key"] = w.MODE_CBC_ENC, kh
                r["src"], r["dst"], r["ivs"] = src.data_ptr(), out.data_ptr(), ivs.data_ptr()
                r["len"], r["unit_size"] = data.size, page
                r["flags"] = kg.REQ_SRC_HOST | kg.REQ_DST_HOST | kg.REQ_IVS_HOST
                rc, st, _ = ctx.serve_poll(ctx.serve_submit(r[0]), 10_000_000_000)
                assert rc == 0 and st == 0
                assert np.array_equal(out.numpy(), ref)
        finally:
            assert ctx.serve_stop(5_000_000_000) == 0
    finally:
        for b in (src, dst, ivs):
            ctx.host_unregister(b)
        ctx.delkey(kh)
