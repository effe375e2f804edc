"""kgpu_crypt and the CPU/GPU crossover (the paper's proposal, section 4: measure
at start-up where the GPU overtakes the CPU and send smaller requests to the
CPU).

Both legs must give the oracle's bytes: the GPU leg (the library's kernels,
through one launch or the serving ring) and the host leg (OpenSSL's
libcrypto on registered host pages).  Routed and unrouted results are
compared with each other and with the oracle; the router must send only
host-resident requests below the measured crossover to the host.
"""
import numpy as np
import pytest

import oracle
import workloads as w

pytestmark = pytest.mark.gpu


class HostPages:
    """Registered pinned input, output and IV buffers of `size` bytes."""

    def __init__(self, ctx, seed, size, page=4096):
        import torch
        self.ctx = ctx
        self.data = w.seeded_bytes(seed, w.STREAM_DATA, size)
        self.ivs_np = w.page_ivs(seed, max(1, size // page))
        self.src = torch.from_numpy(self.data.copy()).pin_memory()
        self.dst = torch.zeros(size, dtype=torch.uint8).pin_memory()
        self.ivs = torch.from_numpy(self.ivs_np.reshape(-1).copy()).pin_memory()
        for t in (self.src, self.dst, self.ivs):
            ctx.host_register(t)

    def close(self):
        for t in (self.src, self.dst, self.ivs):
            self.ctx.host_unregister(t)


def request(kg, mode, key, src, dst, n, unit, sector=0, ivs=None, dir=0, flags=None):
    r = np.zeros(1, dtype=kg.request_dtype())
    r["mode"], r["key"], r["dir"], r["len"], r["unit_size"], r["sector"] = mode, key, dir, n, unit, sector
    r["src"], r["dst"] = src, dst
    r["ivs"] = ivs or 0
    if flags is None:
        flags = kg.REQ_SRC_HOST | kg.REQ_DST_HOST | (kg.REQ_IVS_HOST if ivs else 0)
    r["flags"] = flags
    return r


CASES = [  # mode, key bits, dir, bytes, unit
    ("xts", 256, 0, 64 << 10, 4096), ("xts", 256, 1, 12 << 10, 4096), ("xts", 128, 0, 8 << 10, 512),
    ("xts", 128, 1, 4096, 16), ("cbc_enc", 128, 0, 12 << 10, 4096), ("cbc_enc", 192, 0, 4096, 512),
    ("cbc_enc", 256, 0, 32 << 10, 4096), ("cbc_dec", 128, 0, 12 << 10, 4096), ("cbc_dec", 256, 0, 8192, 1024),
    ("ecb", 128, 0, 4096, 16), ("ecb", 256, 1, 48 << 10, 16), ("ecb", 192, 0, 4112, 16),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join(map(str, c)))
@pytest.mark.parametrize("in_place", [False, True])
def test_host_and_gpu_legs_equal_the_oracle(ctx, case, in_place):
    import torch
    import paper_1305_3345_gb300 as kg
    name, bits, dir, size, unit = case
    seed = 400 + CASES.index(case)
    xts = name == "xts"
    key = w.xts_key(seed, bits) if xts else w.single_key(seed, bits)
    kh = ctx.setkey(key, xts)
    hp = HostPages(ctx, seed, size, unit)
    try:
        mode = {"xts": kg.MODE_XTS, "cbc_enc": kg.MODE_CBC_ENC, "cbc_dec": kg.MODE_CBC_DEC, "ecb": kg.MODE_ECB}[name]
        if name == "xts":
            ref = oracle.xts(key, dir, hp.data, unit, 77)
        elif name == "ecb":
            ref = oracle.ecb(key, dir, hp.data)
        else:
            ref = oracle.cbc(key, 0 if name == "cbc_enc" else 1, hp.data, unit, hp.ivs_np[: size // unit])
        for leg in (kg.DISPATCH_HOST, kg.DISPATCH_GPU):
            hp.src.copy_(torch.from_numpy(hp.data))
            hp.dst.zero_()
            out = hp.src if in_place else hp.dst
            r = request(kg, mode, kh, hp.src.data_ptr(), out.data_ptr(), size, unit, 77,
                        hp.ivs.data_ptr() if name.startswith("cbc") else None, dir)
            st, ran = ctx.crypt(r, leg)
            assert st == 0 and ran == leg
            assert np.array_equal(out.numpy(), ref), (name, bits, leg)
    finally:
        hp.close()
        ctx.delkey(kh)


def test_auto_dispatch_routes_by_the_measured_crossover():
    import torch
    import paper_1305_3345_gb300 as kg
    cfg = kg.KgpuConfig()
    cfg.host_dispatch = 1
    with kg.Context(0, cfg) as c:          # calibrates at creation
        xo = c.crossover()
        assert xo["valid"] and xo["form"] == "launch"
        for name in ("xts", "cbc_dec", "cbc_enc", "ecb"):
            for kb in ("aes128", "aes256"):
                assert xo["bytes"][name][kb] in [4096 << i for i in range(12)]
        key = w.xts_key(420, 256)
        kh = c.setkey(key, True)
        cross = xo["bytes"]["xts"]["aes256"]
        small, big = max(512, cross // 2), cross
        hp = HostPages(c, 420, big, 512)
        dsrc = torch.from_numpy(hp.data.copy()).cuda()
        ddst = torch.zeros_like(dsrc)
        try:
            for n, want in ((small, kg.DISPATCH_HOST), (big, kg.DISPATCH_GPU)):
                hp.dst.zero_()
                r = request(kg, kg.MODE_XTS, kh, hp.src.data_ptr(), hp.dst.data_ptr(), n, 512, 5)
                st, ran = c.crypt(r)
                assert st == 0 and ran == want, (n, cross)
                assert np.array_equal(hp.dst.numpy()[:n], oracle.xts(key, 0, hp.data[:n], 512, 5))
                # the same request forced onto the other leg: the same bytes
                other = kg.DISPATCH_GPU if want == kg.DISPATCH_HOST else kg.DISPATCH_HOST
                first = hp.dst.numpy()[:n].copy()
                hp.dst.zero_()
                assert c.crypt(r, other) == (0, other)
                assert np.array_equal(hp.dst.numpy()[:n], first)
            # device-resident requests always take the GPU leg
            r = request(kg, kg.MODE_XTS, kh, dsrc.data_ptr(), ddst.data_ptr(), small, 512, 5, flags=0)
            assert c.crypt(r) == (0, kg.DISPATCH_GPU)
            torch.cuda.synchronize()
            assert np.array_equal(ddst.cpu().numpy()[:small], oracle.xts(key, 0, hp.data[:small], 512, 5))
            # with the serving ring running, the GPU leg is the ring
            c.serve_start()
            try:
                hp.dst.zero_()
                r = request(kg, kg.MODE_XTS, kh, hp.src.data_ptr(), hp.dst.data_ptr(), big, 512, 5)
                assert c.crypt(r, kg.DISPATCH_GPU) == (0, kg.DISPATCH_GPU)
                assert np.array_equal(hp.dst.numpy(), oracle.xts(key, 0, hp.data, 512, 5))
                xo2, pts = c.calibrate_dispatch()
                assert xo2["form"] == "ring" and len(pts) == 88
            finally:
                c.serve_stop(10_000_000_000)
        finally:
            hp.close()
            c.delkey(kh)


def test_calibration_points_give_the_recorded_crossover(ctx):
    import paper_1305_3345_gb300 as kg
    xo, pts = ctx.calibrate_dispatch()
    assert xo["valid"] and len(pts) == 88
    assert all(p["host_ns"] > 0 and p["gpu_ns"] > 0 for p in pts)
    for name in ("xts", "cbc_dec", "cbc_enc", "ecb"):
        for bits in (128, 256):
            curve = sorted((p for p in pts if p["mode"] == name and p["key_bits"] == bits), key=lambda p: p["bytes"])
            assert [p["bytes"] for p in curve] == [4096 << i for i in range(11)]
            cross = 2 * curve[-1]["bytes"]
            for p in reversed(curve):
                if p["gpu_ns"] >= p["host_ns"]:
                    break
                cross = p["bytes"]
            assert xo["bytes"][name][f"aes{bits}"] == cross
    # the context was made without host_dispatch: AUTO stays on the GPU
    key = w.single_key(421, 128)
    kh = ctx.setkey(key, False)
    hp = HostPages(ctx, 421, 4096)
    try:
        r = request(kg, kg.MODE_ECB, kh, hp.src.data_ptr(), hp.dst.data_ptr(), 4096, 16)
        assert ctx.crypt(r) == (0, kg.DISPATCH_GPU)
        assert np.array_equal(hp.dst.numpy(), oracle.ecb(key, 0, hp.data))
    finally:
        hp.close()
        ctx.delkey(kh)


def test_host_leg_refusals(ctx):
    import torch
    import paper_1305_3345_gb300 as kg
    key = w.single_key(422, 128)
    kh = ctx.setkey(key, False)
    d = torch.zeros(8192, dtype=torch.uint8, device="cuda")
    hp = HostPages(ctx, 422, 8192)
    try:
        # device buffers cannot take the host leg
        r = request(kg, kg.MODE_ECB, kh, d.data_ptr(), d.data_ptr(), 4096, 16, flags=0)
        assert ctx.crypt(r, kg.DISPATCH_HOST)[0] == -22
        # CBC on host pages but with the IVs in device memory
        r = request(kg, kg.MODE_CBC_ENC, kh, hp.src.data_ptr(), hp.dst.data_ptr(), 8192, 4096, ivs=d.data_ptr(),
                    flags=kg.REQ_SRC_HOST | kg.REQ_DST_HOST)
        assert ctx.crypt(r, kg.DISPATCH_HOST)[0] == -22
        # an unknown dispatch value, an empty request, an unknown key
        r = request(kg, kg.MODE_ECB, kh, hp.src.data_ptr(), hp.dst.data_ptr(), 4096, 16)
        assert ctx.crypt(r, 7)[0] == -22
        r0 = request(kg, kg.MODE_ECB, kh, hp.src.data_ptr(), hp.dst.data_ptr(), 0, 16)
        assert ctx.crypt(r0, kg.DISPATCH_HOST)[0] == -22
        r["key"] = 4000
        assert ctx.crypt(r, kg.DISPATCH_HOST)[0] == -2
        assert not hp.dst.numpy().any()
    finally:
        hp.close()
        ctx.delkey(kh)


def test_concurrent_callers_on_both_legs(ctx):
    """Four threads call kgpu_crypt at once, alternating the host and GPU legs
    (each thread keeps its own OpenSSL context), with the serving ring as the
    GPU leg; every output equals the oracle's."""
    import threading
    import paper_1305_3345_gb300 as kg
    key = w.xts_key(430, 256)
    kh = ctx.setkey(key, True)
    nthreads, calls, size = 4, 12, 16 << 10
    hps = [HostPages(ctx, 430 + t, calls * size) for t in range(nthreads)]
    errors = []

    def worker(t):
        try:
            hp = hps[t]
            for i in range(calls):
                leg = kg.DISPATCH_HOST if (i + t) % 2 else kg.DISPATCH_GPU
                r = request(kg, kg.MODE_XTS, kh, hp.src.data_ptr() + i * size, hp.dst.data_ptr() + i * size,
                            size, 4096, 1000 * t + 4 * i)
                st, ran = ctx.crypt(r, leg, 10_000_000_000)
                if st != 0 or ran != leg:
                    errors.append((t, i, st, ran))
        except Exception as e:  # surfaced below
            errors.append((t, repr(e)))

    ctx.serve_start()
    try:
        ths = [threading.Thread(target=worker, args=(t,)) for t in range(nthreads)]
        for th in ths:
            th.start()
        for th in ths:
            th.join()
    finally:
        ctx.serve_stop(10_000_000_000)
    try:
        assert not errors, errors
        for t, hp in enumerate(hps):
            got = hp.dst.numpy().reshape(calls, size)
            for i in range(calls):
                ref = oracle.xts(key, 0, hp.data[i * size:(i + 1) * size], 4096, 1000 * t + 4 * i)
                assert np.array_equal(got[i], ref), (t, i)
    finally:
        for hp in hps:
            hp.close()
        ctx.delkey(kh)
