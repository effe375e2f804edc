"""Serving loop: a persistent kernel fed through a ring in pinned host memory.

Checks bit-exact results against the oracle, that every request's result is
the same alone as in a concurrent mix, admission control (EBUSY), the bounded
idle exit with transparent relaunch, and the trace-replay load generators.
All buffers are prepared before serving starts: while the serving kernel runs
it holds every SM, so the tests only copy memory meanwhile.
"""
import threading
import time

import numpy as np
import pytest

import oracle
import workloads as w

pytestmark = pytest.mark.gpu


class Traffic:
    """Seeded requests (sizes log-uniform lo..hi, mixed modes and keys) over one
    input pool, each with its own output region."""

    def __init__(self, ctx, seed, n, lo, hi, nkeys, ecb=0.1):
        import torch
        import paper_1305_3345_gb300 as kg
        self.ctx = ctx
        mix = w.request_mix(seed, n, lo, hi, nkeys)
        u = w.uniform01(seed, 98, n)
        self.modes = np.where(u < ecb, w.MODE_ECB, mix.modes)
        self.dirs, self.sizes, self.offsets, self.kidx = mix.dirs, mix.sizes, mix.offsets, mix.keys
        self.keys, self.key_bits = w.mix_key_material(seed, mix), mix.key_bits
        self.hx = [ctx.setkey(k[: 2 * b // 8], True) for k, b in zip(self.keys, self.key_bits)]
        self.hs = [ctx.setkey(k[: b // 8], False) for k, b in zip(self.keys, self.key_bits)]
        total = int(self.sizes.sum())
        self.data = w.seeded_bytes(seed, w.STREAM_DATA, total)
        self.src = torch.from_numpy(self.data.copy()).cuda()
        self.out = [torch.zeros_like(self.src) for _ in range(2)]
        npages = self.sizes // 4096
        self.iv_off = np.concatenate([[0], np.cumsum(npages)[:-1]])
        self.ivs_np = w.page_ivs(seed, int(npages.sum()))
        self.ivs = torch.from_numpy(self.ivs_np.reshape(-1).copy()).cuda()
        self.sectors = (w.u64(seed, 7, n) % (1 << 40)).astype(np.uint64)
        torch.cuda.synchronize()
        self.reqs = [self.request(i, 0) for i in range(n)]

    def request(self, i, which):
        import paper_1305_3345_gb300 as kg
        r = np.zeros(1, dtype=kg.request_dtype())[0]
        m, k = int(self.modes[i]), int(self.kidx[i])
        r["mode"] = m
        r["dir"] = int(self.dirs[i]) if m in (w.MODE_XTS, w.MODE_ECB) else 0
        r["key"] = self.hx[k] if m == w.MODE_XTS else self.hs[k]
        r["src"] = self.src.data_ptr() + int(self.offsets[i])
        r["dst"] = self.out[which].data_ptr() + int(self.offsets[i])
        r["len"] = int(self.sizes[i])
        r["unit_size"] = 4096
        r["sector"] = int(self.sectors[i])
        r["ivs"] = self.ivs.data_ptr() + 16 * int(self.iv_off[i]) if m in (w.MODE_CBC_DEC, w.MODE_CBC_ENC) else 0
        return r

    def array(self, which=0):
        import paper_1305_3345_gb300 as kg
        a = np.zeros(len(self.reqs), dtype=kg.request_dtype())
        for i in range(len(self.reqs)):
            a[i] = self.request(i, which)
        return a

    def got(self, i, which=0):
        a, b = int(self.offsets[i]), int(self.offsets[i] + self.sizes[i])
        return self.out[which][a:b].cpu().numpy()

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

    def close(self):
        for h in self.hx + self.hs:
            self.ctx.delkey(h)


def submit_retry(ctx, req, timeout_s=10.0):
    import paper_1305_3345_gb300 as kg
    t0 = time.time()
    while True:
        try:
            return ctx.serve_submit(req)
        except kg.KgpuError as e:
            if e.code != "EBUSY" or time.time() - t0 > timeout_s:
                raise
            time.sleep(0.0001)


def test_serve_one_by_one_vs_oracle(ctx):
    t = Traffic(ctx, seed=71, n=40, lo=4096, hi=256 << 10, nkeys=8)
    ctx.serve_start()
    try:
        for i, r in enumerate(t.reqs):
            tk = ctx.serve_submit(r)
            rc, st, stamps = ctx.serve_poll(tk, 10_000_000_000)
            assert rc == 0 and st == 0
            assert stamps[1] >= stamps[0] > 0
            assert np.array_equal(t.got(i), t.expected(i)), (i, int(t.modes[i]))
    finally:
        assert ctx.serve_stop(5_000_000_000) == 0
    t.close()


def test_serve_same_alone_and_in_the_mix(ctx):
    """Continuous batching: 200 requests submitted back to back run concurrently
    on the device; each result equals the oracle and its result when it is the
    only request in flight."""
    t = Traffic(ctx, seed=73, n=200, lo=4096, hi=1 << 20, nkeys=32)
    alone = t.array(which=1)
    ctx.serve_start()
    try:
        tickets = [submit_retry(ctx, r) for r in t.reqs]
        for tk in tickets:
            rc, st, _ = ctx.serve_poll(tk, 20_000_000_000)
            assert rc == 0 and st == 0
        for i in range(len(t.reqs)):
            tk = ctx.serve_submit(alone[i])
            rc, st, _ = ctx.serve_poll(tk, 10_000_000_000)
            assert rc == 0 and st == 0
        stats = ctx.serve_stats()
    finally:
        assert ctx.serve_stop(5_000_000_000) == 0
    assert stats["completed"] >= 2 * len(t.reqs) - 1
    for i in range(len(t.reqs)):
        mixed = t.got(i, 0)
        assert np.array_equal(mixed, t.got(i, 1)), i
        assert np.array_equal(mixed, t.expected(i)), (i, int(t.modes[i]))
    t.close()


def test_serve_admission_and_ring_limits(ctx):
    import paper_1305_3345_gb300 as kg
    t = Traffic(ctx, seed=79, n=64, lo=64 << 10, hi=256 << 10, nkeys=4)
    ctx.serve_start(ring_slots=8, admit_bytes=256 << 10)
    try:
        tickets, refused = [], 0
        for r in t.reqs:
            while True:
                try:
                    tickets.append(ctx.serve_submit(r))
                    break
                except kg.KgpuError as e:
                    assert e.code == "EBUSY"
                    refused += 1
                    ctx.serve_poll(tickets[-1], 1_000_000)   # let the oldest finish
        for tk in tickets:
            assert ctx.serve_poll(tk, 10_000_000_000)[0] == 0
        stats = ctx.serve_stats()
        assert stats["inflight_bytes"] == 0
    finally:
        assert ctx.serve_stop(5_000_000_000) == 0
    assert refused > 0 and stats["busy_refusals"] == refused
    for i in range(len(t.reqs)):
        assert np.array_equal(t.got(i), t.expected(i)), i
    t.close()


def test_serve_idle_exit_and_relaunch(ctx):
    t = Traffic(ctx, seed=83, n=6, lo=4096, hi=65536, nkeys=2)
    ctx.serve_start(idle_timeout_ns=30_000_000, lifetime_ns=5_000_000_000)
    try:
        tk = ctx.serve_submit(t.reqs[0])
        assert ctx.serve_poll(tk, 10_000_000_000)[0] == 0
        time.sleep(0.4)                          # longer than the idle limit
        stats = ctx.serve_stats()
        assert stats["running"] == 0 and stats["last_exit"] == 2   # idle exit
        for r in t.reqs[1:]:
            tk = ctx.serve_submit(r)              # relaunches the kernel
            assert ctx.serve_poll(tk, 10_000_000_000)[0] == 0
        assert ctx.serve_stats()["launches"] >= 2
    finally:
        assert ctx.serve_stop(5_000_000_000) == 0
    for i in range(len(t.reqs)):
        assert np.array_equal(t.got(i), t.expected(i))
    t.close()


def test_serve_lifetime_bound_relaunches_transparently(ctx):
    t = Traffic(ctx, seed=89, n=120, lo=4096, hi=128 << 10, nkeys=4)
    ctx.serve_start(idle_timeout_ns=2_000_000_000, lifetime_ns=20_000_000)
    try:
        for r in t.reqs:
            tk = ctx.serve_submit(r)
            assert ctx.serve_poll(tk, 10_000_000_000)[0] == 0
            time.sleep(0.001)
        assert ctx.serve_stats()["launches"] >= 2
    finally:
        assert ctx.serve_stop(5_000_000_000) == 0
    for i in range(len(t.reqs)):
        assert np.array_equal(t.got(i), t.expected(i)), i
    t.close()


def test_serve_concurrent_submitters(ctx):
    t = Traffic(ctx, seed=97, n=120, lo=4096, hi=128 << 10, nkeys=8)
    ctx.serve_start()
    errors = []

    def worker(idx):
        try:
            for i in idx:
                tk = submit_retry(ctx, t.reqs[i])
                rc, st, _ = ctx.serve_poll(tk, 10_000_000_000)
                assert rc == 0 and st == 0
        except Exception as e:  # surfaced below
            errors.append(e)

    ths = [threading.Thread(target=worker, args=(range(k, len(t.reqs), 4),)) for k in range(4)]
    try:
        for th in ths:
            th.start()
        for th in ths:
            th.join()
    finally:
        assert ctx.serve_stop(5_000_000_000) == 0
    assert not errors, errors
    for i in range(len(t.reqs)):
        assert np.array_equal(t.got(i), t.expected(i)), i
    t.close()


def test_replay_serve_and_launches(ctx):
    """Open-loop Poisson replay (the serving workload's shape, scaled down):
    both dispatch forms complete every request with identical bytes."""
    n = 3000
    t = Traffic(ctx, seed=5, n=n, lo=4096, hi=1 << 20, nkeys=64)
    arr = (w.poisson_arrivals(5, n, 100_000.0) * 1e9).astype(np.uint64)
    reqs0 = t.array(0)
    reqs1 = t.array(1)
    ctx.serve_start()
    try:
        rc, lat, wall = ctx.replay_serve(reqs0, arr)
    finally:
        assert ctx.serve_stop(5_000_000_000) == 0
    assert rc == 0 and np.all(lat < np.uint64(10**10)) and wall > 0
    rc, lat2, wall2 = ctx.replay_launches(reqs1, arr, nstreams=8)
    assert rc == 0 and np.all(lat2 < np.uint64(10**10))
    import torch
    torch.cuda.synchronize()
    assert torch.equal(t.out[0], t.out[1])
    for i in list(range(0, n, 97)) + [n - 1]:
        assert np.array_equal(t.got(i), t.expected(i)), i
    t.close()


def test_serve_rejects_bad_requests(ctx):
    import paper_1305_3345_gb300 as kg
    t = Traffic(ctx, seed=101, n=2, lo=4096, hi=8192, nkeys=1)
    ctx.serve_start()
    try:
        r = t.reqs[0].copy()
        r["len"] = 0
        with pytest.raises(kg.KgpuError):
            ctx.serve_submit(r)
        r = t.reqs[0].copy()
        r["key"] = 4000
        with pytest.raises(kg.KgpuError):
            ctx.serve_submit(r)
        with pytest.raises(kg.KgpuError):
            ctx.serve_start()            # already running
        with pytest.raises(kg.KgpuError):
            ctx.serve_poll(10**9, 0)      # never issued
    finally:
        assert ctx.serve_stop(5_000_000_000) == 0
    t.close()


def test_serve_submit_many_bursts(ctx):
    """A burst published with one head update: every result equals the oracle;
    with a small ring the accepted prefix runs and the rest is retried."""
    t = Traffic(ctx, seed=79, n=60, lo=4096, hi=128 << 10, nkeys=8)
    ctx.serve_start(ring_slots=16)
    try:
        arr = t.array()
        tickets = []
        k = 0
        while k < len(arr):
            rc, tk = ctx.serve_submit_many(arr[k:])
            assert rc in (0, -16)
            tickets += list(tk)
            k += len(tk)
            if rc == -16 and len(tk) == 0:
                time.sleep(0.0005)
        assert len(tickets) == len(arr)
        for tk in tickets:
            rc, st, _ = ctx.serve_poll(int(tk), 10_000_000_000)
            assert rc == 0 and st == 0
    finally:
        assert ctx.serve_stop(5_000_000_000) == 0
    for i in range(len(t.reqs)):
        assert np.array_equal(t.got(i), t.expected(i)), (i, int(t.modes[i]))
    t.close()


def test_serve_stamps_survive_slot_reuse(ctx):
    """An 8-slot ring cycles each slot many times before the first tickets are
    polled: every poll still returns status 0 and either the request's own
    device stamps (start > 0, done >= start) or (0, 0) once its slot has
    retired a later request -- never another request's or half-cleared
    stamps -- and the last ring's worth of tickets keep theirs.  The trace
    replay on the same small ring gives the same guarantee for its detail."""
    t = Traffic(ctx, seed=79, n=96, lo=4096, hi=64 << 10, nkeys=4)
    ctx.serve_start(ring_slots=8)
    try:
        tickets, k = [], 0
        while k < len(t.reqs):
            rc, tk = ctx.serve_submit_many(t.array(which=0)[k:])
            tickets += [int(x) for x in tk]
            k += len(tk)
        seen = []
        for tk in tickets:
            rc, st, stamps = ctx.serve_poll(tk, 10_000_000_000)
            assert rc == 0 and st == 0
            s0, s1 = int(stamps[0]), int(stamps[1])
            assert (s0, s1) == (0, 0) or s1 >= s0 > 0, (tk, s0, s1)
            seen.append((s0, s1))
        assert all(s[0] > 0 for s in seen[-8:])
        arr = np.cumsum(np.full(len(t.reqs), 200, dtype=np.uint64))   # 5M requests/s: overload
        detail = np.zeros(3 * len(t.reqs), dtype=np.uint64)
        rc, lat, wall = ctx.replay_serve(t.array(which=1), arr, 20_000_000_000, detail=detail)
        assert rc == 0
        d = detail.reshape(-1, 3).astype(np.int64)
        ok = ((d[:, 1] == 0) & (d[:, 2] == 0)) | ((d[:, 1] > 0) & (d[:, 2] >= d[:, 1]))
        assert ok.all(), d[~ok][:4]
        assert (d[:, 1] > 0).sum() >= 8
    finally:
        assert ctx.serve_stop(5_000_000_000) == 0
    for i in range(len(t.reqs)):
        assert np.array_equal(t.got(i, 0), t.expected(i)), i
        assert np.array_equal(t.got(i, 1), t.expected(i)), i
    t.close()


@pytest.mark.parametrize("bits", [128, 192, 256])
def test_serve_cbc_encrypt_four_lanes_per_page(ctx, bits):
    """While the ring keeps up, CBC encryption of device pages runs four lanes
    to a page (tiles of 8 pages).  Requests published one at a time (never a
    backlog) with pages of 1, 3, 256 and 257 blocks and 1 to 19 pages -- one
    tile, several, ragged last tiles -- and in place: every output equals the
    oracle."""
    import torch
    import paper_1305_3345_gb300 as kg
    key = w.single_key(81 + bits, bits)
    kh = ctx.setkey(key, False)
    cases = [(bpp * 16, npg) for bpp in (1, 3, 256, 257) for npg in (1, 7, 8, 9, 19)]
    total = sum(p * n for p, n in cases)
    data = w.seeded_bytes(81, w.STREAM_DATA, total)
    ivs_np = w.page_ivs(81, sum(n for _, n in cases))
    src = torch.from_numpy(data.copy()).cuda()
    dst = torch.zeros_like(src)
    ivs = torch.from_numpy(ivs_np.reshape(-1).copy()).cuda()
    torch.cuda.synchronize()
    reqs, off, ivo = [], 0, 0
    for i, (page, npg) in enumerate(cases):
        r = np.zeros(1, dtype=kg.request_dtype())[0]
        r["mode"], r["key"], r["len"], r["unit_size"] = w.MODE_CBC_ENC, kh, page * npg, page
        inplace = i % 4 == 3
        r["src"] = (dst if inplace else src).data_ptr() + off
        r["dst"] = dst.data_ptr() + off
        r["ivs"] = ivs.data_ptr() + 16 * ivo
        reqs.append((r, off, page, npg, ivo, inplace))
        off += page * npg
        ivo += npg
    for r, o, page, npg, io, inplace in reqs:   # in-place requests read their own region of dst
        if inplace:
            dst[o:o + page * npg].copy_(src[o:o + page * npg])
    torch.cuda.synchronize()
    ctx.serve_start()
    try:
        for r, *_ in reqs:
            rc, st, _ = ctx.serve_poll(ctx.serve_submit(r), 10_000_000_000)
            assert rc == 0 and st == 0
    finally:
        assert ctx.serve_stop(5_000_000_000) == 0
    got = dst.cpu().numpy()
    for r, o, page, npg, io, inplace in reqs:
        ref = oracle.cbc(key, 0, data[o:o + page * npg], page, ivs_np[io:io + npg])
        assert np.array_equal(got[o:o + page * npg], ref), (page, npg, inplace)
    ctx.delkey(kh)


def test_serve_stop_while_other_threads_poll(ctx):
    """kgpu_serve_stop from one thread while others poll tickets (some of them
    already complete, some never issued yet) and another thread keeps trying
    to submit: the stop drains and frees the ring without a reader left on it,
    every poll returns OK or ENOENT, submissions after the stop began are
    refused, and a second stop in parallel returns once the first is done."""
    import threading
    import time
    import paper_1305_3345_gb300 as kg
    t = Traffic(ctx, seed=83, n=120, lo=4096, hi=256 << 10, nkeys=8)
    ctx.serve_start()
    tickets = [submit_retry(ctx, r) for r in t.reqs[:60]]
    results, errors = [], []
    stop_started = threading.Event()

    def poller(ts):
        try:
            for tk in ts:
                try:
                    rc, st, _ = ctx.serve_poll(tk, 20_000_000_000)
                    results.append((tk, rc, st))
                except kg.KgpuError as e:
                    results.append((tk, e.code, None))
        except Exception as e:  # reported below
            errors.append(repr(e))

    def submitter():
        refused = 0
        for r in t.reqs[60:]:
            try:
                ctx.serve_submit(r)
            except kg.KgpuError as e:
                if e.code not in ("EBUSY", "EINVAL"):
                    errors.append(repr(e))
                refused += e.code == "EINVAL"
            if stop_started.is_set() and refused:
                return

    def stopper(out):
        stop_started.set()
        out.append(ctx.serve_stop(30_000_000_000))

    stops = []
    ths = [threading.Thread(target=poller, args=(tickets[i::3],)) for i in range(3)]
    ths += [threading.Thread(target=submitter)]
    for th in ths:
        th.start()
    time.sleep(0.002)
    s1 = threading.Thread(target=stopper, args=(stops,))
    s2 = threading.Thread(target=stopper, args=(stops,))
    s1.start()
    s2.start()
    for th in ths + [s1, s2]:
        th.join(60)
    assert not errors, errors
    assert sorted(stops) == [0, 0]
    assert all(rc in (0, "ENOENT") for _, rc, _ in results)
    assert all(st == 0 for _, rc, st in results if rc == 0)
    # the ring is gone: a poll of an old ticket is ENOENT, and serving restarts cleanly
    with pytest.raises(kg.KgpuError):
        ctx.serve_poll(tickets[0], 0)
    ctx.serve_start()
    tk = ctx.serve_submit(t.reqs[0])
    assert ctx.serve_poll(tk, 10_000_000_000)[0] == 0
    assert ctx.serve_stop(5_000_000_000) == 0
    t.close()


def test_key_slot_reused_while_the_ring_runs(ctx):
    """Keys deleted and set again while the serving kernel stays resident: each
    round's key takes the slot the previous one left (the table hands out the
    lowest free slot), and every request must be served with the key it names,
    never the schedule a warp kept from the slot's previous key.  Two rounds in
    a row use the same mode and direction, so only the key itself differs."""
    import torch
    import paper_1305_3345_gb300 as kg
    n, size = 64, 16 << 10
    data = w.seeded_bytes(611, w.STREAM_DATA, n * size)
    ivs_np = w.page_ivs(611, n * size // 4096)
    src = torch.from_numpy(data.copy()).cuda()
    ivs = torch.from_numpy(ivs_np.reshape(-1).copy()).cuda()
    dst = torch.zeros_like(src)
    torch.cuda.synchronize()
    ctx.serve_start()
    try:
        slots = set()
        for rnd in range(20):
            xts = (rnd // 2) % 2 == 0
            key = w.xts_key(612 + rnd, 256) if xts else w.single_key(612 + rnd, 128)
            kh = ctx.setkey(key, xts)
            slots.add(kh)
            r = np.zeros(n, dtype=kg.request_dtype())
            r["mode"] = kg.MODE_XTS if xts else kg.MODE_CBC_ENC
            r["key"], r["len"], r["unit_size"] = kh, size, 4096
            r["src"] = src.data_ptr() + size * np.arange(n)
            r["dst"] = dst.data_ptr() + size * np.arange(n)
            r["sector"] = 4 * np.arange(n)
            r["ivs"] = 0 if xts else ivs.data_ptr() + 16 * 4 * np.arange(n)
            rc, _, _ = ctx.replay_serve(r, np.zeros(n, np.uint64))
            assert rc == 0
            ref = oracle.xts(key, 0, data, 4096, 0) if xts else oracle.cbc(key, 0, data, 4096, ivs_np)
            assert np.array_equal(dst.cpu().numpy(), ref), rnd
            ctx.delkey(kh)
        assert len(slots) <= 2   # the same slot (or two) served every round
    finally:
        ctx.serve_stop(10_000_000_000)


def test_pages_rewritten_by_the_host_between_requests(ctx):
    """The same device pages reused for request after request while the ring
    runs, their contents rewritten by a host-to-device copy in between (as page
    buffers are reused): every request must read what the copy wrote, never
    lines an SM kept from the previous request."""
    import torch
    import paper_1305_3345_gb300 as kg
    key = w.xts_key(621, 256)
    kh = ctx.setkey(key, True)
    n, size = 16, 8192
    src = torch.zeros(n * size, dtype=torch.uint8, device="cuda")
    dst = torch.zeros_like(src)
    r = np.zeros(n, dtype=kg.request_dtype())
    r["mode"], r["key"], r["len"], r["unit_size"] = kg.MODE_XTS, kh, size, 4096
    r["src"] = src.data_ptr() + size * np.arange(n)
    r["dst"] = dst.data_ptr() + size * np.arange(n)
    r["sector"] = 2 * np.arange(n)
    torch.cuda.synchronize()
    ctx.serve_start()
    try:
        for rnd in range(20):
            data = w.seeded_bytes(622 + rnd, w.STREAM_DATA, n * size)
            src.copy_(torch.from_numpy(data))     # a copy-engine write, no kernel
            torch.cuda.synchronize()
            rc, _, _ = ctx.replay_serve(r, np.zeros(n, np.uint64))
            assert rc == 0
            assert np.array_equal(dst.cpu().numpy(), oracle.xts(key, 0, data, 4096, 0)), rnd
    finally:
        ctx.serve_stop(10_000_000_000)
        ctx.delkey(kh)
