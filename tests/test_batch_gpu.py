"""Batched submission: many uneven requests with mixed keys and modes in one
persistent-kernel launch, each checked bit-exact against the CPU oracle, and
each identical to its result when submitted alone."""
import numpy as np
import pytest

import oracle
import workloads as w

pytestmark = pytest.mark.gpu


class Batch:
    """A seeded mixed batch packed into one input and one output buffer."""

    def __init__(self, ctx, seed, n, lo, hi, nkeys, unit=4096, modes=(0.4, 0.2, 0.2), ecb=0.2,
                 in_place_every=0):
        import torch
        import paper_1305_3345_gb300 as kg
        self.ctx = ctx
        mix = w.request_mix(seed, n, lo, hi, nkeys, mode_split=modes)
        u = w.uniform01(seed, 99, n)
        self.modes = np.where(u < ecb, w.MODE_ECB, mix.modes)
        self.dirs = mix.dirs
        self.sizes = mix.sizes
        self.unit = unit
        self.keys = w.mix_key_material(seed, mix)
        self.key_bits = mix.key_bits
        self.kidx = mix.keys
        self.hx = [ctx.setkey(k[: 2 * b // 8], True) for k, b in zip(self.keys, self.key_bits)]
        self.hs = [ctx.setkey(k[: b // 8], False) for k, b in zip(self.keys, self.key_bits)]
        self.offsets = mix.offsets
        total = int(self.sizes.sum())
        self.data = w.seeded_bytes(seed, w.STREAM_DATA, total)
        self.src = torch.from_numpy(self.data.copy()).cuda()
        self.dst = torch.zeros_like(self.src)
        npages = self.sizes // unit
        self.iv_off = np.concatenate([[0], np.cumsum(npages)[:-1]])
        self.ivs_np = w.page_ivs(seed, int(npages.sum()))
        self.ivs = torch.from_numpy(self.ivs_np.reshape(-1).copy()).cuda()
        self.sectors = (w.u64(seed, 7, n) % (1 << 40)).astype(np.uint64)
        r = np.zeros(n, dtype=kg.request_dtype())
        self.in_place = np.zeros(n, bool)
        if in_place_every:
            self.in_place[::in_place_every] = True
        for i in range(n):
            m = int(self.modes[i])
            k = int(self.kidx[i])
            r[i]["mode"] = m
            r[i]["dir"] = int(self.dirs[i]) if m in (w.MODE_XTS, w.MODE_ECB) else 0
            r[i]["key"] = self.hx[k] if m == w.MODE_XTS else self.hs[k]
            r[i]["src"] = self.src.data_ptr() + int(self.offsets[i])
            r[i]["dst"] = (self.src if self.in_place[i] else self.dst).data_ptr() + int(self.offsets[i])
            r[i]["len"] = int(self.sizes[i])
            r[i]["unit_size"] = unit
            r[i]["sector"] = int(self.sectors[i])
            r[i]["ivs"] = self.ivs.data_ptr() + 16 * int(self.iv_off[i]) if m in (w.MODE_CBC_DEC, w.MODE_CBC_ENC) else 0
        self.reqs = r

    def expected(self, i):
        m, k = int(self.modes[i]), int(self.kidx[i])
        bits = int(self.key_bits[k])
        a, b = int(self.offsets[i]), int(self.offsets[i] + self.sizes[i])
        x = self.data[a:b]
        if m == w.MODE_XTS:
            return oracle.xts(self.keys[k][: 2 * bits // 8], int(self.dirs[i]), x, self.unit, int(self.sectors[i]))
        if m == w.MODE_ECB:
            return oracle.ecb(self.keys[k][: bits // 8], int(self.dirs[i]), x)
        p0 = int(self.iv_off[i])
        ivs = self.ivs_np[p0:p0 + int(self.sizes[i]) // self.unit]
        return oracle.cbc(self.keys[k][: bits // 8], 0 if m == w.MODE_CBC_ENC else 1, x, self.unit, ivs)

    def got(self, i):
        a, b = int(self.offsets[i]), int(self.offsets[i] + self.sizes[i])
        buf = self.src if self.in_place[i] else self.dst
        return buf[a:b].cpu().numpy()

    def close(self):
        for h in self.hx + self.hs:
            self.ctx.delkey(h)


def run(ctx, reqs):
    st = np.full(len(reqs), 7, np.int32)
    t = ctx.submit(reqs, status=st)
    assert ctx.poll(t, -1, st) == 0
    assert np.all(st == 0), st
    return t


def test_mixed_batch_vs_oracle(ctx):
    b = Batch(ctx, seed=41, n=300, lo=4096, hi=256 << 10, nkeys=16, in_place_every=7)
    run(ctx, b.reqs)
    for i in range(len(b.reqs)):
        assert np.array_equal(b.got(i), b.expected(i)), (i, int(b.modes[i]), int(b.sizes[i]))
    b.close()


@pytest.mark.parametrize("unit", [512, 16, 48, 4112])
def test_mixed_batch_unit_sizes(ctx, unit):
    b = Batch(ctx, seed=43 + unit, n=80, lo=4096, hi=64 << 10, nkeys=6, unit=unit)
    # sizes are page multiples of 4096; make them unit multiples
    sizes = (b.sizes // unit) * unit
    b.reqs["len"] = sizes
    b.sizes = sizes
    npages = sizes // unit
    b.iv_off = np.concatenate([[0], np.cumsum(npages)[:-1]])
    b.ivs_np = w.page_ivs(43 + unit, int(npages.sum()))
    import torch
    b.ivs = torch.from_numpy(b.ivs_np.reshape(-1).copy()).cuda()
    for i in range(len(b.reqs)):
        if b.modes[i] in (w.MODE_CBC_DEC, w.MODE_CBC_ENC):
            b.reqs[i]["ivs"] = b.ivs.data_ptr() + 16 * int(b.iv_off[i])
    run(ctx, b.reqs)
    for i in range(len(b.reqs)):
        assert np.array_equal(b.got(i), b.expected(i)), (unit, i, int(b.modes[i]))
    b.close()


def test_cbc_encryption_batch_oversubscribes_the_staging_pool(ctx):
    """A batch of CBC encryption only, of 512-byte pages, with several thousand
    32-page tiles: every warp of the 512-thread kernel runs such a tile at
    once, so some stage through the shared pool's areas and the others find
    none free and run without one.  Every request is the oracle's."""
    b = Batch(ctx, 41, 600, 64 << 10, 256 << 10, 8, unit=512, modes=(0.0, 0.0, 1.0), ecb=0.0)
    ctx.set_tuning(512, 0, 0)  # the variant with the pool
    try:
        assert int((b.sizes // 512).sum()) // 32 > 152 * 16   # more tiles than warps
        run(ctx, b.reqs)
        for i in range(len(b.reqs)):
            assert np.array_equal(b.got(i), b.expected(i)), i
    finally:
        ctx.set_tuning(0, 0, 0)
        b.close()


@pytest.mark.parametrize("threads,tile", [(512, 1), (1024, 8), (512, 128), (1024, 1024)])
def test_tuning_shapes_give_same_bytes(ctx, threads, tile):
    b = Batch(ctx, seed=47, n=60, lo=4096, hi=512 << 10, nkeys=8)
    ctx.set_tuning(threads, tile, 0)
    try:
        run(ctx, b.reqs)
        for i in range(len(b.reqs)):
            assert np.array_equal(b.got(i), b.expected(i)), (threads, tile, i)
    finally:
        ctx.set_tuning(0, 0, 0)
        b.close()


def test_each_request_same_alone_and_in_the_mix(ctx):
    b = Batch(ctx, seed=53, n=120, lo=4096, hi=128 << 10, nkeys=8)
    run(ctx, b.reqs)
    mixed = [b.got(i) for i in range(len(b.reqs))]
    b.dst.zero_()
    for i in range(0, len(b.reqs), 3):
        run(ctx, b.reqs[i:i + 1].copy())
        assert np.array_equal(b.got(i), mixed[i]), i
    b.close()


def test_batch_validation_and_status(ctx):
    import torch
    import paper_1305_3345_gb300 as kg
    b = Batch(ctx, seed=59, n=10, lo=4096, hi=16384, nkeys=2)
    bad = b.reqs.copy()
    bad[3]["len"] = 4000                      # not whole units
    bad[5]["key"] = 9999                      # unknown key
    bad[7]["src"] = bad[7]["src"] + 8         # misaligned
    st = np.zeros(len(bad), np.int32)
    with pytest.raises(kg.KgpuError) as e:
        ctx.submit(bad, status=st)
    assert e.value.rc in (-22, -2)
    assert st[3] == -22 and st[5] == -2 and st[7] == -22
    assert np.count_nonzero(st) == 3
    # wrong key type: an XTS request given a single key
    bad = b.reqs.copy()
    i = int(np.argmax(b.modes == w.MODE_XTS)) if np.any(b.modes == w.MODE_XTS) else None
    if i is not None:
        bad[i]["key"] = b.hs[int(b.kidx[i])]
        with pytest.raises(kg.KgpuError):
            ctx.submit(bad)
    # empty batch: a ticket that is already complete
    t = ctx.submit(b.reqs[:0].copy())
    assert ctx.poll(t, 0) == 0
    torch.cuda.synchronize()
    b.close()


def test_ticket_rotation(ctx):
    import paper_1305_3345_gb300 as kg
    b = Batch(ctx, seed=61, n=20, lo=4096, hi=65536, nkeys=4)
    tickets = [ctx.submit(b.reqs) for _ in range(6)]
    # the last four hold the slots; the first two were complete when their
    # slots were reused, and still poll as complete with every status 0
    assert ctx.poll(tickets[-1], -1) == 0
    for t in tickets[-4:]:
        assert ctx.poll(t, 0) == 0
    for t in tickets[:2]:
        st = np.full(len(b.reqs), 7, np.int32)
        assert ctx.poll(t, 0, status=st) == 0 and not st.any()
        rc, done = ctx.poll_each(t, len(b.reqs))
        assert rc == 0 and not done.any()          # complete, times not kept
    with pytest.raises(kg.KgpuError):
        ctx.poll(tickets[-1] + 1000, 0)              # never issued
    for i in range(len(b.reqs)):
        assert np.array_equal(b.got(i), b.expected(i))
    b.close()


def test_autotune_picks_a_valid_shape(ctx):
    b = Batch(ctx, seed=67, n=200, lo=4096, hi=1 << 20, nkeys=16)
    best, ms = ctx.autotune(b.reqs, iters=2)
    assert best["threads"] in (512, 1024) and best["tile_chunks"] >= 1 and ms > 0
    assert ctx.get_tuning() == best
    b.dst.zero_()
    run(ctx, b.reqs)
    for i in range(0, len(b.reqs), 5):
        assert np.array_equal(b.got(i), b.expected(i))
    ctx.set_tuning(0, 0, 0)
    b.close()


def test_batched_workload_full_shape_sampled(ctx):
    """The batched workload's full shape: 10,000 requests, sizes log-uniform in
    4 KiB..8 MiB (page multiples), 256 keys (AES-128 and AES-256), modes 50% XTS /
    25% CBC-decrypt / 25% CBC-encrypt, in ONE submission.  Inputs are windows of
    one seeded 1 GiB buffer; outputs are disjoint.  Sampled requests are checked
    against the oracle."""
    import torch
    import paper_1305_3345_gb300 as kg
    n = 10000
    mix = w.request_mix(4, n, 4096, 8 << 20, 256)
    keys = w.mix_key_material(4, mix)
    hx = [ctx.setkey(k[: 2 * b // 8], True) for k, b in zip(keys, mix.key_bits)]
    hs = [ctx.setkey(k[: b // 8], False) for k, b in zip(keys, mix.key_bits)]
    src_n = 1 << 30
    src = torch.from_numpy(w.seeded_bytes(4, w.STREAM_DATA, src_n)).cuda()
    total = mix.total_bytes
    dst = torch.empty(total, dtype=torch.uint8, device="cuda")
    npages = mix.sizes // 4096
    ivs_np = w.page_ivs(4, int(npages.sum()))
    ivs = torch.from_numpy(ivs_np.reshape(-1).copy()).cuda()
    iv_off = np.concatenate([[0], np.cumsum(npages)[:-1]])
    src_off = (w.u64(4, 8, n) % ((src_n - (8 << 20)) // 4096)).astype(np.int64) * 4096
    r = np.zeros(n, dtype=kg.request_dtype())
    r["mode"] = mix.modes
    r["dir"] = np.where(mix.modes == w.MODE_XTS, mix.dirs, 0)
    r["key"] = np.where(mix.modes == w.MODE_XTS, np.array(hx)[mix.keys], np.array(hs)[mix.keys])
    r["src"] = src.data_ptr() + src_off
    r["dst"] = dst.data_ptr() + mix.offsets
    r["len"] = mix.sizes
    r["unit_size"] = 4096
    r["sector"] = mix.offsets // 4096
    r["ivs"] = np.where(mix.modes == w.MODE_XTS, 0, ivs.data_ptr() + 16 * iv_off)
    run(ctx, r)
    rng = np.random.default_rng(4)
    for i in sorted(set(rng.integers(0, n, 40).tolist()) | {0, n - 1}):
        m, k = int(mix.modes[i]), int(mix.keys[i])
        bits = int(mix.key_bits[k])
        x = src[int(src_off[i]): int(src_off[i]) + int(mix.sizes[i])].cpu().numpy()
        if m == w.MODE_XTS:
            ref = oracle.xts(keys[k][: 2 * bits // 8], int(mix.dirs[i]), x, 4096, int(mix.offsets[i] // 4096))
        else:
            p0 = int(iv_off[i])
            ref = oracle.cbc(keys[k][: bits // 8], 0 if m == w.MODE_CBC_ENC else 1, x, 4096,
                             ivs_np[p0:p0 + int(npages[i])])
        got = dst[int(mix.offsets[i]): int(mix.offsets[i]) + int(mix.sizes[i])].cpu().numpy()
        assert np.array_equal(got, ref), (i, m, int(mix.sizes[i]))
    for h in hx + hs:
        ctx.delkey(h)
    del src, dst, ivs
    torch.cuda.empty_cache()


def test_poll_each_reports_every_request(ctx):
    """Per-request completion words: every request of a batch is seen complete,
    no earlier than the submission and no later than the batch, with the same
    bytes as a batch waited on as a whole; a zero-length request is complete at
    once."""
    import time
    import torch
    import paper_1305_3345_gb300 as kg
    mix = w.request_mix(61, 120, 4096, 2 << 20, 8)
    keys = w.mix_key_material(61, mix)
    hx = [ctx.setkey(k[: 2 * b // 8], True) for k, b in zip(keys, mix.key_bits)]
    hs = [ctx.setkey(k[: b // 8], False) for k, b in zip(keys, mix.key_bits)]
    src = torch.from_numpy(w.seeded_bytes(61, w.STREAM_DATA, mix.total_bytes)).cuda()
    outs = [torch.zeros_like(src), torch.zeros_like(src)]
    npages = mix.sizes // 4096
    ivs = torch.from_numpy(w.page_ivs(61, int(npages.sum())).reshape(-1).copy()).cuda()
    iv_off = np.concatenate([[0], np.cumsum(npages)[:-1]])
    arrays = []
    for out in outs:
        r = np.zeros(len(mix.sizes), dtype=kg.request_dtype())
        cbc = (mix.modes == w.MODE_CBC_DEC) | (mix.modes == w.MODE_CBC_ENC)
        r["mode"], r["dir"] = mix.modes, np.where(cbc, 0, mix.dirs)
        r["key"] = np.where(mix.modes == w.MODE_XTS, np.array(hx)[mix.keys], np.array(hs)[mix.keys])
        r["src"], r["dst"] = src.data_ptr() + mix.offsets, out.data_ptr() + mix.offsets
        r["len"], r["unit_size"], r["sector"] = mix.sizes, 4096, mix.offsets // 4096
        r["ivs"] = np.where(cbc, ivs.data_ptr() + 16 * iv_off, 0)
        r["len"][5] = 0                      # one empty request
        arrays.append(r)
    torch.cuda.synchronize()
    assert ctx.poll(ctx.submit(arrays[0]), -1) == 0
    st = np.full(len(mix.sizes), 9, np.int32)
    t0 = time.monotonic_ns()
    t = ctx.submit(arrays[1])
    rc, done = ctx.poll_each(t, len(mix.sizes), status=st)
    t1 = time.monotonic_ns()
    assert rc == 0 and not st.any()
    assert (done >= t0).all() and (done <= t1).all()
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[1])
    assert ctx.poll(t, 0) == 0               # the ticket stays valid afterwards
    for h in hx + hs:
        ctx.delkey(h)


def test_concurrent_submitters_share_the_slots(ctx):
    """Four host threads submit and wait on batches through one context at the
    same time (they share the four rotating staging slots, and some wait
    request by request); every output equals the oracle's."""
    import threading
    import torch
    import paper_1305_3345_gb300 as kg
    key = w.xts_key(71, 256)
    kh = ctx.setkey(key, True)
    nthreads, rounds, per = 4, 6, 16
    data = w.seeded_bytes(71, w.STREAM_DATA, nthreads * per * 8192)
    src = torch.from_numpy(data.copy()).cuda()
    outs = [torch.zeros_like(src) for _ in range(nthreads)]
    torch.cuda.synchronize()
    errors = []

    def worker(t):
        try:
            for k in range(rounds):
                r = np.zeros(per, dtype=kg.request_dtype())
                base = t * per * 8192
                r["mode"], r["key"], r["len"], r["unit_size"] = w.MODE_XTS, kh, 8192, 4096
                r["src"] = src.data_ptr() + base + 8192 * np.arange(per)
                r["dst"] = outs[t].data_ptr() + base + 8192 * np.arange(per)
                r["sector"] = (base + 8192 * np.arange(per)) // 4096
                r["dir"] = k % 2                   # encrypt, then decrypt back, ...
                if k % 2 == 0:
                    r["src"] = src.data_ptr() + base + 8192 * np.arange(per)
                else:
                    r["src"] = r["dst"]            # in place on the previous result
                while True:
                    try:
                        tk = ctx.submit(r)
                        break
                    except kg.KgpuError as e:      # the slot is held by a poll_each
                        if e.code != "EBUSY":
                            raise
                if t % 2:
                    rc, _ = ctx.poll_each(tk, per)
                else:
                    rc = ctx.poll(tk, -1)
                assert rc == 0
        except Exception as e:  # reported below
            errors.append(repr(e))

    ths = [threading.Thread(target=worker, args=(t,)) for t in range(nthreads)]
    for th in ths:
        th.start()
    for th in ths:
        th.join(120)
    assert not errors, errors
    torch.cuda.synchronize()
    # an even number of rounds: encrypt/decrypt pairs leave every output equal to the input
    for t in range(nthreads):
        a, b = t * per * 8192, (t + 1) * per * 8192
        assert torch.equal(outs[t][a:b], src[a:b]), t
    # and one encryption equals the oracle
    r = np.zeros(1, dtype=kg.request_dtype())
    r["mode"], r["key"], r["len"], r["unit_size"] = w.MODE_XTS, kh, 8192, 4096
    r["src"], r["dst"], r["sector"] = src.data_ptr(), outs[0].data_ptr(), 0
    assert ctx.poll(ctx.submit(r), -1) == 0
    assert np.array_equal(outs[0][:8192].cpu().numpy(), oracle.xts(key, 0, data[:8192], 4096, 0))
    ctx.delkey(kh)
