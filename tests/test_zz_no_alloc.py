"""kgpu_submit_noalloc: the batched entry point for callers that cannot allocate
memory when they call (an OS-level caller on a writeback or reclaim path, or a
deployment whose memory budget is fixed at start-up).  It keeps its scratch in
a fixed array inside the library instead of allocating.

Its output must equal kgpu_submit's byte for byte (the tolerance of every test
here: AES output is exact) and the oracle's, on two calls in a row -- the
second call reuses the scratch the first one left behind -- both with a
synchronisation between the calls and queued back to back on one stream.
Collected last on purpose, so a failure here leaves every other test already
run.
"""
import numpy as np
import pytest

import oracle
import workloads as w

pytestmark = pytest.mark.gpu


def make_batch(ctx, seed, n, hi):
    """n mixed requests (XTS both ways, CBC decrypt/encrypt, ECB; AES-128/256)
    reading one seeded input, each writing two output buffers: one for the
    existing entry point, one for the allocation-free one."""
    import torch
    import paper_1305_3345_gb300 as kg
    mix = w.request_mix(seed, n, 4096, hi, 8)
    modes = np.where(w.uniform01(seed, 97, n) < 0.15, w.MODE_ECB, mix.modes)
    keys = w.mix_key_material(seed, mix)
    hx = [ctx.setkey(k[: 2 * b // 8], True) for k, b in zip(keys, mix.key_bits)]
    hs = [ctx.setkey(k[: b // 8], False) for k, b in zip(keys, mix.key_bits)]
    data = w.seeded_bytes(seed, w.STREAM_DATA, mix.total_bytes)
    src = torch.from_numpy(data.copy()).cuda()
    outs = [torch.zeros_like(src), torch.zeros_like(src)]
    npages = mix.sizes // 4096
    iv_off = np.concatenate([[0], np.cumsum(npages)[:-1]])
    iv_np = w.page_ivs(seed, int(npages.sum()))
    ivs = torch.from_numpy(iv_np.reshape(-1).copy()).cuda()
    reqs = []
    for out in outs:
        r = np.zeros(n, dtype=kg.request_dtype())
        r["mode"] = modes
        r["dir"] = np.where((modes == w.MODE_XTS) | (modes == w.MODE_ECB), mix.dirs, 0)
        r["key"] = np.where(modes == w.MODE_XTS, np.array(hx)[mix.keys], np.array(hs)[mix.keys])
        r["src"] = src.data_ptr() + mix.offsets
        r["dst"] = out.data_ptr() + mix.offsets
        r["len"] = mix.sizes
        r["unit_size"] = 4096
        r["sector"] = mix.offsets // 4096 + 11
        r["ivs"] = np.where((modes == w.MODE_CBC_DEC) | (modes == w.MODE_CBC_ENC), ivs.data_ptr() + 16 * iv_off, 0)
        reqs.append(r)
    torch.cuda.synchronize()
    return dict(reqs=reqs, outs=outs, src=src, ivs=ivs, keys=hx + hs, mix=mix, modes=modes, data=data,
                key_bytes=keys, iv_np=iv_np, iv_off=iv_off)


def oracle_request(b, i):
    """The oracle's output for request i of batch b."""
    mix, m = b["mix"], int(b["modes"][i])
    k = int(mix.keys[i])
    bits = int(mix.key_bits[k])
    a, e = int(mix.offsets[i]), int(mix.offsets[i] + mix.sizes[i])
    x = b["data"][a:e]
    if m == w.MODE_XTS:
        return oracle.xts(b["key_bytes"][k][: 2 * bits // 8], int(mix.dirs[i]), x, 4096, a // 4096 + 11)
    if m == w.MODE_ECB:
        return oracle.ecb(b["key_bytes"][k][: bits // 8], int(mix.dirs[i]), x)
    p0 = int(b["iv_off"][i])
    iv = b["iv_np"][p0:p0 + (e - a) // 4096]
    return oracle.cbc(b["key_bytes"][k][: bits // 8], 0 if m == w.MODE_CBC_ENC else 1, x, 4096, iv)


def check_against_oracle(b, which, sample):
    """Every sampled request of output `which`, for every mode, against the oracle."""
    mix = b["mix"]
    for i in sample:
        a, e = int(mix.offsets[i]), int(mix.offsets[i] + mix.sizes[i])
        assert np.array_equal(b["outs"][which][a:e].cpu().numpy(), oracle_request(b, i)), (i, int(b["modes"][i]))


def sample_each_mode(b, per_mode=3):
    """A few requests of every mode present (first, middle, last of each)."""
    out = []
    for m in (w.MODE_XTS, w.MODE_CBC_DEC, w.MODE_CBC_ENC, w.MODE_ECB):
        idx = np.flatnonzero(b["modes"] == m)
        if idx.size:
            out += sorted({int(idx[0]), int(idx[idx.size // 2]), int(idx[-1])})[:per_mode]
    return out


def run_submit(ctx, b):
    st = np.zeros(len(b["reqs"][0]), np.int32)
    t = ctx.submit(b["reqs"][0], status=st)
    assert ctx.poll(t, -1, st) == 0 and not st.any()


def free_keys(ctx, *batches):
    for b in batches:
        for h in b["keys"]:
            ctx.delkey(h)


def test_noalloc_matches_submit_on_two_calls_in_a_row(ctx):
    import torch
    first = make_batch(ctx, seed=201, n=60, hi=256 << 10)
    second = make_batch(ctx, seed=202, n=300, hi=128 << 10)
    for b in (first, second):
        run_submit(ctx, b)
        st2 = np.full(len(b["reqs"][1]), 5, np.int32)
        ctx.submit_noalloc(b["reqs"][1], status=st2)
        torch.cuda.synchronize()
        assert not st2.any()
        assert torch.equal(b["outs"][0], b["outs"][1])
        assert not torch.equal(b["outs"][1], b["src"])
    # the bytes are the cipher, for every mode (XTS, CBC both ways, ECB)
    for b in (first, second):
        check_against_oracle(b, 1, sample_each_mode(b))
    free_keys(ctx, first, second)


def test_noalloc_back_to_back_on_one_stream(ctx):
    """Two different batches queued on one side stream with no host
    synchronisation between the calls: the second call's descriptor copy and
    counter clear into the shared array must stay in stream order behind the
    first batch."""
    import torch
    first = make_batch(ctx, seed=211, n=120, hi=512 << 10)
    second = make_batch(ctx, seed=212, n=400, hi=64 << 10)
    for b in (first, second):
        run_submit(ctx, b)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    st1 = np.full(120, 5, np.int32)
    st2 = np.full(400, 5, np.int32)
    ctx.submit_noalloc(first["reqs"][1], stream=s, status=st1)
    ctx.submit_noalloc(second["reqs"][1], stream=s, status=st2)
    s.synchronize()
    assert not st1.any() and not st2.any()
    for b in (first, second):
        assert torch.equal(b["outs"][0], b["outs"][1])
        check_against_oracle(b, 1, sample_each_mode(b))
    free_keys(ctx, first, second)


def test_noalloc_host_page_cbc_encryption(ctx):
    """CBC encryption of registered pinned host pages (the staged path of the
    512-thread kernel; most warps run it one lane per page here) beside device
    requests, against the oracle and kgpu_submit."""
    import torch
    import paper_1305_3345_gb300 as kg
    n, page = 40, 4096
    key = w.single_key(213, 256)
    kh = ctx.setkey(key, False)
    sizes = 4096 * (1 + (w.u64(213, 3, n) % 64).astype(np.int64))
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    total = int(sizes.sum())
    data = w.seeded_bytes(213, w.STREAM_DATA, total)
    iv_np = w.page_ivs(213, total // page)
    hsrc = torch.from_numpy(data.copy()).pin_memory()
    hdst = [torch.zeros(total, dtype=torch.uint8).pin_memory() for _ in range(2)]
    ivs = torch.from_numpy(iv_np.reshape(-1).copy()).cuda()
    for t in [hsrc] + hdst:
        ctx.host_register(t)
    try:
        outs = []
        for j, submit in enumerate((lambda r: ctx.poll(ctx.submit(r), -1), ctx.submit_noalloc)):
            r = np.zeros(n, dtype=kg.request_dtype())
            r["mode"], r["key"], r["len"], r["unit_size"] = kg.MODE_CBC_ENC, kh, sizes, page
            r["src"] = hsrc.data_ptr() + offs
            r["dst"] = hdst[j].data_ptr() + offs
            r["ivs"] = ivs.data_ptr() + 16 * (offs // page)
            r["flags"] = kg.REQ_SRC_HOST | kg.REQ_DST_HOST
            submit(r)
            torch.cuda.synchronize()
            outs.append(hdst[j].numpy().copy())
        ref = oracle.cbc(key, 0, data, page, iv_np)
        assert np.array_equal(outs[1], ref)
        assert np.array_equal(outs[0], outs[1])
    finally:
        for t in [hsrc] + hdst:
            ctx.host_unregister(t)
        ctx.delkey(kh)


def test_noalloc_delkey_waits_for_queued_batch(ctx):
    """A key deleted while a batch that uses it is still queued: the deletion
    waits for the batch, and a key set afterwards (which may take the same
    handle) does not leak into it."""
    import torch
    import paper_1305_3345_gb300 as kg
    key = w.xts_key(214, 256)
    data = w.seeded_bytes(214, w.STREAM_DATA, 64 << 20)
    src = torch.from_numpy(data.copy()).cuda()
    dst = torch.zeros_like(src)
    kh = ctx.setkey(key, True)
    r = np.zeros(1, dtype=kg.request_dtype())
    r["mode"], r["key"], r["src"], r["dst"] = kg.MODE_XTS, kh, src.data_ptr(), dst.data_ptr()
    r["len"], r["unit_size"] = src.numel(), 4096
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        torch.cuda._sleep(200_000_000)   # a bounded spin (~0.1 s) ahead of the batch
    ctx.submit_noalloc(r, stream=s)
    ctx.delkey(kh)
    assert s.query(), "kgpu_aes_delkey returned before the queued batch finished"
    other = ctx.setkey(w.xts_key(215, 256), True)
    torch.cuda.synchronize()
    assert np.array_equal(dst.cpu().numpy(), oracle.xts(key, 0, data, 4096, 0))
    ctx.delkey(other)


def test_noalloc_refuses_a_capturing_stream(ctx):
    import torch
    import paper_1305_3345_gb300 as kg
    b = make_batch(ctx, seed=216, n=4, hi=8192)
    g = torch.cuda.CUDAGraph()
    x = torch.zeros(16, device="cuda")
    refused = None
    with torch.cuda.graph(g):
        try:
            ctx.submit_noalloc(b["reqs"][1])
        except kg.KgpuError as e:
            refused = e.code
        x.add_(1)
    assert refused == "EINVAL"
    torch.cuda.synchronize()
    assert not b["outs"][1].any()          # nothing was queued
    free_keys(ctx, b)


def test_noalloc_rejects_batches_beyond_its_scratch(ctx):
    import torch
    import paper_1305_3345_gb300 as kg
    b = make_batch(ctx, seed=203, n=4, hi=8192)
    big = np.resize(b["reqs"][1], kg.NOALLOC_MAX_REQUESTS + 1)
    with pytest.raises(kg.KgpuError) as e:
        ctx.submit_noalloc(big)
    assert e.value.code == "E2BIG"
    torch.cuda.synchronize()
    assert not b["outs"][1].any()          # nothing was launched
    ctx.submit_noalloc(b["reqs"][1][:0])   # an empty batch is a no-op
    free_keys(ctx, b)
