"""kgpu_submit_noalloc: the batched entry point for callers that cannot allocate
memory when they call (an OS-level caller on a writeback or reclaim path, or a
deployment whose memory budget is fixed at start-up).  It keeps its scratch in
a fixed array inside the library instead of allocating.

Its output must equal kgpu_submit's byte for byte (the tolerance of every test
here: AES output is exact), on two calls in a row -- the second call reuses the
scratch the first one left behind.  Collected last on purpose, so a failure
here leaves every other test already run.
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
    ivs = torch.from_numpy(w.page_ivs(seed, int(npages.sum())).reshape(-1).copy()).cuda()
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
                key_bytes=keys)


def run_both(ctx, b):
    import torch
    st = np.zeros(len(b["reqs"][0]), np.int32)
    t = ctx.submit(b["reqs"][0], status=st)
    assert ctx.poll(t, -1, st) == 0 and not st.any()
    st2 = np.full(len(b["reqs"][1]), 5, np.int32)
    ctx.submit_noalloc(b["reqs"][1], status=st2)
    torch.cuda.synchronize()
    assert not st2.any()


def test_noalloc_matches_submit_on_two_calls_in_a_row(ctx):
    import torch
    first = make_batch(ctx, seed=201, n=60, hi=256 << 10)
    second = make_batch(ctx, seed=202, n=300, hi=128 << 10)
    for b in (first, second):
        run_both(ctx, b)
        assert torch.equal(b["outs"][0], b["outs"][1])
        assert not torch.equal(b["outs"][1], b["src"])
    # and the bytes are the cipher: spot-check the second call against the oracle
    mix, modes = second["mix"], second["modes"]
    for i in (0, 7, 150, 299):
        m, k = int(modes[i]), int(mix.keys[i])
        bits = int(mix.key_bits[k])
        a, e = int(mix.offsets[i]), int(mix.offsets[i] + mix.sizes[i])
        x = second["data"][a:e]
        if m == w.MODE_XTS:
            ref = oracle.xts(second["key_bytes"][k][: 2 * bits // 8], int(mix.dirs[i]), x, 4096, a // 4096 + 11)
        elif m == w.MODE_ECB:
            ref = oracle.ecb(second["key_bytes"][k][: bits // 8], int(mix.dirs[i]), x)
        else:
            continue
        assert np.array_equal(second["outs"][1][a:e].cpu().numpy(), ref), i
    for b in (first, second):
        for h in b["keys"]:
            ctx.delkey(h)


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
    for h in b["keys"]:
        ctx.delkey(h)
