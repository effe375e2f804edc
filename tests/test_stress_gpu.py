"""Randomized stress of the request paths against the oracle (bit-exact).

Each draw builds a batch of small requests with random modes (XTS both ways,
CBC decrypt/encrypt, ECB both ways), key sizes, data-unit / page sizes
(multiples of 16 from 16 B to 8 KiB), lengths, in-place use and launch shape,
and runs it through kgpu_submit (with a random launch shape), through the
serving ring (published in bursts with kgpu_serve_submit_many onto an 8-slot
ring, so most bursts are cut short by EBUSY) and, for every XTS request,
through the per-call entry point.  Every output must equal the oracle.  The
draws are seeded, so a failure names the seed that reproduces it.
"""
import numpy as np
import pytest

import oracle
import workloads as w

pytestmark = pytest.mark.gpu

MODES = (w.MODE_XTS, w.MODE_CBC_DEC, w.MODE_CBC_ENC, w.MODE_ECB)


def draw(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 40))
    reqs = []
    off = 0
    for _ in range(n):
        mode = int(rng.choice(MODES))
        bits = int(rng.choice([128, 256] if mode == w.MODE_XTS else [128, 192, 256]))
        unit = 16 * int(rng.integers(1, 513))
        units = int(rng.integers(1, 9))
        length = 16 * int(rng.integers(1, 600)) if mode == w.MODE_ECB else unit * units
        reqs.append(dict(mode=mode, bits=bits, unit=unit, len=length, off=off, dir=int(rng.integers(0, 2)),
                         sector=int(rng.integers(0, 2**63)), inplace=bool(rng.integers(0, 4) == 0),
                         key=rng.integers(0, 256, 64, dtype=np.uint8).tobytes()))
        off += (length + 255) // 256 * 256
    return reqs, off, rng


def expected(r, data):
    x = data[r["off"]:r["off"] + r["len"]]
    nb = r["bits"] // 8
    if r["mode"] == w.MODE_XTS:
        return oracle.xts(r["key"][:2 * nb], r["dir"], x, r["unit"], r["sector"])
    if r["mode"] == w.MODE_ECB:
        return oracle.ecb(r["key"][:nb], r["dir"], x)
    return oracle.cbc(r["key"][:nb], 0 if r["mode"] == w.MODE_CBC_ENC else 1, x, r["unit"], r["ivs"])


@pytest.mark.parametrize("seed", range(40))
def test_random_batches_through_every_request_path(ctx, seed):
    import torch
    import paper_1305_3345_gb300 as kg
    reqs, total, rng = draw(1000 + seed)
    data = w.seeded_bytes(1000 + seed, w.STREAM_DATA, total)
    handles = []
    for r in reqs:
        nb = r["bits"] // 8
        if r["mode"] == w.MODE_XTS:
            k = r["key"][:2 * nb]
            if k[:nb] == k[nb:]:
                k = k[:nb] + bytes((b ^ 1) for b in k[nb:])
                r["key"] = k + r["key"][2 * nb:]
            r["h"] = ctx.setkey(k, True)
        else:
            r["h"] = ctx.setkey(r["key"][:nb], False)
        handles.append(r["h"])
        if r["mode"] in (w.MODE_CBC_DEC, w.MODE_CBC_ENC):
            r["ivs"] = rng.integers(0, 256, (r["len"] // r["unit"], 16), dtype=np.uint8)
    ivs_all = np.concatenate([r["ivs"].reshape(-1) for r in reqs if "ivs" in r] + [np.zeros(16, np.uint8)])
    div = torch.from_numpy(ivs_all.copy()).cuda()
    iv_off = 0

    def records(out):
        nonlocal iv_off
        arr = np.zeros(len(reqs), dtype=kg.request_dtype())
        iv_off = 0
        for i, r in enumerate(reqs):
            arr[i]["mode"], arr[i]["key"], arr[i]["len"], arr[i]["unit_size"] = r["mode"], r["h"], r["len"], r["unit"]
            arr[i]["dir"] = r["dir"] if r["mode"] in (w.MODE_XTS, w.MODE_ECB) else 0
            arr[i]["sector"] = r["sector"]
            arr[i]["src"] = out.data_ptr() + r["off"] if r["inplace"] else src.data_ptr() + r["off"]
            arr[i]["dst"] = out.data_ptr() + r["off"]
            if "ivs" in r:
                arr[i]["ivs"] = div.data_ptr() + iv_off
                iv_off += r["ivs"].size
        return arr

    src = torch.from_numpy(data.copy()).cuda()
    outs = {}
    # batched, with a random launch shape
    before = ctx.get_tuning()
    ctx.set_tuning(threads=int(rng.choice([512, 1024])), tile_chunks=int(rng.choice([1, 8, 32, 128])))
    outs["batch"] = src.clone()
    st = np.full(len(reqs), 9, np.int32)
    assert ctx.poll(ctx.submit(records(outs["batch"]), status=st), -1) == 0 and not st.any()
    ctx.set_tuning(**before)
    # serving, published in bursts onto a small ring
    outs["serve"] = src.clone()
    arr = records(outs["serve"])
    torch.cuda.synchronize()
    ctx.serve_start(ring_slots=8)
    try:
        tickets, k = [], 0
        while k < len(arr):
            rc, tk = ctx.serve_submit_many(arr[k:])
            tickets += list(tk)
            k += len(tk)
        for t in tickets:
            rc, code, _ = ctx.serve_poll(int(t), 10_000_000_000)
            assert rc == 0 and code == 0
    finally:
        assert ctx.serve_stop(5_000_000_000) == 0
    # per call (XTS)
    outs["call"] = src.clone()
    for r in reqs:
        if r["mode"] == w.MODE_XTS:
            a, b = r["off"], r["off"] + r["len"]
            s_ = outs["call"][a:b] if r["inplace"] else src[a:b]
            ctx.xts_crypt(r["h"], r["dir"], s_, outs["call"][a:b], r["unit"], r["sector"])
    torch.cuda.synchronize()
    for i, r in enumerate(reqs):
        e = expected(r, data)
        a, b = r["off"], r["off"] + r["len"]
        for name in ("batch", "serve") + (("call",) if r["mode"] == w.MODE_XTS else ()):
            assert np.array_equal(outs[name][a:b].cpu().numpy(), e), (seed, i, name, r["mode"], r["unit"], r["len"])
    for h in handles:
        ctx.delkey(h)


@pytest.mark.parametrize("seed", range(12))
def test_random_batches_over_registered_host_pages(ctx, seed):
    """The same draws with every buffer -- input, output, IVs -- in registered
    pinned host memory and the request flags saying so: the kernels read and
    write the pages over the host link (CBC encryption of pages of whole
    128-byte lines through the staged path).  Batched (512 threads, the kernel
    that stages) and served outputs equal the oracle."""
    import torch
    import paper_1305_3345_gb300 as kg
    reqs, total, rng = draw(2000 + seed)
    data = w.seeded_bytes(2000 + seed, w.STREAM_DATA, total)
    for r in reqs:
        nb = r["bits"] // 8
        if r["mode"] == w.MODE_XTS:
            k = r["key"][:2 * nb]
            if k[:nb] == k[nb:]:
                k = k[:nb] + bytes((b ^ 1) for b in k[nb:])
                r["key"] = k + r["key"][2 * nb:]
            r["h"] = ctx.setkey(k, True)
        else:
            r["h"] = ctx.setkey(r["key"][:nb], False)
        if r["mode"] in (w.MODE_CBC_DEC, w.MODE_CBC_ENC):
            r["ivs"] = rng.integers(0, 256, (r["len"] // r["unit"], 16), dtype=np.uint8)
    ivs_all = np.concatenate([r["ivs"].reshape(-1) for r in reqs if "ivs" in r] + [np.zeros(16, np.uint8)])
    src = torch.from_numpy(data.copy()).pin_memory()
    hiv = torch.from_numpy(ivs_all.copy()).pin_memory()
    outs = {name: torch.from_numpy(data.copy()).pin_memory() for name in ("batch", "serve")}
    bufs = [src, hiv] + list(outs.values())
    for b in bufs:
        ctx.host_register(b)
    flags = kg.REQ_SRC_HOST | kg.REQ_DST_HOST | kg.REQ_IVS_HOST

    def records(out):
        arr = np.zeros(len(reqs), dtype=kg.request_dtype())
        iv_off = 0
        for i, r in enumerate(reqs):
            arr[i]["mode"], arr[i]["key"], arr[i]["len"], arr[i]["unit_size"] = r["mode"], r["h"], r["len"], r["unit"]
            arr[i]["dir"] = r["dir"] if r["mode"] in (w.MODE_XTS, w.MODE_ECB) else 0
            arr[i]["sector"] = r["sector"]
            arr[i]["src"] = out.data_ptr() + r["off"] if r["inplace"] else src.data_ptr() + r["off"]
            arr[i]["dst"] = out.data_ptr() + r["off"]
            arr[i]["flags"] = flags if "ivs" in r else kg.REQ_SRC_HOST | kg.REQ_DST_HOST
            if "ivs" in r:
                arr[i]["ivs"] = hiv.data_ptr() + iv_off
                iv_off += r["ivs"].size
        return arr

    try:
        before = ctx.get_tuning()
        ctx.set_tuning(threads=512, tile_chunks=int(rng.choice([1, 8, 32, 128])))
        st = np.full(len(reqs), 9, np.int32)
        try:
            assert ctx.poll(ctx.submit(records(outs["batch"]), status=st), -1) == 0 and not st.any()
        finally:
            ctx.set_tuning(**before)
        arr = records(outs["serve"])
        ctx.serve_start(ring_slots=8)
        try:
            tickets, k = [], 0
            while k < len(arr):
                rc, tk = ctx.serve_submit_many(arr[k:])
                tickets += list(tk)
                k += len(tk)
            for t in tickets:
                rc, code, _ = ctx.serve_poll(int(t), 10_000_000_000)
                assert rc == 0 and code == 0
        finally:
            assert ctx.serve_stop(5_000_000_000) == 0
        for i, r in enumerate(reqs):
            e = expected(r, data)
            a, b = r["off"], r["off"] + r["len"]
            for name in ("batch", "serve"):
                assert np.array_equal(outs[name][a:b].numpy(), e), (seed, i, name, r["mode"], r["unit"], r["len"])
    finally:
        for b in bufs:
            ctx.host_unregister(b)
        for r in reqs:
            ctx.delkey(r["h"])
