"""kgpu_replay_serve_stages: each served request's latency split by stage of the
request path (host publish, dispatcher, tile publication, first tile,
completion, host sighting), with the device's stamps moved to the host clock.

The device stamps are one clock and must be in path order; the host's are
another and must be too; across the two clocks the order may be off by the
offset estimate's error only (bounded here generously, 5 us).  The outputs
must be the cipher's.
"""
import numpy as np
import pytest

import oracle
import workloads as w

pytestmark = pytest.mark.gpu


def test_stage_record_is_ordered_and_outputs_exact(ctx):
    import torch
    import paper_1305_3345_gb300 as kg
    key = w.xts_key(501, 256)
    kh = ctx.setkey(key, True)
    n, size = 400, 8192
    data = w.seeded_bytes(501, w.STREAM_DATA, n * size)
    src = torch.from_numpy(data.copy()).cuda()
    dst = torch.zeros_like(src)
    r = np.zeros(n, dtype=kg.request_dtype())
    r["mode"], r["key"], r["len"], r["unit_size"] = kg.MODE_XTS, kh, size, 4096
    r["src"] = src.data_ptr() + size * np.arange(n)
    r["dst"] = dst.data_ptr() + size * np.arange(n)
    r["sector"] = 2 * np.arange(n)
    # one at a time for the first half, then bursts of 20
    arr = np.concatenate([np.arange(200) * 50_000, 10_000_000 + (np.arange(200) // 20) * 200_000]).astype(np.uint64)
    torch.cuda.synchronize()
    ctx.serve_start()
    try:
        rc, lat, wall, stg, off = ctx.replay_serve_stages(r, arr)
    finally:
        ctx.serve_stop(10_000_000_000)
    assert rc == 0 and off[0] != 0 and off[1] != 0
    assert np.array_equal(dst.cpu().numpy(), oracle.xts(key, 0, data, 4096, 0))
    assert np.array_equal(stg[:, 5], lat.astype(np.int64))
    ok = (stg[:, 1:5] != kg.STAGE_LOST).all(axis=1)
    assert ok.sum() >= n - 5            # a lost stamp needs a slot reused before the host looked
    s = stg[ok]
    assert (s[:, 0] >= 0).all() and (s[:, 0] <= s[:, 5]).all()           # host clock
    assert (np.diff(s[:, 1:5], axis=1) >= 0).all()                        # device clock
    slack = 5_000
    assert (s[:, 1] >= s[:, 0] - slack).all() and (s[:, 4] <= s[:, 5] + slack).all()
    ctx.delkey(kh)
