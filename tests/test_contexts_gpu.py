"""Two library contexts on one device at the same time.  Each context owns its
key table, so the same handle number names different keys in each; per-call
XTS and batched requests issued on both, interleaved, must each use their own
context's keys (bit-exact against the oracle), and deleting a key in one
context must leave the other's untouched."""
import numpy as np
import pytest

import oracle
import workloads as w
from conftest import to_dev, to_np

pytestmark = pytest.mark.gpu


def test_two_contexts_keep_their_own_keys():
    import torch
    import paper_1305_3345_gb300 as kg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    a, b = kg.Context(0), kg.Context(0)
    try:
        ka, kb = w.xts_key(95, 256), w.xts_key(96, 128)
        ha, hb = a.setkey(ka, True), b.setkey(kb, True)
        assert ha == hb  # handles are per context: the same number, different keys
        data = w.seeded_bytes(95, w.STREAM_DATA, 4096 * 64)
        src = to_dev(data)
        outs = {name: torch.empty_like(src) for name in ("a_call", "b_call", "a_batch", "b_batch")}
        # interleaved per-call launches on the two contexts
        a.xts_crypt(ha, 0, src, outs["a_call"], 4096, 7)
        b.xts_crypt(hb, 0, src, outs["b_call"], 4096, 7)

        def batch(ctx, h, out):
            r = np.zeros(4, dtype=kg.request_dtype())
            r["mode"], r["key"], r["len"], r["unit_size"] = w.MODE_XTS, h, 4096 * 16, 4096
            r["src"] = src.data_ptr() + 4096 * 16 * np.arange(4)
            r["dst"] = out.data_ptr() + 4096 * 16 * np.arange(4)
            r["sector"] = 7 + 16 * np.arange(4)
            return ctx.submit(r)

        ta = batch(a, ha, outs["a_batch"])
        tb = batch(b, hb, outs["b_batch"])
        assert a.poll(ta, -1) == 0 and b.poll(tb, -1) == 0
        torch.cuda.synchronize()
        ref_a, ref_b = oracle.xts(ka, 0, data, 4096, 7), oracle.xts(kb, 0, data, 4096, 7)
        assert np.array_equal(to_np(outs["a_call"]), ref_a)
        assert np.array_equal(to_np(outs["a_batch"]), ref_a)
        assert np.array_equal(to_np(outs["b_call"]), ref_b)
        assert np.array_equal(to_np(outs["b_batch"]), ref_b)
        # deleting context a's key leaves b's key under the same number working
        a.delkey(ha)
        with pytest.raises(kg.KgpuError):
            a.xts_crypt(ha, 0, src, outs["a_call"], 4096, 7)
        b.xts_crypt(hb, 0, src, outs["b_call"], 4096, 7)
        torch.cuda.synchronize()
        assert np.array_equal(to_np(outs["b_call"]), ref_b)
        b.delkey(hb)
    finally:
        a.close()
        b.close()
