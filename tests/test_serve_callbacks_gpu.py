"""Completion callbacks of served requests (kgpu_serve_submit_cb): the paper's
service request may carry a callback, and its caller blocks until that has run
instead of busy-waiting on the response queue (section 3.2).

Every callback must run exactly once, on the library's completion thread, after
the request's output is in place (checked against the oracle), including
requests that a callback submits itself; a stop runs every callback still
waiting before it returns; stop and destroy are refused from a callback.
"""
import threading

import numpy as np
import pytest

import oracle
import workloads as w

pytestmark = pytest.mark.gpu


class Pages:
    """n requests of 4..64 KiB over one seeded buffer: XTS-256, CBC-128
    encryption and ECB-128 encryption in turn, each with its own key."""

    def __init__(self, ctx, seed, n):
        import torch
        import paper_1305_3345_gb300 as kg
        self.ctx, self.n = ctx, n
        self.sizes = 4096 * (1 + (w.u64(seed, 1, n) % 16)).astype(np.int64)
        self.offs = np.concatenate([[0], np.cumsum(self.sizes)[:-1]])
        total = int(self.sizes.sum())
        self.data = w.seeded_bytes(seed, w.STREAM_DATA, total)
        self.ivs_np = w.page_ivs(seed, total // 4096)
        self.kx = w.xts_key(seed, 256)
        self.ks = w.single_key(seed + 1, 128)
        self.hx = ctx.setkey(self.kx, True)
        self.hs = ctx.setkey(self.ks, False)
        self.src = torch.from_numpy(self.data.copy()).cuda()
        self.dst = torch.zeros_like(self.src)
        self.ivs = torch.from_numpy(self.ivs_np.reshape(-1).copy()).cuda()
        torch.cuda.synchronize()
        self.modes = [kg.MODE_XTS, kg.MODE_CBC_ENC, kg.MODE_ECB]

    def request(self, i):
        import paper_1305_3345_gb300 as kg
        r = np.zeros(1, dtype=kg.request_dtype())[0]
        m = self.modes[i % 3]
        r["mode"], r["len"], r["unit_size"] = m, int(self.sizes[i]), 4096
        r["key"] = self.hx if m == kg.MODE_XTS else self.hs
        r["src"] = self.src.data_ptr() + int(self.offs[i])
        r["dst"] = self.dst.data_ptr() + int(self.offs[i])
        r["sector"] = int(self.offs[i]) // 4096
        if m == kg.MODE_CBC_ENC:
            r["ivs"] = self.ivs.data_ptr() + 16 * (int(self.offs[i]) // 4096)
        return r

    def check(self, idx):
        got = self.dst.cpu().numpy()
        for i in idx:
            a, b = int(self.offs[i]), int(self.offs[i] + self.sizes[i])
            x, m = self.data[a:b], i % 3
            if m == 0:
                ref = oracle.xts(self.kx, 0, x, 4096, a // 4096)
            elif m == 1:
                ref = oracle.cbc(self.ks, 0, x, 4096, self.ivs_np[a // 4096:b // 4096])
            else:
                ref = oracle.ecb(self.ks, 0, x)
            assert np.array_equal(got[a:b], ref), i

    def close(self):
        self.ctx.delkey(self.hx)
        self.ctx.delkey(self.hs)


class Collector:
    def __init__(self, expect):
        self.expect, self.calls, self.threads = expect, [], set()
        self.lock, self.done = threading.Lock(), threading.Event()

    def __call__(self, ticket, status):
        with self.lock:
            self.calls.append((ticket, status))
            self.threads.add(threading.get_ident())
            if len(self.calls) >= self.expect:
                self.done.set()


def submit_retry(ctx, req, fn):
    import time
    import paper_1305_3345_gb300 as kg
    t0 = time.time()
    while True:
        try:
            return ctx.serve_submit_cb(req, fn)
        except kg.KgpuError as e:
            if e.code != "EBUSY" or time.time() - t0 > 10:
                raise


def test_each_callback_runs_once_after_its_output(ctx):
    p = Pages(ctx, 801, 240)
    col = Collector(p.n)
    ctx.serve_start()
    try:
        tickets = [submit_retry(ctx, p.request(i), col) for i in range(p.n)]
        assert col.done.wait(60)
        assert sorted(t for t, _ in col.calls) == sorted(tickets)   # each ticket exactly once
        assert all(s == 0 for _, s in col.calls)
        assert threading.get_ident() not in col.threads and len(col.threads) == 1
        assert all(ctx.serve_poll(t, 0)[0] == 0 for t in tickets[-8:])  # still pollable
        p.check(range(p.n))
    finally:
        ctx.serve_stop(10_000_000_000)
        p.close()


def test_a_callback_submits_the_next_request(ctx):
    """Request i's callback checks nothing and submits request i + 1, so the
    whole chain runs on the completion thread."""
    p = Pages(ctx, 802, 30)
    done, order, errors = threading.Event(), [], []

    def make(i):
        def cb(ticket, status):
            order.append((i, status))
            try:
                if i + 1 < p.n:
                    submit_retry(ctx, p.request(i + 1), make(i + 1))
                else:
                    done.set()
            except Exception as e:  # surfaced below
                errors.append(e)
                done.set()
        return cb

    ctx.serve_start()
    try:
        submit_retry(ctx, p.request(0), make(0))
        assert done.wait(60)
        assert not errors
        assert order == [(i, 0) for i in range(p.n)]
        p.check(range(p.n))
    finally:
        ctx.serve_stop(10_000_000_000)
        p.close()


def test_stop_and_destroy_are_refused_from_a_callback(ctx):
    import paper_1305_3345_gb300 as kg
    p = Pages(ctx, 803, 2)
    seen, done = [], threading.Event()

    def cb(ticket, status):
        for call in (lambda: ctx.serve_stop(0), ctx.close):
            try:
                call()
                seen.append("returned")
            except kg.KgpuError as e:
                seen.append(e.code)
        done.set()

    ctx.serve_start()
    try:
        submit_retry(ctx, p.request(0), cb)
        assert done.wait(30)
        assert seen == ["EINVAL", "EINVAL"]
        assert ctx.handle is not None and ctx.handle.value   # the context survived
        t = ctx.serve_submit(p.request(1))
        assert ctx.serve_poll(t, 10_000_000_000)[0] == 0
        p.check([1])
    finally:
        ctx.serve_stop(10_000_000_000)
        p.close()


def test_stop_runs_every_waiting_callback_before_it_returns(ctx):
    """Stop with no drain time while requests are in flight, twice (the
    completion thread is started again with the ring): every callback has run
    once when the stop returns; requests that completed are exact, the others
    report KGPU_ENOENT."""
    for rnd in range(2):
        p = Pages(ctx, 804 + rnd, 240)
        col = Collector(p.n)
        ctx.serve_start()
        try:
            tickets = []
            for i in range(p.n):
                try:
                    tickets.append(ctx.serve_submit_cb(p.request(i), col))
                except Exception:
                    break            # ring full: stop with what is in flight
        finally:
            ctx.serve_stop(0)
        assert tickets
        assert sorted(t for t, _ in col.calls) == sorted(tickets)
        st = dict(col.calls)
        assert set(st.values()) <= {0, -2}
        p.check([tickets.index(t) for t, s in st.items() if s == 0])
        p.close()
