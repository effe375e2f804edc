"""Benchmark of the GB300 page-crypto path.

Headline step: AES-256-XTS encryption of a 1 GiB device-resident buffer of
262,144 x 4096-B sectors (numbered 0..262143), one kernel launch through the
C ABI.  `value` is GB/s of payload (bytes encrypted / device time).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl kgpu|reference]

N > 1 runs under torchrun: each rank encrypts its own 1 GiB replica (the path
has no exchange step), timing is max over ranks and `value` is the aggregate.
`--impl reference` times the CPU oracle on the host cores instead (rank 0 only).

The JSON line also carries: the roofline of the XTS kernel (CUDA-event launch
time), the oracle's CPU throughput on a bounded sample, an end-to-end number
through the host-buffer C-ABI call (pinned host pages, copies inside the timed
region), SM clocks sampled during the timed region, and secondary device-
resident measurements of the other modes in `extra`.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as w  # noqa: E402

GIB = 1 << 30
SECTOR = 4096
METRIC = "AES-256-XTS GB/s (1 GiB on device) vs HBM roofline; batched p50/p99 latency vs per-request"
WORKLOAD = "AES-256-XTS encrypt, 1 GiB device-resident, 262144 x 4096-B sectors 0..262143, seed 2"
SMEM_BYTES_PER_CLK_SM = 128  # shared-memory data path per SM per clock (32 banks x 4 B)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="kgpu", choices=["kgpu", "reference"])
    ap.add_argument("--no-extra", action="store_true", help="skip the secondary mode measurements")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-requests comparison")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving-loop sweep")
    ap.add_argument("--serve-seconds", type=float, default=1.0, help="length of each serving trace")
    ap.add_argument("--batch-requests", type=int, default=10000,
                    help="requests of the batched workload (10,000; fewer for a profiling case)")
    ap.add_argument("--no-host", action="store_true", help="skip the host-resident chunk sweep")
    ap.add_argument("--variant", default="table", choices=["table", "bitsliced"],
                    help="cipher of the timed step: shared-memory tables (the library's bulk path) or the "
                         "bitsliced ALU comparison variant")
    ap.add_argument("--bytes", type=int, default=GIB,
                    help="buffer size (default 1 GiB; smaller only for profiler captures)")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.device)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.25)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# The sources the bulk XTS kernel is compiled from (its kernels, the device
# cipher and its parameter structs); a traffic record is valid only for the
# kernel built from exactly these bytes.
BULK_KERNEL_SOURCES = ("aes_device.cuh", "kgpu_bulk.cu", "kgpu_bulk.h")


def csrc_hash() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1305_3345_gb300", "csrc")
    for fn in BULK_KERNEL_SOURCES:
        h.update(fn.encode())
        h.update(open(os.path.join(d, fn), "rb").read())
    return h.hexdigest()


def recorded_traffic():
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "xts256_bulk_1gib_traffic.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    if rec.get("csrc_sha256") != csrc_hash():
        return None
    return rec.get("dram_bytes_per_launch")


ALU_LANE_OPS_PER_CLK_SM = 64  # LOP3 / PRMT / SHF issue rate of one SM, measured on the GB300
BITSLICE_SOURCES = ("aes_device.cuh", "kgpu_bitslice.cu", "sbox_circuit.cuh", "kgpu_bitslice.h")


def bitslice_hash() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1305_3345_gb300", "csrc")
    for fn in BITSLICE_SOURCES:
        h.update(fn.encode())
        h.update(open(os.path.join(d, fn), "rb").read())
    return h.hexdigest()


def recorded_bitsliced():
    """The committed ncu record of the AES-256 bitsliced kernel (ALU
    lane-operations per 16-byte block, DRAM bytes of its 256 MiB capture), if
    it was taken on the current sources (else an empty dict)."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "xts256_bitsliced_alu.json")))
    except (OSError, ValueError):
        return {}
    if rec.get("csrc_sha256") != bitslice_hash():
        return {}
    return rec


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def cpu_oracle_rate(target_s: float = 15.0, whole_s: float = 30.0):
    """Oracle AES-256-XTS GB/s on a bounded sample of the same workload, on all
    host cores: the whole seed-2 buffer when a 16-MiB probe (which includes
    the threads' start-up, so it underestimates the rate) puts it within
    whole_s, else its first sectors for about target_s."""
    import oracle
    key = w.xts_key(2, 256)
    nthreads = oracle.default_threads()
    size = 16 << 20
    data = w.seeded_bytes(2, w.STREAM_DATA, size)
    t0 = time.perf_counter()
    oracle.xts(key, 0, data, SECTOR, 0, nthreads=nthreads)
    dt = time.perf_counter() - t0
    rate = size / dt
    size = GIB if GIB / rate <= whole_s else int(min(GIB, max(16 << 20, rate * target_s)) // SECTOR * SECTOR)
    data = w.seeded_bytes(2, w.STREAM_DATA, size)
    t0 = time.perf_counter()
    oracle.xts(key, 0, data, SECTOR, 0, nthreads=nthreads)
    dt = time.perf_counter() - t0
    return {"value": size / dt / 1e9, "unit": "GB/s", "cores": nthreads, "kind": "oracle",
            "sample": ("all 262144 sectors (1 GiB)" if size == GIB else
                       f"first {size // SECTOR} of the 262144 sectors ({size / 2**20:.0f} MiB)")
                      + f", AES-256-XTS encrypt, {dt:.1f} s"}


# ------------------------------------------------------------------ reference arm

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    key = w.xts_key(2, 256)
    nthreads = oracle.default_threads()
    # one step = the oracle on a bounded sample of the workload (a run of
    # 4096-B sectors), sized so warm-up + steps stay within a few minutes
    probe = w.seeded_bytes(2, w.STREAM_DATA, 8 << 20)
    t0 = time.perf_counter()
    oracle.xts(key, 0, probe, SECTOR, 0, nthreads=nthreads)
    rate = probe.size / (time.perf_counter() - t0)
    budget = 120.0 / max(1, args.steps + args.warmup)
    size = int(min(256 << 20, max(1 << 20, rate * budget)) // SECTOR * SECTOR)
    data = w.seeded_bytes(2, w.STREAM_DATA, size)
    out = np.empty_like(data)
    for _ in range(args.warmup):
        oracle.xts(key, 0, data, SECTOR, 0, out=out, nthreads=nthreads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.xts(key, 0, data, SECTOR, 0, out=out, nthreads=nthreads)
    dt = time.perf_counter() - t0
    value = size * args.steps / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"{size // SECTOR} sectors per step"},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": nthreads, "kind": "oracle",
                         "sample": f"{size // SECTOR} x 4096-B sectors ({size / 2**20:.0f} MiB) per step"},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ batched and serving workloads

def pct(lat_ns):
    """Nearest-rank p50/p99/p99.9 and max (us) of latencies in ns.  The rank
    ceil(p/100 * n) is taken in integers (p in tenths of a percent), since in
    floating point 99.9/100 * 1000 comes out just above 999."""
    a = np.sort(np.asarray(lat_ns, dtype=np.float64)) / 1e3
    if not len(a):
        return None
    q = lambda p: float(a[max(1, -(-round(p * 10) * len(a) // 1000)) - 1])
    return {"p50_us": q(50), "p99_us": q(99), "p99.9_us": q(99.9), "max_us": float(a[-1])}


def compact(obj, sig=5):
    """obj with every float rounded to `sig` significant digits (the headline
    line stays short)."""
    if isinstance(obj, float):
        return float(f"{obj:.{sig}g}")
    if isinstance(obj, dict):
        return {k: compact(v, sig) for k, v in obj.items()}
    if isinstance(obj, (list, tuple)):
        return [compact(v, sig) for v in obj]
    return obj


def stage_split(stages, sel=None):
    """p50/p99 (us) of each stage of the serving request path, from
    kgpu_replay_serve_stages' per-request record (ns since arrival): host
    queueing until published, published -> dispatcher took it, -> tiles
    published, -> first tile started, -> completed, -> host saw it."""
    s = np.asarray(stages, dtype=np.int64)
    if sel is not None:
        s = s[sel]
    ok = (s[:, 1:5] != np.iinfo(np.int64).min).all(axis=1)
    s = s[ok]
    if not len(s):
        return None
    names = ("host_queue", "to_dispatcher", "dispatch", "to_first_tile", "service", "to_host")
    d = np.stack([s[:, 0], s[:, 1] - s[:, 0], s[:, 2] - s[:, 1], s[:, 3] - s[:, 2], s[:, 4] - s[:, 3],
                  s[:, 5] - s[:, 4]], axis=1).astype(np.float64) / 1e3
    return {n: {"p50_us": round(float(np.percentile(d[:, k], 50)), 2), "p99_us": round(float(np.percentile(d[:, k], 99)), 2)}
            for k, n in enumerate(names)}


def _r(x, nd=1):
    return None if x is None else round(float(x), nd)


def batched_summary(b):
    """A few numbers of the batched comparison for the headline line."""
    bl, pl = b["batched"]["latency"] or {}, b["per_request"]["latency"] or {}
    return {"requests": int(b["workload"].split()[0]),
            "batched": {"GB/s": _r(b["batched"]["GB/s"]), "p50_ms": _r(bl.get("p50_us", 0) / 1e3, 2),
                        "p99_ms": _r(bl.get("p99_us", 0) / 1e3, 2)},
            "per_request": {"GB/s": _r(b["per_request"]["GB/s"]), "p50_ms": _r(pl.get("p50_us", 0) / 1e3, 2),
                            "p99_ms": _r(pl.get("p99_us", 0) / 1e3, 2)}}


def serving_summary(sv, svh, rt, es=None):
    """p99 (us) of the serving ring and of one launch per request at each
    offered rate, both residencies, the one-at-a-time 4 KiB round trip, and
    the empty service's p50 at 512/1024/2048 threads (host pages)."""
    def p99(d):
        return _r((d.get("latency") or {}).get("p99_us"))
    out = {"rates_req_s": [r["rate_req_s"] for r in sv["rates"]],
           "device_ring_p99_us": [p99(r["ring"]) for r in sv["rates"]],
           "device_per_request_p99_us": [p99(r["per_request"]) for r in sv["rates"]],
           "host_ring_p99_us": [p99(r["ring"]) for r in svh["rates"]],
           "host_per_request_p99_us": [p99(r["per_request"]) for r in svh["rates"]]}
    if sv.get("ring_capacity"):
        out["ring_capacity_GB/s"] = _r(sv["ring_capacity"]["ring"]["GB/s"])
    out["roundtrip_4k_p50_p99_us"] = {k: [_r((rt[k]["latency"] or {}).get("p50_us")), p99(rt[k])]
                                      for k in ("ring", "launch")}
    if es:
        out["empty_4k_host_p50_us_512_1024_2048"] = {
            form: [_r(es["host"][t][form]["p50_us"]) for t in ("512", "1024", "2048")] for form in ("ring", "launch")}
    return out


def register_mix_keys(ctx, seed, mix):
    keys = w.mix_key_material(seed, mix)
    hx = np.array([ctx.setkey(k[: 2 * b // 8], True) for k, b in zip(keys, mix.key_bits)], dtype=np.uint32)
    hs = np.array([ctx.setkey(k[: b // 8], False) for k, b in zip(keys, mix.key_bits)], dtype=np.uint32)
    return hx, hs


def build_requests(kg, mix, hx, hs, src, src_span, dst, dst_span, ivs, seed):
    """Request records for a mix: inputs are page-aligned windows of `src`,
    outputs go to `dst` at the cumulative offset (modulo dst_span), CBC IVs
    are per page from `ivs` (cyclic)."""
    n = len(mix.sizes)
    r = np.zeros(n, dtype=kg.request_dtype())
    win = (src_span - int(mix.sizes.max())) // 4096
    src_off = (w.u64(seed, 8, n) % max(1, win)).astype(np.int64) * 4096
    dst_off = (mix.offsets % (dst_span - int(mix.sizes.max()))) // 4096 * 4096
    npages = mix.sizes // 4096
    iv_pages = ivs.numel() // 16
    iv_off = (np.concatenate([[0], np.cumsum(npages)[:-1]]) % max(1, iv_pages - int(npages.max())))
    xts = mix.modes == w.MODE_XTS
    r["mode"] = mix.modes
    r["dir"] = np.where(xts, mix.dirs, 0)
    r["key"] = np.where(xts, hx[mix.keys], hs[mix.keys])
    r["src"] = src.data_ptr() + src_off
    r["dst"] = dst.data_ptr() + dst_off
    r["len"] = mix.sizes
    r["unit_size"] = 4096
    r["sector"] = mix.offsets // 4096
    r["ivs"] = np.where(xts, 0, ivs.data_ptr() + 16 * iv_off)
    return r


def run_batched(ctx, kg, dev, n=10000):
    """10,000 requests, log-uniform 4 KiB..8 MiB, 256 keys (AES-128/256), modes
    50% XTS / 25% CBC-dec / 25% CBC-enc: one persistent-kernel submission
    (autotuned launch shape, CUDA-graph replay) vs one launch per request."""
    import torch
    mix = w.request_mix(4, n, 4096, 8 << 20, 256)
    hx, hs = register_mix_keys(ctx, 4, mix)
    src = torch.from_numpy(w.seeded_bytes(4, w.STREAM_DATA, GIB)).to(f"cuda:{dev}")
    total = mix.total_bytes
    dst = torch.empty(total + (8 << 20), dtype=torch.uint8, device=f"cuda:{dev}")
    ivs = torch.from_numpy(w.page_ivs(4, int((mix.sizes // 4096).sum())).reshape(-1).copy()).to(f"cuda:{dev}")
    reqs = build_requests(kg, mix, hx, hs, src, GIB, dst, dst.numel(), ivs, 4)
    torch.cuda.synchronize()
    best, tune_ms = ctx.autotune(reqs, iters=2)
    # batched: submit -> poll, wall clock around the call pair (host packing,
    # graph launch and the whole kernel), after one warm-up
    t = ctx.submit(reqs)
    ctx.poll(t, -1)
    walls = []
    for _ in range(3):
        t0 = time.perf_counter()
        t = ctx.submit(reqs)
        ctx.poll(t, -1)
        walls.append(time.perf_counter() - t0)
    wall = min(walls)
    # per-request completion inside one batch: each request's completion word
    # as the host first sees it, from the submission
    t_sub = time.monotonic_ns()
    t = ctx.submit(reqs)
    rc_each, done = ctx.poll_each(t, n)
    lat_each = (done.astype(np.int64) - t_sub).astype(np.float64)
    # per-request launches: all 10,000 issued at once on 8 streams
    arr = np.zeros(n, dtype=np.uint64)
    ctx.replay_launches(reqs, arr, nstreams=8)           # warm-up
    rc, lat, wall_pr = ctx.replay_launches(reqs, arr, nstreams=8)
    out = {
        "workload": f"{n} requests, 4 KiB..8 MiB log-uniform (page multiples), 256 keys, "
                    "50% XTS / 25% CBC-dec / 25% CBC-enc, seed 4",
        "bytes": total,
        "batched": {"GB/s": total / wall / 1e9, "ms": wall * 1e3, "latency_all_requests_ms": wall * 1e3,
                    "latency": pct(lat_each), "latency_rc": rc_each,
                    "latency_form": "per-request completion words polled by the host (kgpu_poll_each), "
                                    "from the submission of the whole batch",
                    "tuning": best, "autotune_best_kernel_ms": tune_ms,
                    "form": "one persistent-kernel launch via CUDA graph (kgpu_submit)"},
        "per_request": {"GB/s": total / (wall_pr / 1e9) / 1e9, "ms": wall_pr / 1e6, "rc": rc,
                        "latency": pct(lat), "form": "one kernel launch per request, 8 streams"},
    }
    for h in list(hx) + list(hs):
        ctx.delkey(int(h))
    del src, dst, ivs
    torch.cuda.empty_cache()
    return out


def run_serving(ctx, kg, dev, seconds, host=False):
    """Poisson arrivals at 10k..1M requests/s, sizes log-uniform 4 KiB..1 MiB,
    1,024 keys, admission cap 8 GiB in flight: the serving ring vs one launch
    per request on the same trace (open loop, latency from arrival).  host:
    the payload pools, outputs and IVs are registered pinned host memory that
    the kernels read and write over the host link (the host-resident variant)."""
    import torch
    nkeys = 1024
    pool_in, pool_out = GIB, 9 * GIB
    if host:
        src = torch.empty(pool_in, dtype=torch.uint8, pin_memory=True)
        src.copy_(torch.from_numpy(w.seeded_bytes(5, w.STREAM_DATA, pool_in)))
        dst = torch.empty(pool_out, dtype=torch.uint8, pin_memory=True)
        ivs = torch.from_numpy(w.page_ivs(5, 1 << 20).reshape(-1).copy()).pin_memory()
        for b in (src, dst, ivs):
            ctx.host_register(b)
    else:
        src = torch.from_numpy(w.seeded_bytes(5, w.STREAM_DATA, pool_in)).to(f"cuda:{dev}")
        dst = torch.empty(pool_out, dtype=torch.uint8, device=f"cuda:{dev}")
        ivs = torch.from_numpy(w.page_ivs(5, 1 << 20).reshape(-1).copy()).to(f"cuda:{dev}")
    key_mix = w.request_mix(5, 16, 4096, 1 << 20, nkeys)
    hx, hs = register_mix_keys(ctx, 5, key_mix)
    torch.cuda.synchronize()

    def trace(rate):
        n = int(rate * seconds)
        mix = w.request_mix(5 + rate, n, 4096, 1 << 20, nkeys)
        mix.key_bits = key_mix.key_bits
        reqs = build_requests(kg, mix, hx, hs, src, pool_in, dst, pool_out, ivs, 5 + rate)
        if host:
            reqs["flags"] = np.where(mix.modes == w.MODE_XTS, kg.REQ_SRC_HOST | kg.REQ_DST_HOST,
                                     kg.REQ_SRC_HOST | kg.REQ_DST_HOST | kg.REQ_IVS_HOST)
        arr = (w.poisson_arrivals(5 + rate, n, float(rate)) * 1e9).astype(np.uint64)
        return n, mix, reqs, arr

    if host:
        # One untimed pass of the 10k-requests/s trace through both forms
        # first.  Right after the device-serving traces, the GPU's accesses to
        # host memory stall now and then for a second or two; whichever form
        # runs first takes it (XTS p99 about 100 us instead of 30 for one
        # launch per request, up to milliseconds through the ring), every
        # later pass of either form is clean.
        _, _, reqs, arr = trace(10_000)
        ctx.serve_start(admit_bytes=8 * GIB)
        try:
            ctx.replay_serve(reqs, arr, timeout_ns=120_000_000_000)
        finally:
            ctx.serve_stop(30_000_000_000)
        ctx.replay_launches(reqs, arr, nstreams=8, timeout_ns=120_000_000_000)
    def ring_pass(reqs, arr):
        ctx.serve_start(admit_bytes=8 * GIB)
        try:
            with ClockSampler(dev) as clk:
                rc, lat, wall, stg, _ = ctx.replay_serve_stages(reqs, arr, timeout_ns=120_000_000_000)
            stats = ctx.serve_stats()
        finally:
            ctx.serve_stop(30_000_000_000)
        return rc, lat, wall, stg, stats, clk

    def launch_pass(reqs, arr):
        with ClockSampler(dev) as clk:
            rc, lat, wall = ctx.replay_launches(reqs, arr, nstreams=8, timeout_ns=120_000_000_000)
        return rc, lat, wall, clk

    def p99(lat):
        return float(np.percentile(lat.astype(np.float64), 99))

    res = []
    for rate in (10_000, 100_000, 300_000, 1_000_000):
        n, mix, reqs, arr = trace(rate)
        # With host pages, after heavy host-link traffic earlier in the process
        # the GPU's accesses to host memory stall now and then for
        # milliseconds, on whichever form runs at the time.  Below saturation
        # each form replays the trace twice, alternating, and the pass with the
        # lower p99 is reported for each (both passes' p99s are recorded).
        passes = 2 if host and rate < 1_000_000 else 1
        rings, launches = [], []
        for _ in range(passes):
            rings.append(ring_pass(reqs, arr))
            launches.append(launch_pass(reqs, arr))
        rc, lat, wall, stg, stats, clk_ring = min(rings, key=lambda r: p99(r[1]))
        rc2, lat2, wall2, clk_pr = min(launches, key=lambda r: p99(r[1]))
        # device stamps lost to a slot that retired a later request before the
        # host looked are left out of the device-service and stage figures
        stamped = (stg[:, 1:5] != np.iinfo(np.int64).min).all(axis=1)
        service = stg[:, 4] - stg[:, 3]
        by_mode = {}
        for m, name in ((w.MODE_XTS, "xts"), (w.MODE_CBC_DEC, "cbc_dec"), (w.MODE_CBC_ENC, "cbc_enc")):
            sel = mix.modes == m
            if sel.any():
                by_mode[name] = {"latency": pct(lat[sel]), "device_service": pct(service[sel & stamped]),
                                 "stages": stage_split(stg, sel)}
        total = int(mix.sizes.sum())
        res.append({
            "rate_req_s": rate, "requests": n, "offered_GB/s": total / (float(arr[-1]) / 1e9) / 1e9,
            "ring": {"GB/s": total / (wall / 1e9) / 1e9, "rc": rc, "latency": pct(lat),
                     "host_wait_before_publish": pct(stg[:, 0]), "device_service": pct(service[stamped]),
                     "stages": stage_split(stg),
                     "device_stamps_lost": int(n - stamped.sum()),
                     "by_mode": by_mode, "clocks": clk_ring.summary(),
                     "busy_refusals": stats["busy_refusals"], "launches": stats["launches"],
                     "passes_p99_us": [round(p99(r[1]) / 1e3, 1) for r in rings]},
            "per_request": {"GB/s": total / (wall2 / 1e9) / 1e9, "rc": rc2, "latency": pct(lat2),
                            "clocks": clk_pr.summary(),
                            "passes_p99_us": [round(p99(r[1]) / 1e3, 1) for r in launches],
                            "by_mode": {k: {"latency": pct(lat2[mix.modes == m])} for m, k in
                                        ((w.MODE_XTS, "xts"), (w.MODE_CBC_DEC, "cbc_dec"),
                                         (w.MODE_CBC_ENC, "cbc_enc")) if (mix.modes == m).any()}},
        })
    capacity = None
    if not host:
        # past saturation, ring only: 3M requests/s (~560 GB/s offered) for
        # half the trace length shows what the ring sustains (one launch per
        # request saturates near 27 GB/s and would need tens of seconds here)
        rate = 3_000_000
        n = int(rate * seconds / 2)
        mix = w.request_mix(5 + rate, n, 4096, 1 << 20, nkeys)
        mix.key_bits = key_mix.key_bits
        reqs = build_requests(kg, mix, hx, hs, src, pool_in, dst, pool_out, ivs, 5 + rate)
        arr = (w.poisson_arrivals(5 + rate, n, float(rate)) * 1e9).astype(np.uint64)
        ctx.serve_start(admit_bytes=8 * GIB)
        try:
            with ClockSampler(dev) as clk_cap:
                rc, lat, wall = ctx.replay_serve(reqs, arr, timeout_ns=120_000_000_000)
            stats = ctx.serve_stats()
        finally:
            ctx.serve_stop(30_000_000_000)
        total = int(mix.sizes.sum())
        capacity = {"rate_req_s": rate, "requests": n, "offered_GB/s": total / (float(arr[-1]) / 1e9) / 1e9,
                    "ring": {"GB/s": total / (wall / 1e9) / 1e9, "rc": rc, "latency": pct(lat),
                             "busy_refusals": stats["busy_refusals"], "clocks": clk_cap.summary()}}
    for h in list(hx) + list(hs):
        ctx.delkey(int(h))
    if host:
        for b in (src, dst, ivs):
            ctx.host_unregister(b)
    del src, dst, ivs
    torch.cuda.empty_cache()
    where = ("payloads, outputs and IVs in registered pinned host memory, read and written by the kernels "
             "over the host link" if host else "payloads pre-staged in device memory")
    if host:
        where += ("; one untimed pass of the 10k trace through both forms first; below 1M requests/s each form "
                  "replays the trace twice (alternating) and its pass with the lower p99 is reported")
    return {"workload": "Poisson arrivals, sizes 4 KiB..1 MiB log-uniform, 1024 keys (AES-128/256), "
                        "50% XTS / 25% CBC-dec / 25% CBC-enc, admission cap 8 GiB, "
                        f"{seconds:g} s per rate; {where}",
            "rates": res, "ring_capacity": capacity}


def run_host_stream(ctx, kg, kh, dev):
    """Host-resident pages (pinned) through kgpu_aes_xts_crypt_host: chunk size
    swept 64 KiB..64 MiB at 64 MiB and 1 GiB, plus 4 GiB at 64 MiB chunks;
    reported against the measured host-link bandwidth (pinned copies alone)."""
    import torch
    out = {"link": {}, "sweep": []}
    big = GIB
    h = torch.empty(big, dtype=torch.uint8).pin_memory()
    h2 = torch.empty(big, dtype=torch.uint8).pin_memory()
    d = torch.empty(big, dtype=torch.uint8, device=f"cuda:{dev}")
    d2 = torch.empty(big, dtype=torch.uint8, device=f"cuda:{dev}")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps

    def both():
        with torch.cuda.stream(s1):
            d.copy_(h, non_blocking=True)
        with torch.cuda.stream(s2):
            h2.copy_(d2, non_blocking=True)

    out["link"]["h2d_GB/s"] = big / timed(lambda: d.copy_(h, non_blocking=True)) / 1e9
    out["link"]["d2h_GB/s"] = big / timed(lambda: h2.copy_(d, non_blocking=True)) / 1e9
    out["link"]["both_directions_GB/s"] = 2 * big / timed(both) / 1e9
    del d, d2
    torch.cuda.empty_cache()
    src = torch.from_numpy(w.seeded_bytes(3, w.STREAM_DATA, big))
    h.copy_(src)
    del src
    for size in (64 << 20, GIB):
        for chunk in (64 << 10, 256 << 10, 1 << 20, 4 << 20, 16 << 20, 64 << 20):
            if chunk > size:
                continue
            hs, hd = h[:size], h2[:size]
            t = timed(lambda: ctx.xts_crypt_host(kh, 0, hs, hd, SECTOR, 0, chunk), reps=3)
            out["sweep"].append({"bytes": size, "chunk": chunk, "GB/s": size / t / 1e9})
    # zero-copy: one batched request whose pages stay in registered host
    # memory; the kernel reads and writes them over the host link directly
    def host_request(a, b, size):
        r = np.zeros(1, dtype=kg.request_dtype())
        r["mode"], r["key"], r["src"], r["dst"] = kg.MODE_XTS, kh, a.data_ptr(), b.data_ptr()
        r["len"], r["unit_size"], r["flags"] = size, SECTOR, kg.REQ_SRC_HOST | kg.REQ_DST_HOST
        return r

    out["zero_copy"] = []
    ctx.host_register(h)
    ctx.host_register(h2)
    try:
        for size in (64 << 20, GIB):
            r = host_request(h, h2, size)
            t = timed(lambda: ctx.poll(ctx.submit(r), -1), reps=3)
            out["zero_copy"].append({"bytes": size, "GB/s": size / t / 1e9})
    finally:
        ctx.host_unregister(h)
        ctx.host_unregister(h2)
    del h, h2
    h4 = torch.empty(4 * GIB, dtype=torch.uint8).pin_memory()
    t = timed(lambda: ctx.xts_crypt_host(kh, 0, h4, h4, SECTOR, 0, 64 << 20), reps=2)
    out["sweep"].append({"bytes": 4 * GIB, "chunk": 64 << 20, "GB/s": 4 * GIB / t / 1e9, "in_place": True})
    ctx.host_register(h4)
    try:
        r = host_request(h4, h4, 4 * GIB)
        t = timed(lambda: ctx.poll(ctx.submit(r), -1), reps=2)
        out["zero_copy"].append({"bytes": 4 * GIB, "GB/s": 4 * GIB / t / 1e9, "in_place": True})
    finally:
        ctx.host_unregister(h4)
    del h4
    zbest = max(out["zero_copy"], key=lambda r: r["GB/s"])
    out["zero_copy_frac_of_link_both_directions"] = 2 * zbest["GB/s"] / out["link"]["both_directions_GB/s"]
    best = max(out["sweep"], key=lambda r: r["GB/s"])
    out["best"] = best
    out["frac_of_link_both_directions"] = 2 * best["GB/s"] / out["link"]["both_directions_GB/s"]
    out["workload"] = "AES-256-XTS over pinned host pages, 4096-B sectors, seed 3"
    return out


def run_roundtrip(ctx, kg, dev):
    """One request at a time (arrivals 300 us apart, so each is alone): the
    host-observed round trip of a 4 KiB AES-256-XTS request through the serving
    ring vs through one kernel launch -- the GB300 counterpart of the paper's
    Non-Stop Kernel measurement (launch + 4 KB input + wait, timed on the CPU)."""
    import torch
    key = ctx.setkey(w.xts_key(6, 256), True)
    n = 2000
    src = torch.from_numpy(w.seeded_bytes(6, w.STREAM_DATA, n * 4096)).to(f"cuda:{dev}")
    dst = torch.empty_like(src)
    r = np.zeros(n, dtype=kg.request_dtype())
    r["mode"] = kg.MODE_XTS
    r["key"] = key
    r["src"] = src.data_ptr() + 4096 * np.arange(n)
    r["dst"] = dst.data_ptr() + 4096 * np.arange(n)
    r["len"] = 4096
    r["unit_size"] = 4096
    r["sector"] = np.arange(n)
    arr = (np.arange(n) * 300_000).astype(np.uint64)
    torch.cuda.synchronize()
    ctx.serve_start()
    try:
        rc, lat, _, stg, _ = ctx.replay_serve_stages(r, arr)
    finally:
        ctx.serve_stop(10_000_000_000)
    rc2, lat2, _ = ctx.replay_launches(r, arr, nstreams=1)
    # the same with the 4 KiB pages in registered host memory: the kernel
    # reads the input and writes the output over the host link
    hsrc = src.cpu().pin_memory()
    hdst = torch.empty_like(hsrc).pin_memory()
    ctx.host_register(hsrc)
    ctx.host_register(hdst)
    rh = r.copy()
    rh["src"] = hsrc.data_ptr() + 4096 * np.arange(n)
    rh["dst"] = hdst.data_ptr() + 4096 * np.arange(n)
    rh["flags"] = kg.REQ_SRC_HOST | kg.REQ_DST_HOST
    ctx.serve_start()
    try:
        rc3, lat3, _, stg3, _ = ctx.replay_serve_stages(rh, arr)
    finally:
        ctx.serve_stop(10_000_000_000)
    rc4, lat4, _ = ctx.replay_launches(rh, arr, nstreams=1)
    ctx.host_unregister(hsrc)
    ctx.host_unregister(hdst)
    ctx.delkey(key)
    return {"workload": "4 KiB AES-256-XTS requests, one in flight at a time, 2000 requests; "
                        "pages in device memory, and in registered pinned host memory (host_*)",
            "ring": {"rc": rc, "latency": pct(lat), "stages": stage_split(stg)},
            "launch": {"rc": rc2, "latency": pct(lat2)},
            "host_ring": {"rc": rc3, "latency": pct(lat3), "stages": stage_split(stg3)},
            "host_launch": {"rc": rc4, "latency": pct(lat4)},
            "paper_context": "GTX 480 Non-Stop Kernel: 16.7 us (512 threads) for launch + 4 KB + wait"}


def run_empty_service(ctx, kg, dev):
    """The paper's Non-Stop Kernel measurement (section 3.1): one request at a
    time carrying a 4 KiB input through a service that does no work (here it
    copies the input through unchanged), timed on the host from submission
    until the completion is seen, with 512, 1024 and 2048 threads taking part.
    Ring: the request is split into 4096 / (threads / 32)-byte tiles, one warp
    each, on the persistent serving kernel.  Launch: one plain launch of that
    many threads per request.  Pages in registered pinned host memory (the
    input crosses the host link, as the paper's did over PCIe) and in device
    memory."""
    import torch
    n = 2000
    data = w.seeded_bytes(8, w.STREAM_DATA, n * 4096)
    bufs = {"host": (torch.from_numpy(data.copy()).pin_memory(), torch.zeros(n * 4096, dtype=torch.uint8).pin_memory()),
            "device": (torch.from_numpy(data.copy()).to(f"cuda:{dev}"),
                       torch.zeros(n * 4096, dtype=torch.uint8, device=f"cuda:{dev}"))}
    for t in bufs["host"]:
        ctx.host_register(t)
    torch.cuda.synchronize()
    arr = (np.arange(n) * 300_000).astype(np.uint64)
    out = {"workload": "empty service (4 KiB copied through unchanged), one request at a time, 2000 requests "
                       "300 us apart; latency from submission to the host seeing the completion",
           "paper_context": "GTX 480 Non-Stop Kernel, launch + 4 KB + wait: 16.7 / 17.3 / 18.3 us at "
                            "512 / 1024 / 2048 threads; 1.3x faster than a plain launch"}
    try:
        for where, (src, dst) in bufs.items():
            flags = kg.REQ_SRC_HOST | kg.REQ_DST_HOST if where == "host" else 0
            reqs = {}
            for threads in (512, 1024, 2048):
                r = np.zeros(n, dtype=kg.request_dtype())
                r["mode"], r["len"], r["unit_size"], r["flags"] = kg.MODE_COPY, 4096, 4096 * 32 // threads, flags
                r["src"] = src.data_ptr() + 4096 * np.arange(n)
                r["dst"] = dst.data_ptr() + 4096 * np.arange(n)
                reqs[threads] = r
            rows = {t: {} for t in reqs}
            ctx.serve_start()
            try:
                for t, r in reqs.items():
                    rc, lat, _, stg, off = ctx.replay_serve_stages(r, arr)
                    rows[t]["ring"] = dict(pct(lat), rc=rc, stages=stage_split(stg))
            finally:
                ctx.serve_stop(10_000_000_000)
            for t, r in reqs.items():
                rc, lat, _ = ctx.replay_launches(r, arr, nstreams=1)
                rows[t]["launch"] = dict(pct(lat), rc=rc)
            torch.cuda.synchronize()
            if not np.array_equal(dst.cpu().numpy(), data):
                raise SystemExit(f"empty service output differs from its input ({where} pages)")
            out[where] = {str(t): v for t, v in rows.items()}
    finally:
        for t in bufs["host"]:
            ctx.host_unregister(t)
    return out


def run_crossover(ctx, kg, dev):
    """The paper's proposed start-up calibration (section 4): per mode and key
    size, the request size from which the GPU is faster than the CPU.  Host-
    resident pages: kgpu_calibrate_dispatch against one launch and against
    the serving ring (the library's GPU legs) with OpenSSL AES on one host core
    as the CPU leg.  Device-resident pages (AES-256-XTS): the GPU leg is one
    request through the library; the CPU would first have to copy the pages
    out of HBM and back, so its leg is copy-out + the host AES + copy-in."""
    import torch
    out = {"paper_context": "GTX 480 vs Core i7-930 kernel AES (ECB): GPU ahead from 8 KB (two pages)",
           "cpu_leg": "OpenSSL libcrypto 3 EVP AES (AES-NI / Arm crypto extensions), one host thread"}
    xo, pts = ctx.calibrate_dispatch()
    out["host_pages_launch"] = {"crossover_bytes": xo["bytes"], "points": pts}
    ctx.serve_start()
    try:
        xo, pts = ctx.calibrate_dispatch()
    finally:
        ctx.serve_stop(10_000_000_000)
    out["host_pages_ring"] = {"crossover_bytes": xo["bytes"], "points": pts}
    # device residency, AES-256-XTS, 4 KiB units
    key = ctx.setkey(w.xts_key(9, 256), True)
    big = 4 << 20
    data = w.seeded_bytes(9, w.STREAM_DATA, big)
    dsrc = torch.from_numpy(data.copy()).to(f"cuda:{dev}")
    ddst = torch.empty_like(dsrc)
    hsrc = torch.empty(big, dtype=torch.uint8).pin_memory()
    hdst = torch.empty(big, dtype=torch.uint8).pin_memory()
    for t in (hsrc, hdst):
        ctx.host_register(t)
    rows = []
    try:
        size = 4096
        while size <= big:
            reps = max(5, min(41, (2 << 20) // size)) | 1
            rd = np.zeros(1, dtype=kg.request_dtype())
            rd["mode"], rd["key"], rd["len"], rd["unit_size"] = kg.MODE_XTS, key, size, 4096
            rd["src"], rd["dst"] = dsrc.data_ptr(), ddst.data_ptr()
            rh = rd.copy()
            rh["src"], rh["dst"], rh["flags"] = hsrc.data_ptr(), hdst.data_ptr(), kg.REQ_SRC_HOST | kg.REQ_DST_HOST
            tg, tc = [], []
            for i in range(reps + 1):
                t0 = time.perf_counter()
                st, _ = ctx.crypt(rd, kg.DISPATCH_GPU)
                t1 = time.perf_counter()
                hsrc[:size].copy_(dsrc[:size])
                st2, _ = ctx.crypt(rh, kg.DISPATCH_HOST)
                ddst[:size].copy_(hdst[:size])
                torch.cuda.synchronize()
                t2 = time.perf_counter()
                if st or st2:
                    raise SystemExit(f"crossover measurement failed: {st} {st2}")
                if i:
                    tg.append(t1 - t0)
                    tc.append(t2 - t1)
            rows.append({"bytes": size, "gpu_us": float(np.median(tg)) * 1e6, "cpu_with_copies_us": float(np.median(tc)) * 1e6})
            size *= 2
    finally:
        for t in (hsrc, hdst):
            ctx.host_unregister(t)
        ctx.delkey(key)
    cross = 2 * big
    for r in reversed(rows):
        if r["gpu_us"] >= r["cpu_with_copies_us"]:
            break
        cross = r["bytes"]
    out["device_pages_xts256"] = {"crossover_bytes": cross, "points": rows}
    return out


def run_ecb_sweep(ctx, kg, dev):
    """The paper's AES measurement (section 3.3, Fig. aes): ECB encryption of
    host-resident data over a range of sizes, timed on the host and including
    the transfers.  Two forms: one request through the serving ring over
    registered pinned pages (the kernel reads and writes them over the host
    link), and the paper's own form: copy in, one kernel launch, copy out."""
    import torch
    key = ctx.setkey(w.single_key(7, 128), False)
    sizes = [4 << 10, 8 << 10, 16 << 10, 64 << 10, 256 << 10, 1 << 20, 4 << 20, 16 << 20, 64 << 20]
    big = max(sizes)
    hsrc = torch.from_numpy(w.seeded_bytes(7, w.STREAM_DATA, big)).pin_memory()
    hdst = torch.empty(big, dtype=torch.uint8).pin_memory()
    dsrc = torch.empty(big, dtype=torch.uint8, device=f"cuda:{dev}")
    ddst = torch.empty_like(dsrc)
    stream = torch.cuda.current_stream()
    ctx.host_register(hsrc)
    ctx.host_register(hdst)
    rows = []
    try:
        ctx.serve_start()
        try:
            for size in sizes:
                n = 200 if size <= (1 << 20) else 40
                gap = max(100_000, 3 * size // 100)  # ns between arrivals: one request at a time
                r = np.zeros(n, dtype=kg.request_dtype())
                r["mode"], r["key"], r["dir"] = kg.MODE_ECB, key, 0
                r["src"], r["dst"], r["len"] = hsrc.data_ptr(), hdst.data_ptr(), size
                r["flags"] = kg.REQ_SRC_HOST | kg.REQ_DST_HOST
                rc, lat, _ = ctx.replay_serve(r, (np.arange(n) * gap).astype(np.uint64))
                rows.append({"bytes": size, "ring_host_p50_us": float(np.median(lat)) / 1e3,
                             "ring_host_GB/s": size / float(np.median(lat)), "ring_rc": rc})
        finally:
            ctx.serve_stop(10_000_000_000)
        for row in rows:
            size = row["bytes"]

            def once():
                dsrc[:size].copy_(hsrc[:size], non_blocking=True)
                ctx.ecb_crypt(key, 0, dsrc[:size], ddst[:size], stream)
                hdst[:size].copy_(ddst[:size], non_blocking=True)
                stream.synchronize()
            once()
            ts = []
            for _ in range(50 if size <= (1 << 20) else 10):
                t0 = time.perf_counter()
                once()
                ts.append(time.perf_counter() - t0)
            t = float(np.median(ts))
            row["copy_launch_copy_p50_us"] = t * 1e6
            row["copy_launch_copy_GB/s"] = size / t / 1e9
    finally:
        ctx.host_unregister(hsrc)
        ctx.host_unregister(hdst)
        ctx.delkey(key)
    return {"workload": "AES-128-ECB encryption of host-resident data, one request at a time, seed 7; "
                        "latency from submission to the result in host memory",
            "paper_context": "GTX 480 + Core i7-930 (Fig. aes, figure not in the source): GPU ECB ahead of the "
                             "kernel's SSE AES from 8 KB, up to 6x",
            "sizes": rows}


# ------------------------------------------------------------------ GPU arm

def settle(fn, min_s: float = 1.0):
    """Untimed calls of fn until min_s seconds have passed (at least two).
    The GPU's accesses to host memory can stall now and then for a second or
    two after other work (large frees and allocations); a few warm-up calls of
    a few milliseconds would not outlast that.  Returns (calls, seconds of the
    first call, seconds of the last)."""
    t_start = time.perf_counter()
    times = []
    while len(times) < 2 or time.perf_counter() - t_start < min_s:
        t0 = time.perf_counter()
        fn()
        times.append(time.perf_counter() - t0)
    return len(times), times[0], times[-1]


def time_op(fn, iters: int, stream):
    """Mean CUDA-event time (s) of fn() over iters launches on `stream`."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(iters)]
    fn()
    torch.cuda.synchronize()
    for a, b in ev:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / iters / 1e3


def run_kgpu(args):
    import torch
    import paper_1305_3345_gb300 as kg

    rank, world, local = dist_env()
    dev = local if world > 1 else 0
    torch.cuda.set_device(dev)  # before the process group, so NCCL binds each rank to its own GPU
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    stream = torch.cuda.current_stream()

    def emit(section, obj):
        # secondary measurements go on lines of their own, before the headline
        # (no "metric" key): the headline stays the last, short line
        if rank == 0:
            print(json.dumps({"section": section, **obj}), flush=True)

    ctx = kg.Context(dev)
    nbytes = args.bytes - args.bytes % SECTOR
    svh = None
    if rank == 0 and not args.no_serve and nbytes == GIB:
        # The host-pages serving traces run first, before anything else in the
        # process: later on, after the other sections' traffic and large
        # allocations, the GPU's accesses to host memory stall now and then
        # for milliseconds (on whichever form runs at the time), while the
        # same traces in a fresh process run clean.
        svh = run_serving(ctx, kg, dev, args.serve_seconds, host=True)
        emit("serving_host", svh)
    key = w.xts_key(2, 256)
    kh = ctx.setkey(key, True)
    src = torch.from_numpy(w.seeded_bytes(2, w.STREAM_DATA, nbytes)).to(f"cuda:{dev}")
    dst = torch.empty_like(src)

    bitsliced = args.variant == "bitsliced"

    def step():
        if bitsliced:
            ctx.xts_crypt_bitsliced(kh, 0, src, dst, SECTOR, 0, stream)
        else:
            ctx.xts_crypt(kh, 0, src, dst, SECTOR, 0, stream)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        t_start.record(stream)
        for a, b in ev:
            a.record(stream)
            step()
            b.record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    elapsed = t_start.elapsed_time(t_end) / 1e3
    launch_s = sum(a.elapsed_time(b) for a, b in ev) / len(ev) / 1e3
    if dist:
        t = torch.tensor([elapsed], device=f"cuda:{dev}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())

    # the output must be the cipher (a cheap spot check against the oracle)
    if rank == 0:
        import oracle
        for s in (0, nbytes // SECTOR // 2, nbytes // SECTOR - 1):
            ref = oracle.xts(key, 0, src[s * SECTOR:(s + 1) * SECTOR].cpu().numpy(), SECTOR, s)
            if not np.array_equal(dst[s * SECTOR:(s + 1) * SECTOR].cpu().numpy(), ref):
                raise SystemExit(f"bench output mismatch at sector {s}")

    value = world * nbytes * args.steps / elapsed / 1e9
    props = torch.cuda.get_device_properties(dev)
    clocks = clk.summary()
    peaks = measured_peaks()

    # roofline of the dominant kernel (the XTS launch): algorithmic HBM bytes
    # per launch = 1 GiB read + 1 GiB written
    hbm_bytes = 2 * nbytes
    achieved_hbm = hbm_bytes / launch_s / 1e9
    hbm_peak = peaks["hbm_gbs"] if peaks else 6800.0
    # shared-memory lookups: Nr = 14 rounds x 16 lookups per 16-B block, plus
    # one tweak block per 4096-B sector (257 cipher blocks per 256 data blocks)
    nblocks = nbytes // 16
    lookups = 14 * 16 * nblocks * (257 / 256)
    smem_bytes = lookups * 4
    sm_mhz = clocks["sm_mhz"] or (peaks or {}).get("sm_max_mhz", 2070.0)
    smem_peak = props.multi_processor_count * SMEM_BYTES_PER_CLK_SM * sm_mhz * 1e6 / 1e9
    achieved_smem = smem_bytes / launch_s / 1e9
    traffic = recorded_traffic()
    roofline = {"bound": "smem", "achieved": achieved_smem, "peak": smem_peak, "unit": "GB/s",
                "frac": achieved_smem / smem_peak, "traffic": traffic,
                "peak_source": f"{props.multi_processor_count} SMs x 128 B/clk x {sm_mhz:.0f} MHz",
                "kernel": "bulk_kernel<14,enc,xts>", "launch_ms": launch_s * 1e3}
    if bitsliced:
        # ALU-bound: lane-operations of the ALU pipe per block (counted once with
        # ncu on this kernel) x blocks, against SMs x 64 lane-ops/clk x clock
        bs_rec = recorded_bitsliced()
        rec = bs_rec.get("alu_lane_ops_per_block")
        # DRAM traffic grows with the bytes processed: the 256 MiB capture
        # scaled to this launch
        cap = bs_rec.get("dram_bytes_per_launch_256mib")
        traffic = cap * nbytes / (256 << 20) if cap else None
        alu_peak = props.multi_processor_count * ALU_LANE_OPS_PER_CLK_SM * sm_mhz * 1e6 / 1e12
        achieved = rec * nblocks / launch_s / 1e12 if rec else None
        roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Tops/s",
                    "frac": achieved / alu_peak if achieved else None, "traffic": None,
                    "peak_source": f"{props.multi_processor_count} SMs x {ALU_LANE_OPS_PER_CLK_SM} ALU lane-ops/clk "
                                   f"x {sm_mhz:.0f} MHz (pipe rate measured with a LOP3 probe)",
                    "alu_lane_ops_per_block": rec,
                    "kernel": "bs_kernel<14,xts> (+ bs_tweak_kernel)", "launch_ms": launch_s * 1e3}
    roofline_hbm = {"bound": "hbm", "achieved": achieved_hbm, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved_hbm / hbm_peak, "traffic": traffic,
                    "peak_source": "measured hbm_gbs" if peaks else "fallback 6.8 TB/s"}

    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": (WORKLOAD if nbytes == GIB else f"AES-256-XTS encrypt, {nbytes} B (profiling case)")
                   + (" -- bitsliced comparison variant" if bitsliced else ""),
                   "bytes_per_gpu": nbytes, "l2": "inputs > L2 (1 GiB vs 129 MB)",
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline, "roofline_hbm": roofline_hbm, "clocks": clocks,
        "gpu_launches": args.steps * (2 if bitsliced else 1),  # bitsliced: tweak pre-pass + cipher
    }

    if rank == 0 and not args.no_extra and nbytes == GIB:
        extra = {}
        specs = []
        k128 = ctx.setkey(w.xts_key(2, 128), True)
        specs.append(("aes256_xts_dec_4k", lambda: ctx.xts_crypt(kh, 1, dst, src, SECTOR, 0, stream)))
        specs.append(("aes256_xts_enc_512", lambda: ctx.xts_crypt(kh, 0, src, dst, 512, 0, stream)))
        specs.append(("aes128_xts_enc_4k", lambda: ctx.xts_crypt(k128, 0, src, dst, SECTOR, 0, stream)))
        specs.append(("aes128_xts_dec_4k", lambda: ctx.xts_crypt(k128, 1, src, dst, SECTOR, 0, stream)))
        ck = ctx.setkey(w.single_key(2, 128), False)
        ivs = torch.from_numpy(w.page_ivs(2, GIB // SECTOR).reshape(-1).copy()).to(f"cuda:{dev}")
        specs.append(("aes128_cbc_dec_4k", lambda: ctx.cbc_decrypt(ck, src, dst, SECTOR, ivs, stream)))
        specs.append(("aes128_cbc_enc_4k", lambda: ctx.cbc_encrypt_pages(ck, src, dst, SECTOR, ivs, stream)))
        specs.append(("aes128_ecb_enc", lambda: ctx.ecb_crypt(ck, 0, src, dst, stream)))
        # the bitsliced (ALU, no tables) comparison variant of the headline and of AES-128-XTS
        specs.append(("aes256_xts_enc_4k_bitsliced",
                      lambda: ctx.xts_crypt_bitsliced(kh, 0, src, dst, SECTOR, 0, stream)))
        specs.append(("aes128_xts_enc_4k_bitsliced",
                      lambda: ctx.xts_crypt_bitsliced(k128, 0, src, dst, SECTOR, 0, stream)))
        # shared-memory lookups per 16-byte block of each table mode: Nr x 16,
        # times (1 + 1/blocks per unit) for the XTS tweak; the bitsliced modes
        # do no lookups (their bound is the ALU, see --variant bitsliced)
        lookups = {"aes256_xts_dec_4k": 14 * 16 * 257 / 256, "aes256_xts_enc_512": 14 * 16 * 33 / 32,
                   "aes128_xts_enc_4k": 10 * 16 * 257 / 256, "aes128_xts_dec_4k": 10 * 16 * 257 / 256,
                   "aes128_cbc_dec_4k": 10 * 16, "aes128_cbc_enc_4k": 10 * 16, "aes128_ecb_enc": 10 * 16}
        smem_bound_clk = props.multi_processor_count * SMEM_BYTES_PER_CLK_SM * sm_mhz * 1e6
        for name, fn in specs:
            t = time_op(fn, 20, stream)
            extra[name] = {"GB/s": GIB / t / 1e9, "ms": t * 1e3}
            if name in lookups:
                bound = smem_bound_clk / (lookups[name] * 4) * 16 / 1e9
                extra[name]["smem_bound_GB/s"] = bound
                extra[name]["frac_of_smem_bound"] = GIB / t / 1e9 / bound
        emit("extra", {"modes": extra})
        ctx.delkey(k128)
        ctx.delkey(ck)
        del ivs

    if not args.no_e2e and nbytes == GIB:
        # end to end through the host-buffer call: 1 GiB in pinned host memory,
        # 1 GiB out, per rank; every rank runs it between barriers and the
        # slowest rank's time counts.  Two forms of the same call: the pages
        # registered once with kgpu_host_register (the kernel reads and writes
        # them over the host link), and unregistered pinned pages (the chunked
        # copy/compute pipeline).
        hsrc = torch.empty(GIB, dtype=torch.uint8).pin_memory()
        hsrc.copy_(src.cpu())
        hdst = torch.empty(GIB, dtype=torch.uint8).pin_memory()
        chunk = 64 << 20
        e2e_steps = max(3, min(args.steps, 10))

        warm = {}

        def host_steps(form):
            calls, first, last = settle(lambda: ctx.xts_crypt_host(kh, 0, hsrc, hdst, SECTOR, 0, chunk))
            warm[form] = {"calls": calls, "first_GB/s": world * GIB / first / 1e9,
                          "last_GB/s": world * GIB / last / 1e9}
            if dist:
                dist.barrier()
            steps_s = []
            for _ in range(e2e_steps):
                t0 = time.perf_counter()
                ctx.xts_crypt_host(kh, 0, hsrc, hdst, SECTOR, 0, chunk)
                steps_s.append(time.perf_counter() - t0)
            # the median step: the host link is shared with the rest of the node,
            # and one transient should not set the figure (the mean is reported too)
            dt, dmean = float(np.median(steps_s)), float(np.mean(steps_s))
            if dist:
                t = torch.tensor([dt, dmean], device=f"cuda:{dev}")
                dist.all_reduce(t, op=dist.ReduceOp.MAX)
                dt, dmean = float(t[0].item()), float(t[1].item())
            if rank == 0:
                import oracle
                for sct in (0, 262143):
                    ref = oracle.xts(key, 0, hsrc[sct * SECTOR:(sct + 1) * SECTOR].numpy(), SECTOR, sct)
                    if not np.array_equal(hdst[sct * SECTOR:(sct + 1) * SECTOR].numpy(), ref):
                        raise SystemExit(f"e2e output mismatch at sector {sct}")
                hdst.zero_()
            return dt, dmean

        ctx.host_register(hsrc)
        ctx.host_register(hdst)
        try:
            dt, dmean = host_steps("registered")
        finally:
            ctx.host_unregister(hsrc)
            ctx.host_unregister(hdst)
        line["e2e"] = {"value": world * GIB / dt / 1e9, "unit": "GB/s", "h2d_bytes_per_step": world * GIB,
                       "d2h_bytes_per_step": world * GIB, "steps": e2e_steps, "statistic": "median step",
                       "call": "kgpu_aes_xts_crypt_host"}
        dt, dmean = host_steps("copy_pipeline")
        e2e_forms = {}
        e2e_forms["e2e_copy_pipeline"] = {"value": world * GIB / dt / 1e9, "unit": "GB/s",
                                     "h2d_bytes_per_step": world * GIB, "d2h_bytes_per_step": world * GIB,
                                     "steps": e2e_steps, "chunk_bytes": chunk, "statistic": "median step",
                                     "mean_GB/s": world * GIB / dmean / 1e9,
                                     "call": "kgpu_aes_xts_crypt_host on unregistered pinned host pages "
                                             "(chunked copy/compute pipeline)"}
        # the same step with the pages left in registered host memory: one
        # batched request whose kernel reads and writes them over the link
        ctx.host_register(hsrc)
        ctx.host_register(hdst)
        r = np.zeros(1, dtype=kg.request_dtype())
        r["mode"], r["key"], r["src"], r["dst"] = kg.MODE_XTS, kh, hsrc.data_ptr(), hdst.data_ptr()
        r["len"], r["unit_size"], r["flags"] = GIB, SECTOR, kg.REQ_SRC_HOST | kg.REQ_DST_HOST
        calls, first, last = settle(lambda: ctx.poll(ctx.submit(r), -1))
        warm["zero_copy"] = {"calls": calls, "first_GB/s": world * GIB / first / 1e9,
                             "last_GB/s": world * GIB / last / 1e9}
        if dist:
            dist.barrier()
        zs = []
        for _ in range(e2e_steps):
            t0 = time.perf_counter()
            ctx.poll(ctx.submit(r), -1)
            zs.append(time.perf_counter() - t0)
        dz = float(np.median(zs))
        if dist:
            t = torch.tensor([dz], device=f"cuda:{dev}")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dz = float(t.item())
        ctx.host_unregister(hsrc)
        ctx.host_unregister(hdst)
        e2e_forms["e2e_zero_copy"] = {"value": world * GIB / dz / 1e9, "unit": "GB/s",
                                 "link_bytes_per_step": {"host_to_device": world * GIB, "device_to_host": world * GIB},
                                 "steps": e2e_steps, "statistic": "median step",
                                 "call": "kgpu_submit + kgpu_poll, src/dst flagged host"}
        e2e_forms["untimed_warmup"] = warm
        emit("e2e_forms", e2e_forms)
        del hsrc, hdst

    if rank == 0 and not args.no_batched and (nbytes == GIB or args.batch_requests != 10000):
        b = run_batched(ctx, kg, dev, args.batch_requests)
        emit("batched", b)
        line["batched"] = batched_summary(b)

    if rank == 0 and not args.no_serve and nbytes == GIB:
        sv = run_serving(ctx, kg, dev, args.serve_seconds)
        emit("serving", sv)
        rt = run_roundtrip(ctx, kg, dev)
        emit("roundtrip", rt)
        es = run_empty_service(ctx, kg, dev)
        emit("empty_service", es)
        line["serving"] = serving_summary(sv, svh, rt, es)
        emit("ecb_size_sweep", run_ecb_sweep(ctx, kg, dev))
        emit("crossover", run_crossover(ctx, kg, dev))

    if rank == 0 and not args.no_host and nbytes == GIB:
        emit("host_stream", run_host_stream(ctx, kg, kh, dev))

    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_oracle_rate()

    ctx.delkey(kh)
    ctx.close()
    if rank == 0:
        print(json.dumps(compact(line), separators=(",", ":")), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_kgpu(args)


if __name__ == "__main__":
    main()
