"""Host-side helpers of bench.py, checked on the CPU: the latency quantiles,
the float rounding of the headline line, the serving stage split, and the
size of the batched and serving summaries that ride on the headline line
(which must stay a short, parseable last line)."""
import json

import numpy as np

import bench

I64_MIN = np.iinfo(np.int64).min


def test_pct_is_nearest_rank_in_microseconds():
    lat_ns = np.arange(1, 1001, dtype=np.int64) * 1000  # 1..1000 us, shuffled below
    rng = np.random.default_rng(0)
    rng.shuffle(lat_ns)
    q = bench.pct(lat_ns)
    assert q == {"p50_us": 500.0, "p99_us": 990.0, "p99.9_us": 999.0, "max_us": 1000.0}
    assert bench.pct([]) is None
    assert bench.pct([7000]) == {"p50_us": 7.0, "p99_us": 7.0, "p99.9_us": 7.0, "max_us": 7.0}


def test_compact_rounds_floats_only():
    obj = {"a": 1.23456789, "b": [672.954321, {"c": 0.000123456789}], "n": 10000, "s": "x", "t": (2.0, 3)}
    out = bench.compact(obj)
    assert out == {"a": 1.2346, "b": [672.95, {"c": 0.00012346}], "n": 10000, "s": "x", "t": [2.0, 3]}
    assert isinstance(out["n"], int)
    assert bench.compact(123456789.0) == 123460000.0


def test_stage_split_differences_and_dropped_rows():
    n = 100
    # stamps in ns since arrival: published, taken, tiles out, first tile, done, host saw it
    inc = np.array([400, 2800, 1400, 1900, 4900, 100], dtype=np.int64)
    s = np.tile(np.cumsum(inc), (n, 1))
    s[:, 4] += np.arange(n) * 10  # service grows by 10 ns per request, host sighting with it
    s[:, 5] += np.arange(n) * 10
    bad = s.copy()[:5]
    bad[:, 2] = I64_MIN  # a request whose stamps were never written
    out = bench.stage_split(np.concatenate([s, bad]))
    assert out["host_queue"] == {"p50_us": 0.4, "p99_us": 0.4}
    assert out["to_dispatcher"] == {"p50_us": 2.8, "p99_us": 2.8}
    assert out["dispatch"] == {"p50_us": 1.4, "p99_us": 1.4}
    assert out["to_first_tile"] == {"p50_us": 1.9, "p99_us": 1.9}
    assert out["service"]["p50_us"] == round(float(np.percentile(4900 + np.arange(n) * 10, 50)) / 1e3, 2)
    assert out["to_host"] == {"p50_us": 0.1, "p99_us": 0.1}
    assert bench.stage_split(bad) is None
    sel = np.zeros(n, dtype=bool)
    sel[:10] = True
    assert bench.stage_split(s, sel)["service"]["p99_us"] <= 4.99


def _lat(p50, p99):
    return {"p50_us": p50, "p99_us": p99, "p99.9_us": p99 * 1.1, "max_us": p99 * 1.2}


def test_summaries_stay_short_with_long_numbers():
    # batched: worst-case-length figures
    b = {"workload": "10000 requests, ...",
         "batched": {"GB/s": 646.3456789, "latency": _lat(1396.2881234, 15961.47212)},
         "per_request": {"GB/s": 134.5678912, "latency": _lat(40431.123456, 79711.987654)}}
    bs = bench.batched_summary(b)
    assert bs == {"requests": 10000,
                  "batched": {"GB/s": 646.3, "p50_ms": 1.4, "p99_ms": 15.96},
                  "per_request": {"GB/s": 134.6, "p50_ms": 40.43, "p99_ms": 79.71}}
    # serving: four rates, saturated rates with multi-second p99s
    rates = [10_000, 100_000, 300_000, 1_000_000]

    def form(p99):
        return {"latency": _lat(p99 / 10, p99)}

    sv = {"rates": [{"rate_req_s": r, "ring": form(180.0 + 1e-6 * r), "per_request": form(1234567.891 * (k + 1))}
                    for k, r in enumerate(rates)],
          "ring_capacity": {"ring": {"GB/s": 522.3987654}}}
    svh = {"rates": [{"rate_req_s": r, "ring": form(987654.321 * (k + 1)), "per_request": form(7654321.987)}
                     for k, r in enumerate(rates)]}
    rt = {"ring": {"latency": _lat(12.16, 16.544)}, "launch": {"latency": _lat(21.504, 23.712)}}
    es = {"host": {t: {"ring": {"p50_us": 9.1876}, "launch": {"p50_us": 12.8765}} for t in ("512", "1024", "2048")}}
    ss = bench.serving_summary(sv, svh, rt, es)
    assert ss["rates_req_s"] == rates
    assert ss["ring_capacity_GB/s"] == 522.4
    assert ss["roundtrip_4k_p50_p99_us"] == {"ring": [12.2, 16.5], "launch": [21.5, 23.7]}
    assert ss["empty_4k_host_p50_us_512_1024_2048"]["launch"] == [12.9, 12.9, 12.9]
    line = bench.compact({"batched": bs, "serving": ss})
    text = json.dumps(line, separators=(",", ":"))
    assert json.loads(text) == line
    # the rest of the headline line is about 1.3 KB of fixed-shape fields
    assert len(text) < 650, len(text)
