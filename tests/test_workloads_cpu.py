"""The seeded input generators shared by the oracle tests, the GPU tests and the
bench (workloads/), checked on the CPU: SplitMix64 against its published
output for seed 0, the counter form's slicing, the byte order, and the shape of
the batched and serving workload recipes."""
import numpy as np

import workloads as w


def test_splitmix64_matches_its_published_sequence():
    # SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) from state 0 yields, in order,
    # these words; the counter form's word i is mix((i + 1) * GAMMA) from base 0
    expect = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    with np.errstate(over="ignore"):
        got = w._mix(np.arange(1, 5, dtype=np.uint64) * w.GAMMA)
    assert [int(x) for x in got] == expect


def test_counter_form_slices_without_the_prefix():
    whole = w.u64(9, w.STREAM_DATA, 1000)
    assert np.array_equal(w.u64(9, w.STREAM_DATA, 100, start=437), whole[437:537])
    assert not np.array_equal(w.u64(9, w.STREAM_KEY, 1000), whole)   # streams differ
    assert not np.array_equal(w.u64(10, w.STREAM_DATA, 1000), whole)  # seeds differ


def test_bytes_are_the_words_little_endian():
    words = w.u64(3, w.STREAM_IV, 4)
    b = w.seeded_bytes(3, w.STREAM_IV, 29)
    assert b.dtype == np.uint8 and b.size == 29
    expect = b"".join(int(x).to_bytes(8, "little") for x in words)[:29]
    assert bytes(b) == expect
    assert w.page_ivs(3, 2).shape == (2, 16)
    assert bytes(w.page_ivs(3, 2).reshape(-1)) == bytes(w.seeded_bytes(3, w.STREAM_IV, 32))


def test_keys():
    k = w.xts_key(2, 256)
    assert len(k) == 64 and k[:32] != k[32:]
    assert len(w.xts_key(2, 128)) == 32
    assert w.single_key(2, 192) == w.xts_key(2, 256)[:24]  # one key stream, prefixes


def test_batched_workload_shape():
    mix = w.request_mix(4, 10000, 4096, 8 << 20, 256)
    assert (mix.sizes % 4096 == 0).all()
    assert mix.sizes.min() >= 4096 and mix.sizes.max() <= 8 << 20
    # log-uniform: about half the requests below the geometric midpoint (181 KiB)
    below = (mix.sizes < np.sqrt(4096 * (8 << 20))).mean()
    assert 0.47 < below < 0.53
    share = np.bincount(mix.modes, minlength=3) / mix.modes.size
    assert abs(share[w.MODE_XTS] - 0.5) < 0.02 and abs(share[w.MODE_CBC_DEC] - 0.25) < 0.02
    assert abs(share[w.MODE_CBC_ENC] - 0.25) < 0.02
    assert list(np.unique(mix.key_bits[:128])) == [128] and list(np.unique(mix.key_bits[128:])) == [256]
    assert mix.keys.min() >= 0 and mix.keys.max() < 256
    assert np.array_equal(mix.offsets, np.concatenate([[0], np.cumsum(mix.sizes)[:-1]]))
    assert 10e9 < mix.total_bytes < 12e9  # about 10-11 GB


def test_serving_arrivals():
    rate = 100_000
    t = w.poisson_arrivals(7, rate, float(rate))
    assert (np.diff(t) > 0).all()
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() * rate - 1) < 0.02  # mean gap 1 / rate
    assert abs(gaps.std() * rate - 1) < 0.03   # exponential: std equals the mean
