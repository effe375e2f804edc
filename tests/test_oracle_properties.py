"""Property-based pins for the CPU oracle (hypothesis draws the cases; CPU only).

For random keys, data-unit sizes (including sizes that end in a partial block),
unit counts and sector numbers anywhere in the 64-bit range, the oracle must
equal OpenSSL's XTS, CBC and ECB byte for byte, and decryption must invert
encryption.  A mistake that only shows for some sizes or unit numbers (a carry
across the 32-bit halves of the sector number, a stealing tail of one
particular length) is what these draws are for.
"""
import numpy as np
import pytest

import oracle

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
crypto = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
given, settings = hyp.given, hyp.settings
Cipher, algorithms, modes = crypto.Cipher, crypto.algorithms, crypto.modes


def _ossl_xts(key, dir, data, du, first):
    out = bytearray()
    for u in range(len(data) // du):
        c = Cipher(algorithms.AES(key), modes.XTS(((first + u) % 2**64).to_bytes(16, "little")))
        op = c.encryptor() if dir == 0 else c.decryptor()
        out += op.update(data[u * du:(u + 1) * du]) + op.finalize()
    return bytes(out)


xts_keys = st.sampled_from([32, 64]).flatmap(
    lambda n: st.binary(min_size=n, max_size=n).filter(lambda k: k[: n // 2] != k[n // 2:]))


@settings(max_examples=60, deadline=None)
@given(key=xts_keys, du=st.integers(16, 600), units=st.integers(1, 5), first=st.integers(0, 2**64 - 6),
       seed=st.integers(0, 2**32 - 1))
def test_xts_matches_openssl(key, du, units, first, seed):
    data = np.random.default_rng(seed).integers(0, 256, du * units, dtype=np.uint8)
    c = oracle.xts(key, 0, data, du, first)
    assert c.tobytes() == _ossl_xts(key, 0, data.tobytes(), du, first)
    assert oracle.xts(key, 1, c, du, first).tobytes() == data.tobytes()


@settings(max_examples=40, deadline=None)
@given(bits=st.sampled_from([128, 192, 256]), page=st.integers(1, 40).map(lambda b: 16 * b),
       npages=st.integers(1, 6), seed=st.integers(0, 2**32 - 1))
def test_cbc_matches_openssl(bits, page, npages, seed):
    rng = np.random.default_rng(seed)
    key = rng.integers(0, 256, bits // 8, dtype=np.uint8).tobytes()
    data = rng.integers(0, 256, page * npages, dtype=np.uint8)
    ivs = rng.integers(0, 256, (npages, 16), dtype=np.uint8)
    c = oracle.cbc(key, 0, data, page, ivs)
    ref = bytearray()
    for p in range(npages):
        e = Cipher(algorithms.AES(key), modes.CBC(ivs[p].tobytes())).encryptor()
        ref += e.update(data[p * page:(p + 1) * page].tobytes()) + e.finalize()
    assert c.tobytes() == bytes(ref)
    assert oracle.cbc(key, 1, c, page, ivs).tobytes() == data.tobytes()


@settings(max_examples=40, deadline=None)
@given(bits=st.sampled_from([128, 192, 256]), nblocks=st.integers(1, 70), seed=st.integers(0, 2**32 - 1))
def test_ecb_matches_openssl(bits, nblocks, seed):
    rng = np.random.default_rng(seed)
    key = rng.integers(0, 256, bits // 8, dtype=np.uint8).tobytes()
    data = rng.integers(0, 256, 16 * nblocks, dtype=np.uint8)
    e = Cipher(algorithms.AES(key), modes.ECB()).encryptor()
    assert oracle.ecb(key, 0, data).tobytes() == e.update(data.tobytes()) + e.finalize()
    assert oracle.ecb(key, 1, oracle.ecb(key, 0, data)).tobytes() == data.tobytes()
