"""Pins for the CPU oracle, against things other than the oracle itself.

Each pin is chosen so that a plausible slip in the oracle (a wrong reduction
polynomial, a dropped affine term, a transposed state, a wrong shift direction,
a big-endian tweak, a wrong Rcon step, a mis-chained CBC) fails at least one:

* field axioms and a second, independent GF(2^8) multiplication (polynomial
  long division) -- FIPS-197 section 4.2;
* S-box structure that the definition fixes (bijection, S(0) = 0x63 from the
  affine constant, no fixed or opposite-fixed points) -- FIPS-197 5.1.1;
* MixColumns as polynomial multiplication modulo x^4 + 1 -- FIPS-197 4.3/5.1.3;
* byte equality with OpenSSL (through the `cryptography` package), a library
  routine, for the block cipher, XTS (IEEE 1619) and CBC (SP 800-38A);
* the XTS tweak step against brute-force GF(2^128) arithmetic on Python ints;
* round trips and in-place operation.
"""
import numpy as np
import pytest

import oracle
import workloads as w

crypto = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
Cipher, algorithms, modes = crypto.Cipher, crypto.algorithms, crypto.modes


# ----------------------------------------------------------------- GF(2^8)

def _polymod_mul(a: int, b: int) -> int:
    """Carry-less product, then remainder by x^8+x^4+x^3+x+1 by long division."""
    p = 0
    for i in range(8):
        if (b >> i) & 1:
            p ^= a << i
    for deg in range(14, 7, -1):
        if (p >> deg) & 1:
            p ^= 0x11B << (deg - 8)
    return p


@pytest.fixture(scope="module")
def mul_table():
    return np.array([[oracle.gf_mul(a, b) for b in range(256)] for a in range(256)], dtype=np.uint8)


def test_gf_mul_matches_long_division(mul_table):
    ref = np.array([[_polymod_mul(a, b) for b in range(256)] for a in range(256)], dtype=np.uint8)
    assert np.array_equal(mul_table, ref)


def test_gf_field_axioms(mul_table):
    T = mul_table.astype(np.int64)
    a = np.arange(256)
    assert np.array_equal(T, T.T)                      # commutative
    assert np.array_equal(T[:, 1], a)                  # identity
    assert np.all(T[:, 0] == 0)
    # distributive over xor, all 2^24 triples
    for x in range(256):
        lhs = T[x][a[:, None] ^ a[None, :]]
        rhs = T[x][:, None] ^ T[x][None, :]
        assert np.array_equal(lhs, rhs)
    # {03} generates the multiplicative group (order 255), which requires the
    # modulus to be irreducible and the multiplication to be right
    seen, g = set(), 1
    for _ in range(255):
        seen.add(g)
        g = int(T[g, 3])
    assert g == 1 and len(seen) == 255


def test_gf_inverse(mul_table):
    assert oracle.gf_inv(0) == 0
    for a in range(1, 256):
        assert mul_table[a, oracle.gf_inv(a)] == 1


# ----------------------------------------------------------------- S-box

def test_sbox_structure():
    s = oracle.sbox()
    inv = oracle.inv_sbox()
    assert sorted(s.tolist()) == list(range(256))     # bijection
    assert np.array_equal(inv[s], np.arange(256))      # InvS o S = id
    assert s[0] == 0x63                                # affine constant, inv(0) = 0
    assert not np.any(s == np.arange(256))             # no fixed points
    assert not np.any(s == (np.arange(256) ^ 0xFF))    # no opposite fixed points


def test_sbox_is_affine_of_inverse():
    # S(a) = A * inv(a) + c with A the circulant matrix of 0x1F over GF(2);
    # written here as a matrix product, not the oracle's bit loop.
    A = np.zeros((8, 8), dtype=np.int64)
    for i in range(8):
        for k in (0, 4, 5, 6, 7):
            A[i, (i + k) % 8] = 1
    s = oracle.sbox()
    for a in range(256):
        inv = oracle.gf_inv(a)
        bits = np.array([(inv >> j) & 1 for j in range(8)])
        out = (A @ bits) % 2
        val = sum(int(b) << j for j, b in enumerate(out)) ^ 0x63
        assert s[a] == val


# ----------------------------------------------------------------- MixColumns

def _poly4_mul(col, coeffs):
    """(sum col[i] x^i) * (sum coeffs[i] x^i) mod x^4 + 1 over GF(2^8)."""
    out = [0, 0, 0, 0]
    for i in range(4):
        for j in range(4):
            out[(i + j) % 4] ^= _polymod_mul(col[i], coeffs[j])
    return out


def test_mix_columns_polynomial():
    rng = np.random.default_rng(7)
    for _ in range(200):
        col = rng.integers(0, 256, 4).tolist()
        assert oracle.mix_column(col).tolist() == _poly4_mul(col, [0x02, 0x01, 0x01, 0x03])
        assert oracle.inv_mix_column(col).tolist() == _poly4_mul(col, [0x0E, 0x09, 0x0D, 0x0B])
        assert oracle.inv_mix_column(oracle.mix_column(col)).tolist() == col


# ----------------------------------------------------------------- block cipher

@pytest.mark.parametrize("klen", [16, 24, 32])
def test_block_cipher_vs_openssl(klen):
    rng = np.random.default_rng(klen)
    for _ in range(64):
        key = rng.integers(0, 256, klen, dtype=np.uint8).tobytes()
        blk = rng.integers(0, 256, 16, dtype=np.uint8).tobytes()
        enc = Cipher(algorithms.AES(key), modes.ECB()).encryptor()
        ref = enc.update(blk) + enc.finalize()
        assert oracle.block(key, 0, blk) == ref
        assert oracle.block(key, 1, ref) == blk


def test_key_expansion_prefix_and_length():
    for klen, nr in ((16, 10), (24, 12), (32, 14)):
        key = bytes(range(klen))
        ks = oracle.key_expansion(key)
        assert ks.shape == (4 * (nr + 1), 4)
        assert ks[: klen // 4].tobytes() == key       # first Nk words are the key


@pytest.mark.parametrize("klen", [16, 32])
def test_ecb_vs_openssl(klen):
    key = w.single_key(11, klen * 8)
    data = w.seeded_bytes(11, w.STREAM_DATA, 1 << 16)
    enc = Cipher(algorithms.AES(key), modes.ECB()).encryptor()
    ref = enc.update(data.tobytes()) + enc.finalize()
    assert oracle.ecb(key, 0, data).tobytes() == ref
    assert np.array_equal(oracle.ecb(key, 1, np.frombuffer(ref, np.uint8)), data)


# ----------------------------------------------------------------- XTS

def _gf128_mul_xj(t: bytes, j: int) -> bytes:
    """t * x^j in GF(2^128) mod x^128 + x^7 + x^2 + x + 1, by brute force on ints."""
    v = int.from_bytes(t, "little") << j
    poly = (1 << 128) | 0x87
    for deg in range(v.bit_length() - 1, 127, -1):
        if (v >> deg) & 1:
            v ^= poly << (deg - 128)
    return v.to_bytes(16, "little")


def test_xts_alpha_step_vs_bruteforce():
    rng = np.random.default_rng(3)
    for _ in range(8):
        t0 = rng.integers(0, 256, 16, dtype=np.uint8).tobytes()
        t = t0
        for j in range(1, 300):
            t = oracle.xts_mul_alpha(t)
            assert t == _gf128_mul_xj(t0, j)
    # the carry out of byte 15 folds back as 0x87
    assert oracle.xts_mul_alpha(bytes(15) + b"\x80") == b"\x87" + bytes(15)


def _openssl_xts(key, dir, data: bytes, du, first):
    out = bytearray()
    for u in range(len(data) // du):
        tw = (first + u).to_bytes(16, "little")
        c = Cipher(algorithms.AES(key), modes.XTS(tw))
        op = c.encryptor() if dir == 0 else c.decryptor()
        out += op.update(data[u * du:(u + 1) * du]) + op.finalize()
    return bytes(out)


@pytest.mark.parametrize("bits,du,first", [(256, 4096, 0), (128, 4096, 0), (256, 512, 0),
                                           (128, 512, 2**40 + 12345), (256, 16, 7),
                                           (256, 4112, 3), (128, 48, 2**63 - 5)])
def test_xts_vs_openssl(bits, du, first):
    key = w.xts_key(5, bits)
    n = du * 24
    data = w.seeded_bytes(5, w.STREAM_DATA, n)
    c = oracle.xts(key, 0, data, du, first)
    assert c.tobytes() == _openssl_xts(key, 0, data.tobytes(), du, first)
    p = oracle.xts(key, 1, c, du, first)
    assert np.array_equal(p, data)


def test_xts_config1_vs_openssl():
    """1 MiB = 256 x 4096-B sectors, AES-256-XTS, sectors 0..255."""
    key = w.xts_key(1, 256)
    data = w.seeded_bytes(1, w.STREAM_DATA, 1 << 20)
    c = oracle.xts(key, 0, data, 4096, 0)
    assert c.tobytes() == _openssl_xts(key, 0, data.tobytes(), 4096, 0)


def test_xts_rejects():
    key = w.xts_key(1, 256)
    d = np.zeros(4096, np.uint8)
    with pytest.raises(oracle.OracleError):
        oracle.xts(key[:32] + key[:32], 0, d, 4096)    # K1 == K2
    with pytest.raises(oracle.OracleError):
        oracle.xts(key, 0, d[:4000], 4096)              # not a whole data unit
    with pytest.raises(oracle.OracleError):
        oracle.xts(key, 0, d, 24)                       # 4096 is not a whole number of 24-B units
    with pytest.raises(oracle.OracleError):
        oracle.xts(key, 0, d[:4088], 8)                 # a unit shorter than one block
    with pytest.raises(oracle.OracleError):
        oracle.xts(key[:48], 0, d, 4096)                # bad key length


@pytest.mark.parametrize("bits", [128, 256])
@pytest.mark.parametrize("du,first", [(17, 0), (31, 5), (33, 2**40), (100, 7), (527, 2**63 - 3), (4100, 11)])
def test_xts_ciphertext_stealing_vs_openssl(bits, du, first):
    """IEEE 1619 5.3.2 / 5.4.2: a unit ending in a partial block steals the tail
    of the previous block's ciphertext; OpenSSL implements the same rule."""
    key = w.xts_key(6, bits)
    data = w.seeded_bytes(6 + du, w.STREAM_DATA, du * 13)
    c = oracle.xts(key, 0, data, du, first)
    assert c.tobytes() == _openssl_xts(key, 0, data.tobytes(), du, first)
    assert oracle.xts(key, 1, c, du, first).tobytes() == data.tobytes()
    assert oracle.xts(key, 1, c, du, first).tobytes() == _openssl_xts(key, 1, c.tobytes(), du, first)
    # in place, threaded
    buf = data.copy()
    oracle.xts(key, 0, buf, du, first, out=buf, nthreads=5)
    assert np.array_equal(buf, c)


def test_xts_in_place_and_threads():
    key = w.xts_key(2, 128)
    data = w.seeded_bytes(2, w.STREAM_DATA, 64 * 512)
    ref = oracle.xts(key, 0, data, 512, 9, nthreads=1)
    buf = data.copy()
    oracle.xts(key, 0, buf, 512, 9, out=buf, nthreads=7)
    assert np.array_equal(buf, ref)


# ----------------------------------------------------------------- CBC

def _openssl_cbc(key, dir, data: bytes, page, ivs):
    out = bytearray()
    for p in range(len(data) // page):
        c = Cipher(algorithms.AES(key), modes.CBC(ivs[p].tobytes()))
        op = c.encryptor() if dir == 0 else c.decryptor()
        out += op.update(data[p * page:(p + 1) * page]) + op.finalize()
    return bytes(out)


@pytest.mark.parametrize("bits,page", [(128, 4096), (256, 4096), (128, 512), (128, 16), (256, 4112)])
def test_cbc_vs_openssl(bits, page):
    key = w.single_key(8, bits)
    npages = 20
    data = w.seeded_bytes(8, w.STREAM_DATA, page * npages)
    ivs = w.page_ivs(8, npages)
    c = oracle.cbc(key, 0, data, page, ivs)
    assert c.tobytes() == _openssl_cbc(key, 0, data.tobytes(), page, ivs)
    p = oracle.cbc(key, 1, c, page, ivs)
    assert np.array_equal(p, data)
    assert p.tobytes() == _openssl_cbc(key, 1, c.tobytes(), page, ivs)


def test_cbc_decrypt_in_place():
    key = w.single_key(9, 128)
    data = w.seeded_bytes(9, w.STREAM_DATA, 4096 * 8)
    ivs = w.page_ivs(9, 8)
    c = oracle.cbc(key, 0, data, 4096, ivs)
    buf = c.copy()
    oracle.cbc(key, 1, buf, 4096, ivs, out=buf)
    assert np.array_equal(buf, data)


def test_cbc_parallel_form_equals_chain():
    """P_i = D(C_i) xor C_{i-1}: the block-parallel reading of SP 800-38A 6.2
    (what the GPU decrypt computes) equals the oracle's sequential chain."""
    key = w.single_key(10, 128)
    data = w.seeded_bytes(10, w.STREAM_DATA, 4096 * 2)
    ivs = w.page_ivs(10, 2)
    c = oracle.cbc(key, 0, data, 4096, ivs)
    d = oracle.ecb(key, 1, c).reshape(-1, 16)
    prev = np.concatenate([ivs[:, None, :], c.reshape(2, 256, 16)[:, :-1, :]], axis=1).reshape(-1, 16)
    assert np.array_equal((d ^ prev).reshape(-1), data)


# ----------------------------------------------------------------- stored digests

def test_golden_digests_match_openssl():
    """The stored oracle digests (tests/golden/oracle_digests.json, written by
    tests/golden/make_golden.py from the oracle) agree with OpenSSL."""
    import hashlib
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_digests.json")
    gold = json.load(open(path))
    d1 = w.seeded_bytes(1, w.STREAM_DATA, 1 << 20).tobytes()
    assert hashlib.sha256(_openssl_xts(w.xts_key(1, 256), 0, d1, 4096, 0)).hexdigest() == gold["xts256_1mib"]
    d2 = w.seeded_bytes(2, w.STREAM_DATA, 64 * 512).tobytes()
    assert hashlib.sha256(_openssl_xts(w.xts_key(2, 128), 0, d2, 512, 1000)).hexdigest() == gold["xts128_512"]
    d3 = w.seeded_bytes(2, w.STREAM_DATA, 64 * 4096).tobytes()
    ivs = w.page_ivs(2, 64)
    k = w.single_key(2, 128)
    assert hashlib.sha256(_openssl_cbc(k, 0, d3, 4096, ivs)).hexdigest() == gold["cbc128_enc"]
    assert hashlib.sha256(_openssl_cbc(k, 1, d3, 4096, ivs)).hexdigest() == gold["cbc128_dec"]
