"""Plants plausible mistakes in a copy of the oracle (on the CPU) and checks that
the library cross-checks used as pins catch every one of them.

Each mutant is a one-token edit of aes_oracle.c, compiled to a temporary shared
object; the original source is never modified.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import workloads as w

crypto = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
Cipher, algorithms, modes = crypto.Cipher, crypto.algorithms, crypto.modes

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "aes_oracle.c")

MUTANTS = {
    "tweak_poly": ("t[0] ^= 0x87;", "t[0] ^= 0x86;"),
    "tweak_big_endian": ("ival[k] = (uint8_t)(sector >> (8 * k));", "ival[15 - k] = (uint8_t)(sector >> (8 * k));"),
    "state_transposed": ("s[r][c] = in[r + 4 * c];", "s[r][c] = in[4 * r + c];"),
    "field_modulus": ("if (hi) r ^= 0x1b;", "if (hi) r ^= 0x1d;"),
    "shift_rows_direction": ("row[c] = s[r][(c + r) % 4];", "row[c] = s[r][(c + 4 - r) % 4];"),
    "aes256_subword_dropped": ("nk > 6 && i % nk == 4", "nk > 8 && i % nk == 4"),
    "cbc_chain_plaintext": ("memcpy(prev, y, 16);", "memcpy(prev, x, 16);"),
    "affine_constant": ("((0x63 >> i) & 1)", "((0x62 >> i) & 1)"),
    "rcon_step": ("rcon = xtime(rcon);", "rcon = (uint8_t)(rcon + 1);"),
    "mixcol_coeff": ("oracle_gf_mul(3, a1) ^ a2 ^ a3);", "oracle_gf_mul(2, a1) ^ a2 ^ a3);"),
    "cts_first_tweak": ("xts_block(jb, 0, last, x, t);", "xts_block(jb, 0, last, x, t_last);"),
    "cts_second_tweak": ("xts_block(jb, 0, y, out + 16 * (m - 1), t_last);",
                         "xts_block(jb, 0, y, out + 16 * (m - 1), t);"),
}


def _build(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-pthread", str(path), "-o", str(so)])
    lib = ctypes.CDLL(str(so))
    v = ctypes.c_void_p
    lib.oracle_xts.argtypes = [v, ctypes.c_int, ctypes.c_int, v, v, ctypes.c_size_t, ctypes.c_size_t,
                               ctypes.c_uint64, ctypes.c_int]
    lib.oracle_cbc.argtypes = [v, ctypes.c_int, ctypes.c_int, v, v, ctypes.c_size_t, ctypes.c_size_t, v,
                               ctypes.c_int]
    return lib


def _pins_pass(lib) -> bool:
    """The same library cross-checks the real oracle passes."""
    ok = True
    for bits in (128, 256):
        key = w.xts_key(21, bits)
        data = w.seeded_bytes(21, w.STREAM_DATA, 2 * 512)
        out = np.zeros_like(data)
        lib.oracle_xts(key, len(key), 0, data.ctypes.data, out.ctypes.data, data.size, 512, 300, 1)
        ref = b""
        for u in range(2):
            c = Cipher(algorithms.AES(key), modes.XTS((300 + u).to_bytes(16, "little"))).encryptor()
            ref += c.update(data[u * 512:(u + 1) * 512].tobytes()) + c.finalize()
        ok &= out.tobytes() == ref
        # ciphertext stealing: units of 2 full blocks and 1 byte
        cts = data[: 2 * 33]
        out2 = np.zeros_like(cts)
        lib.oracle_xts(key, len(key), 0, cts.ctypes.data, out2.ctypes.data, cts.size, 33, 300, 1)
        ref = b""
        for u in range(2):
            c = Cipher(algorithms.AES(key), modes.XTS((300 + u).to_bytes(16, "little"))).encryptor()
            ref += c.update(cts[u * 33:(u + 1) * 33].tobytes()) + c.finalize()
        ok &= out2.tobytes() == ref
        k1 = key[: bits // 8]
        ivs = w.page_ivs(21, 2)
        lib.oracle_cbc(k1, len(k1), 0, data.ctypes.data, out.ctypes.data, data.size, 512, ivs.ctypes.data, 1)
        ref = b""
        for p in range(2):
            c = Cipher(algorithms.AES(k1), modes.CBC(ivs[p].tobytes())).encryptor()
            ref += c.update(data[p * 512:(p + 1) * 512].tobytes()) + c.finalize()
        ok &= out.tobytes() == ref
    return ok


def test_unmutated_copy_passes(tmp_path):
    lib = _build(tmp_path, "none", "#define OR_OK 0", "#define OR_OK 0")
    assert _pins_pass(lib)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    lib = _build(tmp_path, name, old, new)
    assert not _pins_pass(lib), f"pins did not catch mutant {name}"
