"""The bitsliced kernel's S-box circuit (csrc/sbox_circuit.cuh) on the CPU.

The committed header is evaluated gate by gate in Python over all 256 inputs
at once (one input per bit of a 256-bit integer) and must equal the oracle's
S-box, which the oracle builds from the field inverse and the affine map.  The
generator must also reproduce the committed header exactly, so the header is
what the generator (and its own exhaustive check) says it is.
"""
import os
import re
import subprocess
import sys

import numpy as np

import oracle

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1305_3345_gb300", "csrc")


def evaluate_header():
    text = open(os.path.join(CSRC, "sbox_circuit.cuh")).read()
    full = (1 << 256) - 1
    env = {f"x{i}": sum(((a >> i) & 1) << a for a in range(256)) for i in range(8)}
    gates = 0
    for name, a, op, b in re.findall(r"const uint32_t (\w+) = (\w+) ([&^]) (\w+);", text):
        env[name] = env[a] & env[b] if op == "&" else env[a] ^ env[b]
        gates += 1
    out = {}
    for i, neg, src in re.findall(r"\bx(\d) = (~?)(\w+);", text):
        v = env[src] if src != "0u" else 0
        out[int(i)] = v ^ full if neg else v
    assert sorted(out) == list(range(8))
    table = [sum(((out[i] >> a) & 1) << i for i in range(8)) for a in range(256)]
    return np.array(table, dtype=np.uint8), gates


def test_circuit_equals_the_sbox():
    table, gates = evaluate_header()
    assert np.array_equal(table, oracle.sbox())
    assert 100 <= gates <= 200


def test_generator_reproduces_the_header():
    r = subprocess.run([sys.executable, os.path.join(CSRC, "gen_sbox_circuit.py"), "--check"],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
