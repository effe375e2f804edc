"""Writes tests/golden/oracle_digests.json: SHA-256 digests of oracle outputs on
the seeded small workloads.  Calls only `oracle/` and `workloads/`; rerun it
whenever a workload recipe changes (`python tests/golden/make_golden.py`).

Cases (seeded, synthetic):
  xts256_1mib   AES-256-XTS encrypt, 256 x 4096-B sectors 0..255, seed 1
                (data stream 1, key K1||K2 from the key stream)
  xts128_512    AES-128-XTS encrypt, 64 x 512-B sectors from 1000, seed 2
  cbc128_enc    AES-128-CBC encrypt, 64 x 4096-B pages, per-page IVs, seed 2
  cbc128_dec    AES-128-CBC decrypt of the same bytes, seed 2
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads as w  # noqa: E402


def cases():
    d1 = w.seeded_bytes(1, w.STREAM_DATA, 1 << 20)
    yield "xts256_1mib", oracle.xts(w.xts_key(1, 256), 0, d1, 4096, 0)
    d2 = w.seeded_bytes(2, w.STREAM_DATA, 64 * 512)
    yield "xts128_512", oracle.xts(w.xts_key(2, 128), 0, d2, 512, 1000)
    d3 = w.seeded_bytes(2, w.STREAM_DATA, 64 * 4096)
    ivs = w.page_ivs(2, 64)
    yield "cbc128_enc", oracle.cbc(w.single_key(2, 128), 0, d3, 4096, ivs)
    yield "cbc128_dec", oracle.cbc(w.single_key(2, 128), 1, d3, 4096, ivs)


def main():
    out = {name: hashlib.sha256(buf.tobytes()).hexdigest() for name, buf in cases()}
    with open(os.path.join(HERE, "oracle_digests.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
