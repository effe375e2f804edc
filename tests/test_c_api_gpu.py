"""The C ABI from a C program alone (tests/c_api_example.c), with no Python
binding and no PyTorch on the path: compiled with gcc against include/kgpu.h
and the in-tree libkgpu.so, run on the GPU, and its two ciphertexts (per-call
AES-256-XTS, batched AES-128-CBC encryption) compared byte for byte with the
oracle.  The program also decrypts the XTS ciphertext through the serving ring
with a completion callback, and checks the plaintext itself."""
import os
import shutil
import subprocess

import pytest

import oracle
import workloads as w

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_c_program_through_the_abi(tmp_path):
    from paper_1305_3345_gb300 import build
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc not available")
    build.build()
    cuda = build.cuda_home()
    cuda_lib = os.path.join(cuda, "lib64")
    exe = str(tmp_path / "c_api_example")
    subprocess.run([gcc, "-O2", "-std=c11", "-pthread", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(cuda, "include"), os.path.join(HERE, "c_api_example.c"), "-o", exe,
                    "-L", build.OUT_DIR, "-lkgpu", "-L", cuda_lib, "-lcudart",
                    f"-Wl,-rpath,{build.OUT_DIR}", f"-Wl,-rpath,{cuda_lib}"], check=True)
    npages = 300
    key64, key16 = w.xts_key(91, 256), w.single_key(91, 128)
    data = w.seeded_bytes(91, w.STREAM_DATA, 4096 * npages)
    ivs = w.page_ivs(91, npages)
    files = {k: str(tmp_path / k) for k in ("k64", "k16", "ivs", "plain", "xts", "cbc")}
    for k, v in (("k64", key64), ("k16", key16), ("ivs", ivs.tobytes()), ("plain", data.tobytes())):
        with open(files[k], "wb") as f:
            f.write(v)
    r = subprocess.run([exe] + [files[k] for k in ("k64", "k16", "ivs", "plain", "xts", "cbc")],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "c_api_example ok" in r.stdout, (r.returncode, r.stdout, r.stderr)
    with open(files["xts"], "rb") as f:
        assert f.read() == oracle.xts(key64, 0, data, 4096, 5).tobytes()
    with open(files["cbc"], "rb") as f:
        assert f.read() == oracle.cbc(key16, 0, data, 4096, ivs).tobytes()
