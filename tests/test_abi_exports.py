"""The C-ABI library builds, loads on a host without a GPU, and exports every
function include/kgpu.h declares.  No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(kgpu_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def cdll():
    import paper_1305_3345_gb300 as kg
    return ctypes.CDLL(kg.ensure_built())


def test_header_declares_the_service_calls():
    names = declared_functions()
    for required in ("kgpu_init", "kgpu_destroy", "kgpu_aes_setkey", "kgpu_aes_xts_crypt",
                     "kgpu_aes_cbc_decrypt", "kgpu_aes_cbc_encrypt_pages"):
        assert required in names


def test_every_declared_symbol_is_exported(cdll):
    missing = [n for n in declared_functions() if not hasattr(cdll, n)]
    assert not missing, missing


def test_no_device_calls_fail_cleanly(cdll):
    import paper_1305_3345_gb300 as kg
    assert kg.kgpu_version() >= 0
    assert kg.kgpu_strerror(-22) == "invalid argument"
    ctx = ctypes.c_void_p()
    # device index out of range: KGPU_ENODEV with or without a GPU present
    assert kg.lib().kgpu_init(ctypes.byref(ctx), 4096, None) == -19
    assert not ctx.value
    assert kg.lib().kgpu_destroy(None) == 0


def test_library_has_no_libcuda_link_dependency():
    import subprocess
    import paper_1305_3345_gb300 as kg
    out = subprocess.run(["readelf", "-d", kg.ensure_built()], capture_output=True, text=True).stdout
    needed = re.findall(r"\[(.*?)\]", "\n".join(l for l in out.splitlines() if "NEEDED" in l))
    assert not any(n.startswith("libcuda.so") for n in needed), needed
