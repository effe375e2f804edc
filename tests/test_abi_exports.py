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


def declared_prototypes():
    """{name: (return type, [parameter declarations])} from include/*.h."""
    out = {}
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            for ret, name, params in re.findall(r"([A-Za-z_][\w \t*]*?)\b(kgpu_[a-z0-9_]+)\s*\(([^()]*)\)\s*;",
                                                text):
                ps = [" ".join(p.split()) for p in params.split(",")]
                out[name] = (" ".join(ret.split()), [] if ps == ["void"] else ps)
    return out


def c_kind(decl):
    """'p' (a pointer), 'i64' or 'i32' for a C parameter or return type."""
    if "*" in decl:
        return "p"
    words = decl.replace("const ", "").split()
    t = " ".join(words[:-1]) if len(words) > 1 and words[-1] not in ("int",) else " ".join(words)
    if t in ("kgpu_stream", "kgpu_done_fn"):
        return "p"
    if t in ("uint64_t", "int64_t", "size_t", "kgpu_ticket"):
        return "i64"
    if t in ("int", "uint32_t", "int32_t", "kgpu_key", "unsigned", "unsigned int"):
        return "i32"
    raise AssertionError(f"unclassified C type in {decl!r}")


def py_kind(t):
    if t in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(t, (ctypes._Pointer, ctypes._CFuncPtr)):
        return "p"
    if ctypes.sizeof(t) == 8:
        return "i64"
    if ctypes.sizeof(t) == 4:
        return "i32"
    raise AssertionError(f"unclassified ctypes type {t!r}")


def test_binding_signatures_match_the_prototypes():
    """Each function the binding calls takes, position by position, the
    argument kinds (pointer, 64-bit or 32-bit integer) its prototype gives,
    and returns the declared kind."""
    import paper_1305_3345_gb300 as kg
    L = kg.lib()
    protos = declared_prototypes()
    assert set(protos) == set(declared_functions())
    checked = 0
    for name, (ret, params) in protos.items():
        f = getattr(L, name)
        if f.argtypes is None:  # not called through the binding
            continue
        assert [py_kind(a) for a in f.argtypes] == [c_kind(p) for p in params], name
        assert py_kind(f.restype) == c_kind(ret + " r"), name
        checked += 1
    assert checked >= 30
