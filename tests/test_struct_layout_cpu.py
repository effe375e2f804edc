"""The Python binding's copies of the C ABI's structs (ctypes structures and the
numpy record of kgpu_request) have the layout include/kgpu.h gives them: the
same size, and each field at the same offset with the same width.  A C
program generated from the binding's field lists prints sizeof and offsetof
as gcc lays the header out; a field the header lacks fails to compile."""
import ctypes
import os
import shutil
import subprocess

import pytest

import paper_1305_3345_gb300 as kg

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

STRUCTS = {
    "kgpu_request": kg.KgpuRequest,
    "kgpu_tuning": kg.KgpuTuning,
    "kgpu_serve_config": kg.KgpuServeConfig,
    "kgpu_serve_stats": kg.KgpuServeStats,
    "kgpu_config": kg.KgpuConfig,
    "kgpu_crossover": kg.KgpuCrossover,
    "kgpu_dispatch_point": kg.KgpuDispatchPoint,
}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc")
    if not cc:
        pytest.skip("gcc is not available")
    d = tmp_path_factory.mktemp("layout")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "kgpu.h"', "int main(void) {"]
    for name, cls in STRUCTS.items():
        lines.append(f'  printf("{name} . %zu %zu\\n", sizeof({name}), (size_t)0);')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu %zu\\n", offsetof({name}, {field}), '
                         f'sizeof((({name} *)0)->{field}));')
    lines += ["  return 0;", "}"]
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = str(d / "layout")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", exe], check=True)
    out = {}
    for line in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.splitlines():
        name, field, a, b = line.split()
        out[(name, field)] = (int(a), int(b))
    return out


@pytest.mark.parametrize("name", list(STRUCTS))
def test_ctypes_layout_matches_the_header(c_layout, name):
    cls = STRUCTS[name]
    assert ctypes.sizeof(cls) == c_layout[(name, ".")][0]
    for field, _ in cls._fields_:
        desc = getattr(cls, field)
        assert (desc.offset, desc.size) == c_layout[(name, field)], field


def test_request_record_matches_the_header(c_layout):
    dt = kg.request_dtype()
    assert dt.itemsize == c_layout[("kgpu_request", ".")][0]
    assert list(dt.names) == [f for f, _ in kg.KgpuRequest._fields_]
    for field in dt.names:
        sub, off = dt.fields[field][:2]
        assert (off, sub.itemsize) == c_layout[("kgpu_request", field)], field
