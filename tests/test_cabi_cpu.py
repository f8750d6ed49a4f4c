"""CPU-side checks of the boundary: the library builds for sm_103a, loads,
and exports every entry point include/hot_mpm.h declares; the binding's
struct layouts match the header's sizes."""
import ctypes
import os
import re

import pytest

from paper_1911_07913_gb300 import build as B
from paper_1911_07913_gb300 import hot

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hot_mpm.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:mpm_status|const char \*|int64_t)\s*(mpm_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    return B.build()


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(hot.EXPORTED)


def test_struct_sizes_match_header(lib_path):
    # sizes follow from the C layout rules on LP64 (x86-64 and aarch64 alike)
    assert ctypes.sizeof(hot.mpm_material) == 40
    assert ctypes.sizeof(hot.mpm_bc) == 8 + 12 * 8 + 8 + 8
    assert ctypes.sizeof(hot.mpm_solver_opts) == 8 + 8 * 4 + 3 * 8 + 8 + 8
    assert ctypes.sizeof(hot.mpm_step_stats) == 16 + 24 + 8 + 128 + 8 + 8


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(hot, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(hot, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        hot.load()


def test_struct_field_offsets_match_header(tmp_path):
    """Every field of every ctypes structure in the binding sits at the offset
    a C compiler gives the field of the same name in include/hot_mpm.h, and
    every structure has the C size: a field added, dropped, retyped or moved
    on one side only fails here."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [hot.mpm_material, hot.mpm_bc, hot.mpm_scene_desc, hot.mpm_solver_opts, hot.mpm_step_stats]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "hot_mpm.h"', "int main(void) {"]
    for st in structs:
        name = st.__name__
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in st._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "offsets.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "offsets"
    include = os.path.join(ROOT, "include")
    subprocess.run([cc, "-std=c99", "-I", include, str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines()
    c_layout = {(a, b): int(c) for a, b, c in (l.split() for l in out)}
    for st in structs:
        name = st.__name__
        assert c_layout[(name, "sizeof")] == ctypes.sizeof(st), name
        for field, _ in st._fields_:
            assert c_layout[(name, field)] == getattr(st, field).offset, (name, field)


def test_binding_argument_counts_match_header():
    """The binding declares argument types for every function of
    include/hot_mpm.h, as many as the header's prototype takes (an untyped
    call would pass Python integers as C int)."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    protos = {}
    for m in re.finditer(r"^\s*(?:mpm_status|const char \*|int64_t|void)\s*(mpm_\w+)\s*\(([^)]*)\)\s*;", src,
                         flags=re.M | re.S):
        params = m.group(2).strip()
        protos[m.group(1)] = 0 if params in ("", "void") else len(params.split(","))
    lib = hot.load()
    checked = 0
    for name, n in protos.items():
        fn = getattr(lib, name)
        assert fn.argtypes is not None, name
        assert len(fn.argtypes) == n, (name, len(fn.argtypes), n)
        checked += 1
    assert checked == len(declared_functions())


def test_null_handles_are_rejected_without_a_device():
    """Argument marshalling of the residency and wait-limit calls: a NULL
    scene or server is refused with MPM_ERR_INVALID_ARG before any CUDA call."""
    lib = hot.load()
    invalid = 1
    assert lib.mpm_scene_park(None) == invalid
    assert lib.mpm_scene_unpark(None) == invalid
    assert lib.mpm_set_wait_limit(None, ctypes.c_int64(1 << 40)) == invalid
    p, b = ctypes.c_int32(7), ctypes.c_int64(7)
    assert lib.mpm_scene_residency(None, ctypes.byref(p), ctypes.byref(b)) == invalid
    w = [ctypes.c_int64(7) for _ in range(5)]
    assert lib.mpm_server_residency(None, *[ctypes.byref(x) for x in w]) == invalid
    assert p.value == 7 and b.value == 7 and all(x.value == 7 for x in w)
