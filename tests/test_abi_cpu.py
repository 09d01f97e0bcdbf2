"""CPU checks of the C-ABI boundary: the library builds, loads without a GPU,
exports every entry point include/hbx.h declares, and the Python binding has
the same names.  The product package must not reach the oracle, and must fail
loudly when its CUDA library is missing."""
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hbx.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hbx_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_2208_00613_gb300 as hbx
    hbx.build()
    return hbx.lib()


def test_header_declares_entry_points():
    names = declared()
    for must in ["hbx_create", "hbx_set_allocator", "hbx_graph_create", "hbx_imm", "hbx_submit", "hbx_wait",
                 "hbx_pool_export_set", "hbx_graph_destroy", "hbx_destroy", "hbx_strerror"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing


def test_binding_has_same_names(lib):
    import paper_2208_00613_gb300 as hbx
    for n in declared():
        assert hasattr(hbx, n), n


def test_no_compute_without_gpu(lib):
    import ctypes
    import paper_2208_00613_gb300 as hbx
    assert lib.hbx_strerror(-5).decode().startswith("LT in-weights")
    o = hbx.hbx_default_options()
    assert o.density_cut == 32 and o.encode == 1 and o.form == 1
    h = ctypes.c_void_p()
    # with no GPU visible the context cannot be created and the call says so
    import torch
    if not torch.cuda.is_available():
        assert lib.hbx_create(ctypes.byref(h), 0, None) == -1


def test_missing_library_fails_loudly(tmp_path):
    code = ("import paper_2208_00613_gb300 as h; h.LIB_PATH = '/nonexistent/libhbx.so'; h._lib = None\n"
            "try:\n    h.lib()\nexcept ImportError as e:\n    print('raised', e)\n")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT)
    assert "raised" in r.stdout


def test_product_never_reaches_oracle():
    pkg = os.path.join(ROOT, "paper_2208_00613_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", txt, re.M), f
                assert "liboracle" not in txt and "oracle.cpp" not in txt, f


def _arities():
    """Parameter count of every function include/hbx.h declares."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for name, params in re.findall(r"\b(hbx_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S):
        p = params.strip()
        # commas inside function-pointer parameters belong to those parameters
        depth, count = 0, 0 if p in ("", "void") else 1
        for ch in p:
            depth += ch == "("
            depth -= ch == ")"
            count += ch == "," and depth == 0
        out[name] = count
    return out


def test_binding_argtypes_match_header(lib):
    ar = _arities()
    assert len(ar) >= 20
    for name, n in ar.items():
        f = getattr(lib, name)
        assert f.argtypes is not None, name
        assert len(f.argtypes) == n, (name, len(f.argtypes), n)


def test_struct_layout_matches_header(lib, tmp_path):
    """The binding's ctypes structs against the C compiler's layout of the
    header's structs: sizes and every field offset."""
    import ctypes
    import paper_2208_00613_gb300 as hbx
    fields = {"hbx_options": [f for f, _ in hbx.hbx_options._fields_],
              "hbx_stats": [f for f, _ in hbx.hbx_stats._fields_]}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "hbx.h"', "int main(void) {"]
    for st, fs in fields.items():
        lines.append(f'printf("{st} size %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'printf("{st} {f} %zu\\n", offsetof({st}, {f}));')
    lines += ["return 0;", "}"]
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        st, key, val = line.split()
        got[(st, key)] = int(val)
    for st, cls in (("hbx_options", hbx.hbx_options), ("hbx_stats", hbx.hbx_stats)):
        assert got[(st, "size")] == ctypes.sizeof(cls), st
        for f in fields[st]:
            assert got[(st, f)] == getattr(cls, f).offset, (st, f)
