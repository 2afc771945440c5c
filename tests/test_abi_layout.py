"""The Python binding agrees with include/fgk.h without a GPU: every report
struct has the same field offsets and size in ctypes as the C compiler gives
it from the header, and every function's ctypes argtypes/restype match the
prototype's parameter kinds (pointer, or integer/float of the same width and
signedness), with typed pointers naming the same pointee."""

import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fgk.h")

STRUCTS = ["fgk_cg_info", "fgk_precond_report", "fgk_slq_report", "fgk_grad_report", "fgk_plan_info"]
# opaque handles, streams and callbacks: pointers on both sides
POINTER_TYPEDEFS = {"fgk_stream_t", "fgk_handle", "fgk_precond", "fgk_batch", "fgk_alloc_fn", "fgk_free_fn"}
SCALARS = {"int": ("i", 4), "int32_t": ("i", 4), "int64_t": ("i", 8), "uint32_t": ("u", 4), "uint64_t": ("u", 8),
           "size_t": ("u", 8), "double": ("f", 8), "float": ("f", 4), "uint8_t": ("u", 1), "char": ("c", 1)}
CTYPES_CODES = {"i": ("i", 4), "l": ("i", 8), "q": ("i", 8), "I": ("u", 4), "L": ("u", 8), "Q": ("u", 8),
                "d": ("f", 8), "f": ("f", 4), "B": ("u", 1), "b": ("i", 1), "c": ("c", 1)}


def _fgk():
    from paper_2508_01864_gb300 import fgk

    return fgk


@pytest.fixture(scope="module")
def lib():
    from paper_2508_01864_gb300 import build

    build.build()
    return _fgk().load()


def _c_layout(tmp_path):
    """sizeof and offsetof of every binding field, as gcc lays out the header's structs."""
    fgk = _fgk()
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "fgk.h"', "int main(void) {"]
    for s in STRUCTS:
        lines.append(f'printf("{s} sizeof %zu\\n", sizeof({s}));')
        for name, _ in getattr(fgk, s)._fields_:
            lines.append(f'printf("{s} {name} %zu\\n", offsetof({s}, {name}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {(a, b): int(c) for a, b, c in (ln.split() for ln in out.splitlines())}


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs a C compiler")
def test_report_structs_have_the_header_layout(tmp_path):
    fgk = _fgk()
    layout = _c_layout(tmp_path)
    for s in STRUCTS:
        cls = getattr(fgk, s)
        assert ctypes.sizeof(cls) == layout[(s, "sizeof")], s
        for name, _ in cls._fields_:
            assert getattr(cls, name).offset == layout[(s, name)], (s, name)


def _prototypes():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    src = re.sub(r"typedef[^;]*;", "", src)  # callback typedefs look like prototypes
    out = {}
    for ret, name, args in re.findall(r"([A-Za-z_][\w\s\*]*?)\b(fgk_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", src, re.S):
        params = [] if args.strip() in ("", "void") else [" ".join(a.split()) for a in args.split(",")]
        out[name] = (" ".join(ret.split()), params)
    return out


def _c_kind(decl: str, with_name: bool):
    """('p', pointee or None) for a pointer, else the scalar's (kind, width)."""
    decl = decl.replace("const", " ")
    if "*" in decl:
        base = decl.split("*")[0].split()
        stars = decl.count("*")
        return ("p", base[-1] if stars == 1 else None)
    words = decl.split()
    base = words[-2] if with_name else words[-1]
    if base in POINTER_TYPEDEFS:
        return ("p", None)
    return SCALARS[base]


def _ctypes_kind(t):
    if t is None:
        return ("void", 0)
    if t in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(t, ctypes._CFuncPtr):
        return ("p", None)
    if issubclass(t, ctypes._Pointer):
        return ("p", t._type_)
    return CTYPES_CODES[t._type_]


def _same_pointee(c_pointee, py_pointee):
    if py_pointee is None or c_pointee is None:
        return True  # void*, an opaque handle or a pointer to pointers: passed as an address
    if isinstance(py_pointee, type) and issubclass(py_pointee, ctypes.Structure):
        return py_pointee.__name__ == c_pointee
    if c_pointee in POINTER_TYPEDEFS:
        return py_pointee is ctypes.c_void_p
    return c_pointee in SCALARS and _ctypes_kind(py_pointee) == SCALARS[c_pointee]


def test_binding_signatures_match_the_header(lib):
    protos = _prototypes()
    assert sorted(protos) == sorted(_fgk().EXPORTS)
    for name, (ret, params) in protos.items():
        f = getattr(lib, name)
        assert f.argtypes is not None, name
        assert len(f.argtypes) == len(params), name
        for i, (p, t) in enumerate(zip(params, f.argtypes)):
            ck, pk = _c_kind(p, with_name=True), _ctypes_kind(t)
            assert ck[0] == pk[0], (name, i, p, t)
            if ck[0] == "p":
                assert _same_pointee(ck[1], pk[1]), (name, i, p, t)
            else:
                assert ck == pk, (name, i, p, t)
        rk = _c_kind(ret, with_name=False)
        assert rk[0] == _ctypes_kind(f.restype)[0], (name, ret, f.restype)
        if rk[0] != "p":
            assert rk == _ctypes_kind(f.restype), (name, ret, f.restype)


def test_a_planted_mismatch_is_caught():
    """The comparison itself: a 32-bit integer where the header has int64_t,
    and a struct pointer of the wrong type, are both told apart."""
    fgk = _fgk()
    assert _c_kind("int64_t N", True) != _ctypes_kind(ctypes.c_int32)
    assert _c_kind("size_t n", True) != _ctypes_kind(ctypes.c_int64)
    assert not _same_pointee("fgk_cg_info", fgk.fgk_plan_info)
    assert not _same_pointee("double", ctypes.c_float)
    assert _same_pointee("fgk_cg_info", fgk.fgk_cg_info)
