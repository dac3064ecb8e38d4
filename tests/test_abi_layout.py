"""The Python binding against the C ABI's header, without a GPU: the ctypes
mirrors of its structs (qh_opts, qh_result, qh_debug_record) have the
header's fields, in its order, at the offsets and total size a C compiler
gives them (a field added to one side only would shift every later field of
every call that passes the struct), and every function's ctypes signature
has the prototype's arity and, per argument and result, its ABI class
(pointer, 32-bit, 64-bit integer, size_t)."""
import ctypes
import os
import re
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qh.h")
CTYPE = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64}


def _header_fields(name):
    src = open(HEADER).read()
    m = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), src, re.S)
    assert m, name
    body = re.sub(r"/\*.*?\*/", "", m.group(1), flags=re.S)
    out = []
    for t, decl in re.findall(r"(\w+)\s+([^;]+);", body):
        for d in decl.split(","):
            f, n = re.fullmatch(r"\s*(\w+)\s*(?:\[(\d+)\])?\s*", d).groups()
            out.append((f, t, int(n) if n else 0))
    return out


def _mirror(name):
    from paper_1201_2936_gb300 import _native
    return {"qh_opts": _native.QhOpts, "qh_result": _native.QhResult,
            "qh_debug_record": _native.QhDebugRecord}[name]


NAMES = ["qh_opts", "qh_result", "qh_debug_record"]


@pytest.mark.parametrize("name", NAMES)
def test_mirror_has_the_header_fields_in_order(name):
    fields = _header_fields(name)
    mirror = _mirror(name)
    assert [f for f, _, _ in fields] == [f for f, _ in mirror._fields_]
    for (f, t, n), (_, ct) in zip(fields, mirror._fields_):
        want = CTYPE[t] * n if n else CTYPE[t]
        assert ctypes.sizeof(ct) == ctypes.sizeof(want), f
        base = ct._type_ if n else ct
        assert base == CTYPE[t], f


def test_offsets_and_sizes_match_the_c_compiler():
    cc = shutil.which("gcc") or shutil.which("cc")
    cuda_inc = "/usr/local/cuda/include"
    if not cc or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime_api.h")):
        pytest.skip("no C compiler or CUDA headers")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "qh.h"', "int main(void) {"]
    for name in NAMES:
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for f, _, _ in _header_fields(name):
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines += ["return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        c, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(c, "w").write("\n".join(lines) + "\n")
        subprocess.run([cc, "-I", os.path.join(ROOT, "include"), "-I", cuda_inc, c, "-o", exe],
                       check=True, capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    got = {}
    for ln in out.splitlines():
        name, key, val = ln.split()
        got[(name, key)] = int(val)
    for name in NAMES:
        mirror = _mirror(name)
        assert got[(name, "size")] == ctypes.sizeof(mirror), name
        for f, _ in mirror._fields_:
            assert got[(name, f)] == getattr(mirror, f).offset, (name, f)


def _prototypes():
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    src = "\n".join(ln for ln in src.splitlines() if not ln.lstrip().startswith("#"))
    protos = {}
    for ret, name, params in re.findall(r"([A-Za-z_][\w\s\*]*?)\b(qh_\w+)\s*\(([^()]*)\)\s*;",
                                        src):
        ps = [p.strip() for p in params.split(",")] if params.strip() not in ("", "void") else []
        protos[name] = (" ".join(ret.split()), ps)
    return protos


def _kind(decl):
    """ABI class of a C parameter or return type: pointer, int32, int64,
    size, or void."""
    d = " ".join(decl.replace("*", " * ").split())
    if "*" in d or d.split()[0] == "cudaStream_t":
        return "ptr"
    base = [t for t in d.split() if t not in ("const",)][0]
    return {"int32_t": "i32", "int": "i32", "qh_status": "i32", "int64_t": "i64",
            "size_t": "size", "void": "void"}[base]


def _ctype_kind(t):
    if t is None:
        return "void"
    if t in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(t, ctypes._Pointer):
        return "ptr"
    if t in (ctypes.c_int32, ctypes.c_int):
        return "i32"
    if t is ctypes.c_size_t:
        return "size"
    if t is ctypes.c_int64:
        return "i64"
    raise AssertionError(t)


def test_binding_signatures_match_the_prototypes():
    from paper_1201_2936_gb300 import _native
    protos = _prototypes()
    assert set(protos) == set(_native.exported_names())
    for name, res, args in _native.SIGNATURES:
        ret, params = protos[name]
        assert _ctype_kind(res) == _kind(ret), name
        assert len(args) == len(params), (name, len(args), params)
        for i, (a, p) in enumerate(zip(args, params)):
            assert _ctype_kind(a) == _kind(p), (name, i, p)
