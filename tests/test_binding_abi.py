"""CPU checks that the Python binding describes the C ABI of include/gbmg.h: every
declared function has a ctypes signature with the same number of parameters and the
same kind (pointer, int, long long, double) at each position and the same return kind;
the option and statistics structs have the header's fields in the header's order with
matching types (checked also by size against a C compiler's layout); the status codes
and the binding's convergence statuses match the header's enum."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

import paper_2607_10983_gb300 as gb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbmg.h")


def _header_text():
    text = open(HEADER).read()
    return re.sub(r"/\*.*?\*/", " ", text, flags=re.S)


def _kind_c(decl: str) -> str:
    decl = decl.strip()
    if "*" in decl:
        return "P"
    words = decl.replace("const ", "").split()
    if "double" in words:
        return "D"
    if words[:2] == ["long", "long"]:
        return "LL"
    return "I"  # int and the enum types (gbmg_status and the like)


def _kind_ctypes(t) -> str:
    if t is None:
        return "void"
    if t in (ctypes.c_void_p, ctypes.c_char_p) or hasattr(t, "_type_") and issubclass(t, ctypes._Pointer):
        return "P"
    if t is ctypes.c_double:
        return "D"
    if t is ctypes.c_longlong:
        return "LL"
    if t is ctypes.c_int:
        return "I"
    raise AssertionError(f"unexpected ctypes type {t}")


def _prototypes():
    protos = {}
    for m in re.finditer(r"^\s*([A-Za-z_][\w \*]*?)\s*\b((?:mg|gbmg)_\w+)\s*\(([^)]*)\)\s*;", _header_text(),
                         flags=re.M):
        ret, name, params = m.group(1), m.group(2), m.group(3).strip()
        plist = [] if params in ("", "void") else [p for p in params.split(",")]
        protos[name] = ("void" if ret.strip() == "void" else _kind_c(ret), [_kind_c(p) for p in plist])
    return protos


def test_every_declared_function_has_a_matching_signature():
    protos = _prototypes()
    assert len(protos) >= 40
    assert set(protos) == set(gb._SIGS), set(protos) ^ set(gb._SIGS)
    for name, (ret, params) in protos.items():
        rt, argt = gb._SIGS[name]
        assert _kind_ctypes(rt) == ret, name
        assert [_kind_ctypes(a) for a in argt] == params, name


def _struct_fields(tag: str):
    m = re.search(r"typedef\s+struct\s*\{([^{}]*)\}\s*" + tag + r"\s*;", _header_text())
    assert m, tag
    fields = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        typ, names = decl.split(None, 1)
        for nm in names.split(","):
            nm = nm.strip()
            arr = re.match(r"(\w+)\[(\d+)\]", nm)
            fields.append((arr.group(1), typ, int(arr.group(2))) if arr else (nm, typ, 1))
    return fields


@pytest.mark.parametrize("tag, cls", [("gbmg_opts", gb._Opts), ("gbmg_stats", gb._Stats)])
def test_structs_match_the_header(tag, cls):
    want = _struct_fields(tag)
    got = cls._fields_
    assert [f[0] for f in want] == [g[0] for g in got]
    for (name, typ, n), (_, ct) in zip(want, got):
        base = ct._type_ if n > 1 else ct
        assert (n > 1) == hasattr(ct, "_length_") and (n == 1 or ct._length_ == n), name
        assert base is {"int": ctypes.c_int, "double": ctypes.c_double}[typ], name


@pytest.mark.parametrize("tag, cls", [("gbmg_opts", gb._Opts), ("gbmg_stats", gb._Stats)])
def test_struct_sizes_match_a_c_compiler(tmp_path, tag, cls):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "size.c"
    src.write_text('#include <stdio.h>\n#include "gbmg.h"\nint main(void) { printf("%%zu", sizeof(%s)); return 0; }\n'
                   % tag)
    exe = tmp_path / "size"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    assert int(subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout) == ctypes.sizeof(cls)


def test_status_codes_match_the_header():
    codes = {}
    for m in re.finditer(r"\b(GBMG_(?:OK|ERR_\w+))\s*=\s*(\d+)", _header_text()):
        codes[m.group(1)] = int(m.group(2))
    assert sorted(codes.values()) == sorted(gb.STATUS)
    assert set(gb.CONVERGENCE_STATUSES) == {codes["GBMG_ERR_NOT_CONVERGED"], codes["GBMG_ERR_NONFINITE"],
                                            codes["GBMG_ERR_DIVERGED"]}
