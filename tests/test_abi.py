"""The C ABI library builds, loads without a GPU and exports every function declared in include/gbmg.h."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", text, flags=re.M):
            name = m.group(1)
            if name not in ("if", "while", "for", "sizeof") and not name.isupper():
                names.append(name)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2607_10983_gb300 import _build
    return _build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mg_setup", "mg_solve", "mg_destroy", "mg_solve_host"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_bad_arguments_without_gpu(libpath):
    import paper_2607_10983_gb300 as pkg
    L = pkg.lib()
    for code in range(8):
        assert L.mg_status_string(code)
    # argument validation happens before any CUDA call
    ctx = ctypes.c_void_p()
    assert L.mg_setup(ctypes.byref(ctx), 2, 8, 8, 0, 3, None, None) == 1
    assert b"must be >= 4" in L.mg_last_error()
    assert L.mg_setup(None, 8, 8, 8, 0, 3, None, None) == 1
    assert L.mg_solve(None, None, None, None, 1e-6, 10, None) == 1
    assert L.mg_solve_host_sequence(None, 0, None, None, None, 1e-6, 10, None) == 1


def test_python_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2607_10983_gb300 as pkg
    monkeypatch.setattr(pkg, "_LIB", None)
    monkeypatch.setattr(pkg._build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        pkg.lib()
