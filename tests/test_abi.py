"""Host-side checks of the C ABI: the library builds, loads without a GPU and
exports every function declared in include/fde.h; the Python structs mirror
the C structs field by field. No compute calls (no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fde.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*\*?\s*\**\s*(fde_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def _lib():
    import paper_1907_13428_gb300 as F
    if not os.path.exists(F.LIB_PATH):
        from paper_1907_13428_gb300 import build
        build.build()
    return F, F.lib()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("fde_setup", "fde_matvec", "fde_precond", "fde_admm_solve", "fde_admm_grad", "fde_destroy",
                     "fde_strerror"):
        assert required in names, names


def test_library_exports_every_declared_symbol():
    F, L = _lib()
    for name in _declared_functions():
        assert hasattr(L, name), name
        assert name in F.EXPORTED, f"binding lacks a signature for {name}"


def _struct_fields(name):
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), src, flags=re.S).group(1)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        typ, rest = decl.split(None, 1)
        for f in rest.split(","):
            fields.append((typ, f.strip()))
    return fields


@pytest.mark.parametrize("cname,pyname", [("fde_params", "fde_params"), ("fde_admm_opts", "fde_admm_opts"),
                                          ("fde_admm_stats", "fde_admm_stats")])
def test_python_structs_mirror_header(cname, pyname):
    import paper_1907_13428_gb300 as F
    py = getattr(F, pyname)._fields_
    c = _struct_fields(cname)
    assert [n for n, _ in py] == [n for _, n in c]
    cmap = {"int": ctypes.c_int, "double": ctypes.c_double}
    assert [t for _, t in py] == [cmap[t] for t, _ in c]


def test_status_strings_without_gpu():
    F, L = _lib()
    assert L.fde_strerror(0) == b"ok"
    assert b"invalid" in L.fde_strerror(-1)
    assert L.fde_size(None) == 0
