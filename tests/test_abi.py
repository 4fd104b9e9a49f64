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


def test_binding_tile_precision_and_host_buffer_checks():
    """Host-side argument checks of the binding: the tile precision selector and the
    host-buffer validation of admm_solve_host (no GPU call is made)."""
    import torch

    import paper_1907_13428_gb300 as F
    assert F._tile_prec(False, False) == F.FDE_FP32
    assert F._tile_prec(True, False) == F.FDE_MIXED_DF
    assert F._tile_prec(False, True) == F.FDE_FP64
    with pytest.raises(ValueError):
        F._tile_prec(True, True)
    t = torch.zeros(12, dtype=torch.float64)
    assert F._host_ptr(None, 12) is None
    assert F._host_ptr(t, 12).value == t.data_ptr()
    for bad in (torch.zeros(11, dtype=torch.float64), torch.zeros(12, dtype=torch.float32),
                torch.zeros(24, dtype=torch.float64)[::2]):
        with pytest.raises(ValueError):
            F._host_ptr(bad, 12)


def test_host_solve_rejects_null_arguments_without_gpu():
    """fde_admm_solve_host validates its arguments before any CUDA call."""
    F, L = _lib()
    st = F.fde_admm_stats()
    o = F.AdmmOptions().c()
    buf = (ctypes.c_double * 4)()
    args = [None, ctypes.byref(o), buf, None, None, None, None, None, 0.0, 0.0, 0.0, 0.0, buf, buf, None, None,
            ctypes.byref(st), None]
    assert L.fde_admm_solve_host(*args) == F.FDE_EINVAL


def test_setup_rejects_invalid_parameters_without_gpu():
    """fde_setup checks the problem description before any CUDA call: orders
    outside (1, 2) and (0, 1], empty or oversized axes, a non-positive gamma or
    final time, negative coefficients and unknown modes."""
    F, L = _lib()
    good = dict(nx=8, ny=8, nt=4, T=1.0, beta_x=1.5, beta_y=1.5, alpha_t=1.0, dp=1.0, dm=0.5, ep=0.8, em=0.3,
                gamma=1e-3, weights=0, time_step_mode=0)
    bad = [dict(beta_x=1.0), dict(beta_y=2.0), dict(alpha_t=0.0), dict(alpha_t=1.5), dict(nx=0), dict(nt=0),
           dict(gamma=0.0), dict(T=0.0), dict(dm=-1.0), dict(weights=2), dict(time_step_mode=3),
           dict(beta_x=float("nan"))]
    for kw in bad:
        ps = F.fde_params(**{**good, **kw})
        h = ctypes.c_void_p()
        assert L.fde_setup(ctypes.byref(ps), ctypes.byref(h), None) == F.FDE_EINVAL, kw
        assert not h.value
    ps = F.fde_params(**{**good, "nx": 4097})
    h = ctypes.c_void_p()
    assert L.fde_setup(ctypes.byref(ps), ctypes.byref(h), None) == F.FDE_EUNSUPPORTED
    assert L.fde_setup(None, ctypes.byref(h), None) == F.FDE_EINVAL


def test_iterate_calls_reject_null_problem_without_gpu():
    F, L = _lib()
    assert L.fde_admm_get_iterates(None, None, None, None, None, None, None, None, None) == F.FDE_EINVAL
    assert L.fde_admm_set_iterates(None, None, None, None, None, None, None, None, None) == F.FDE_EINVAL
