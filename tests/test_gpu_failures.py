"""Failure paths of the solve, caused from the host (no GPU fault is involved):
a non-finite desired state, an iteration cap, invalid options and bounds.
The status codes are those of include/fde.h."""
import math

import numpy as np
import pytest
import torch

import fde_inputs as fi
import oracle as O
from gpu_util import dev, host, lib, need_gpu, params, relerr

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec_name,inner_solver", [("FDE_FP64", 0), ("FDE_MIXED", 0), ("FDE_MIXED_DFV", 0),
                                                    ("FDE_FP64", 1)])
def test_nonfinite_desired_state_is_reported(prec_name, inner_solver):
    """A NaN (or an Inf) in ybar reaches the first reduction of the first
    sub-problem and the solve returns FDE_ENONFINITE; the problem stays usable."""
    need_gpu()
    F = lib()
    p = params(12, 10, 4)
    prob = F.Problem(p)
    fo = F.AdmmOptions(delta=1.0, rho=1.618, max_admm=3, fixed_iters=True, inner_tol_mode=1, inner_tol=1e-10,
                       precision=getattr(F, prec_name), inner_solver=inner_solver)
    for bad in (math.nan, math.inf):
        yb = fi.desired_state_sine(p, 2).ravel().copy()
        yb[37] = bad
        with pytest.raises(F.FdeError) as e:
            prob.admm_solve(fo, dev(yb), ua=-0.1, ub=0.1)
        assert e.value.status == F.FDE_ENONFINITE
    # the same handle then solves a finite problem correctly
    inst = fi.FdeInstance(p, fi.desired_state_sine(p, 2), None, None, None, -0.1, 0.1, 2)
    ref = O.admm_direct(inst, O.AdmmOptions(delta=1.0, rho=1.618), iters=3)
    fo.inner_tol = 1e-13 if prec_name == "FDE_FP64" else 1e-12
    r = prob.admm_solve(fo, dev(inst.ybar), ua=-0.1, ub=0.1)
    assert relerr(host(r["y"]), ref.y) < (1e-10 if prec_name == "FDE_FP64" else 1e-8)
    prob.close()


def test_iteration_cap_returns_enoconv_with_the_last_iterate():
    """max_admm reached before tol_admm: FDE_ENOCONV, and y, u, p, z_u and the
    stats hold the last iterate (equal to a fixed-iteration run of that length)."""
    need_gpu()
    F = lib()
    p = params(10, 8, 4)
    inst = fi.FdeInstance(p, fi.desired_state_sine(p, 6), None, None, 0.3, -0.05, 0.05, 6)
    prob = F.Problem(p)
    K = 5
    capped = F.AdmmOptions(delta=1.0, rho=1.618, tol_admm=1e-14, max_admm=K, inner_tol_mode=1, inner_tol=1e-13)
    with pytest.raises(F.FdeError) as e:
        prob.admm_solve(capped, dev(inst.ybar), yb=0.3, ua=-0.05, ub=0.05)
    assert e.value.status == F.FDE_ENOCONV
    r = prob.admm_solve(capped, dev(inst.ybar), yb=0.3, ua=-0.05, ub=0.05, allow_noconv=True)
    assert r["status"] == F.FDE_ENOCONV and r["stats"]["admm_iters"] == K
    fixed = F.AdmmOptions(**{**capped.__dict__, "fixed_iters": True})
    f = prob.admm_solve(fixed, dev(inst.ybar), yb=0.3, ua=-0.05, ub=0.05)
    assert f["status"] == F.FDE_OK
    for k in ("y", "u", "p", "zu"):
        assert torch.equal(r[k], f[k]), k
    ref = O.admm_direct(inst, O.AdmmOptions(delta=1.0, rho=1.618), iters=K)
    assert relerr(host(r["y"]), ref.y) < 1e-10
    # the last iterate is kept for a warm start
    assert prob.iterates(("y",))["y"].equal(r["y"])
    prob.close()


def test_invalid_options_and_bounds_are_rejected():
    """Options outside their domains (Section 3.1 and Algorithm 2: delta > 0,
    rho in (0, golden ratio), Algorithm 2 with rho <= 1, c_y >= 1, c_u >= gamma),
    unknown modes, caps below one and NaN bounds give FDE_EINVAL before any work."""
    need_gpu()
    F = lib()
    p = params(8, 8, 3, gamma=1e-3)
    prob = F.Problem(p)
    ybar = dev(fi.desired_state_sine(p, 1))
    good = dict(delta=1.0, rho=1.618, max_admm=2, fixed_iters=True)
    bad_opts = [dict(delta=0.0), dict(delta=-1.0), dict(delta=math.nan), dict(rho=0.0), dict(rho=1.62),
                dict(precision=7), dict(precision=F.FDE_FP32), dict(max_admm=0), dict(max_pcg=0),
                dict(algorithm=3), dict(inner_solver=2), dict(precond=2), dict(warm_start=2),
                dict(algorithm=2, rho=1.2, c_y=1.0, c_u=1e-3), dict(algorithm=2, rho=1.0, c_y=0.5, c_u=1e-3),
                dict(algorithm=2, rho=1.0, c_y=1.0, c_u=1e-4)]
    for kw in bad_opts:
        with pytest.raises(F.FdeError) as e:
            prob.admm_solve(F.AdmmOptions(**{**good, **kw}), ybar)
        assert e.value.status == F.FDE_EINVAL, kw
    for kw in (dict(ya=math.nan), dict(ub=math.nan)):
        with pytest.raises(F.FdeError) as e:
            prob.admm_solve(F.AdmmOptions(**good), ybar, **kw)
        assert e.value.status == F.FDE_EINVAL, kw
    # a warm start without a previous solve
    with pytest.raises(F.FdeError) as e:
        prob.admm_solve(F.AdmmOptions(**good, warm_start=True), ybar)
    assert e.value.status == F.FDE_EINVAL
    # the valid options still solve
    r = prob.admm_solve(F.AdmmOptions(**good), ybar)
    assert r["status"] == F.FDE_OK and np.isfinite(r["stats"]["objective"])
    prob.close()
