"""Generalized ADMM (Section 3.3.2, Algorithm 2) on the GPU against the oracle.

R_y = c_y I - J1 and R_u = c_u I - J2 make M1, Q and M2 scalars; the right-hand
sides gain the proximal pulls rho R_y y^j and rho R_u u^j. Parity after K
iterations against the oracle's exact sub-solves: FP64 1e-10, MIXED and
MIXED_DF 1e-8 (the tolerances of Algorithm 1)."""
import numpy as np
import pytest

import fde_inputs as fi
import oracle as O
from gpu_util import dev, host, lib, need_gpu, params, relerr

pytestmark = pytest.mark.gpu


def _instance(nx, ny, nt, seed=3, weights=0, **boxes):
    p = params(nx, ny, nt, gamma=1e-3, weights=weights)
    ybar = fi.desired_state_sine(p, seed)
    g = 0.05 * fi.random_field(seed + 11, (nt, nx, ny))
    return fi.FdeInstance(p, ybar, g, boxes.get("ya"), boxes.get("yb"), boxes.get("ua"), boxes.get("ub"), seed)


def _solve(F, inst, fo):
    prob = F.Problem(inst.params)
    r = prob.admm_solve(fo, dev(inst.ybar), g=None if inst.g is None else dev(inst.g), ya=inst.ya, yb=inst.yb,
                        ua=inst.ua, ub=inst.ub, allow_noconv=True)
    prob.close()
    return r


BOXES = [dict(ua=-0.05, ub=0.05), dict(ya=-0.1, yb=0.25, ua=-0.2, ub=0.1), dict()]


@pytest.mark.parametrize("boxes", BOXES)
@pytest.mark.parametrize("dims", [(5, 4, 3), (16, 12, 8), (20, 30, 5)])
def test_generalized_fixed_iterations_fp64(dims, boxes):
    need_gpu()
    F = lib()
    inst = _instance(*dims, **boxes)
    K = 10
    c_y, c_u = 1.25, 2e-3
    ref = O.admm_direct(inst, O.AdmmOptions(delta=0.8, rho=0.95, algorithm=2, c_y=c_y, c_u=c_u), iters=K)
    fo = F.AdmmOptions(delta=0.8, rho=0.95, max_admm=K, fixed_iters=True, inner_tol_mode=1, inner_tol=1e-13,
                       precision=F.FDE_FP64, algorithm=2, c_y=c_y, c_u=c_u)
    r = _solve(F, inst, fo)
    for k in ("y", "u", "p", "zu"):
        assert relerr(host(r[k]), getattr(ref, k)) < 1e-10, (k, relerr(host(r[k]), getattr(ref, k)))
    res = (r["stats"]["res_eq"], r["stats"]["res_y"], r["stats"]["res_u"])
    assert np.allclose(res, ref.residuals, rtol=1e-6, atol=1e-12)


@pytest.mark.parametrize("prec_name", ["FDE_MIXED", "FDE_MIXED_DF"])
def test_generalized_fixed_iterations_mixed(prec_name):
    need_gpu()
    F = lib()
    inst = _instance(24, 20, 6, ua=-0.1, ub=0.1, yb=0.3)
    K = 8
    ref = O.admm_direct(inst, O.AdmmOptions(delta=1.0, rho=1.0, algorithm=2, c_y=1.5, c_u=5e-3), iters=K)
    fo = F.AdmmOptions(delta=1.0, rho=1.0, max_admm=K, fixed_iters=True, inner_tol_mode=1, inner_tol=1e-12,
                       precision=getattr(F, prec_name), algorithm=2, c_y=1.5, c_u=5e-3)
    r = _solve(F, inst, fo)
    assert r["stats"]["refine_steps"] > 0
    for k in ("y", "u", "p"):
        assert relerr(host(r[k]), getattr(ref, k)) < 1e-8, k


def test_generalized_with_zero_proximal_terms_is_algorithm_1():
    """Uniform weights, c_y = 1, c_u = gamma: R = 0 and the GPU's Algorithm 2
    reproduces its Algorithm 1 (rho = 1)."""
    need_gpu()
    F = lib()
    inst = _instance(12, 10, 4, weights=1, ua=-0.05, ub=0.05)
    K = 6
    base = dict(delta=0.9, rho=1.0, max_admm=K, fixed_iters=True, inner_tol_mode=1, inner_tol=1e-13,
                precision=F.FDE_FP64)
    r1 = _solve(F, inst, F.AdmmOptions(**base))
    r2 = _solve(F, inst, F.AdmmOptions(**base, algorithm=2, c_y=1.0, c_u=inst.params.gamma))
    for k in ("y", "u", "p"):
        assert relerr(host(r2[k]), host(r1[k])) < 1e-11, k


def test_generalized_converges_to_polished_kkt():
    need_gpu()
    F = lib()
    inst = _instance(8, 6, 5, ua=-0.05, ub=0.05, yb=0.3)
    p = inst.params
    o = O.AdmmOptions(delta=1.0, rho=1.0, tol=1e-11, max_iter=40000, algorithm=2, c_y=1.2, c_u=1.2 * p.gamma)
    sol = O.polish(inst, O.admm_direct(inst, o))
    fo = F.AdmmOptions(delta=1.0, rho=1.0, tol_admm=1e-11, max_admm=40000, inner_tol_mode=1, inner_tol=1e-13,
                       algorithm=2, c_y=1.2, c_u=1.2 * p.gamma)
    r = _solve(F, inst, fo)
    assert r["status"] == F.FDE_OK
    assert relerr(host(r["y"]), sol.y) < 1e-8 and relerr(host(r["u"]), sol.u) < 1e-8
    assert abs(r["stats"]["objective"] - sol.J) <= 1e-8 * abs(sol.J)


def test_generalized_options_rejected():
    need_gpu()
    F = lib()
    inst = _instance(8, 8, 4)
    prob = F.Problem(inst.params)
    for bad in (dict(rho=1.2, c_y=2.0, c_u=1.0), dict(rho=1.0, c_y=0.9, c_u=1.0),
                dict(rho=1.0, c_y=1.0, c_u=0.5 * inst.params.gamma), dict(rho=1.0, c_y=1.0, c_u=1.0, algorithm=3)):
        kw = {"algorithm": 2, **bad}
        with pytest.raises(F.FdeError) as e:
            prob.admm_solve(F.AdmmOptions(max_admm=2, **kw), dev(inst.ybar))
        assert e.value.status == F.FDE_EINVAL
    prob.close()


def test_generalized_batch_matches_oracle():
    need_gpu()
    F = lib()
    insts = []
    for k, (nx, ny, nt) in enumerate([(16, 16, 4), (24, 20, 3), (30, 18, 5)]):
        p = fi.FdeParams(nx=nx, ny=ny, nt=nt, T=1.0, beta_x=1.4, beta_y=1.7, alpha_t=1.0, dp=1.0, dm=0.5, ep=0.8,
                         em=0.3, gamma=1e-3)
        insts.append(fi.FdeInstance(p, fi.desired_state_sine(p, 900 + k), None, None, None, -0.05, 0.05, 900 + k))
    K = 4
    b = F.Batch([i.params for i in insts])
    fo = F.AdmmOptions(delta=0.9, rho=1.0, max_admm=K, inner_tol=1e-12, precision=F.FDE_MIXED,
                       inner_tol_mixed=1e-5, max_refine=5, max_pcg=40, algorithm=2, c_y=1.3, c_u=2e-3)
    ys, us, stats = b.admm_solve(fo, [dev(i.ybar) for i in insts], ua=[i.ua for i in insts],
                                 ub=[i.ub for i in insts])
    for inst, y, u, s in zip(insts, ys, us, stats):
        ref = O.admm_direct(inst, O.AdmmOptions(delta=0.9, rho=1.0, algorithm=2, c_y=1.3, c_u=2e-3), iters=K)
        assert s["max_sub_relres"] <= 1e-12, s
        assert relerr(host(y), ref.y) < 1e-8
        assert relerr(host(u), ref.u) < 1e-8
    b.close()


def test_generalized_medium_workload_properties():
    """256^2 x 64: a few Algorithm 2 iterations in MIXED precision; every sub-solve
    meets its target, iterates are finite and the copies stay in the box."""
    need_gpu()
    F = lib()
    inst = fi.config_medium()
    fo = F.AdmmOptions(delta=1.0, rho=1.0, max_admm=2, fixed_iters=True, inner_tol_mode=1, inner_tol=1e-8,
                       precision=F.FDE_MIXED, algorithm=2, c_y=1.1, c_u=1.1 * inst.params.gamma, max_pcg=500)
    prob = F.Problem(inst.params)
    r = prob.admm_solve(fo, dev(inst.ybar), ya=inst.ya, yb=inst.yb, ua=inst.ua, ub=inst.ub, allow_noconv=True)
    s = r["stats"]
    assert s["max_sub_relres"] <= 1e-8
    zu = host(r["zu"])
    assert np.all(np.isfinite(host(r["y"]))) and np.all(np.isfinite(zu))
    assert np.all(zu >= inst.ua) and np.all(zu <= inst.ub)
    prob.close()
