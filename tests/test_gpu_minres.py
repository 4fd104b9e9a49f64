"""Saddle-point sub-problems by MINRES with the block-diagonal preconditioner
K-tilde (Section 3.3.1) on the GPU, against the oracle.

Parity: after K ADMM iterations against the oracle's exact sub-solves (FP64
1e-10 with MINRES to 1e-13; MIXED / MIXED_DF 1e-8 with refinement to 1e-12);
MINRES counts against the oracle's MINRES on the same sub-problems; the
converged solve against the polished KKT point."""
import numpy as np
import pytest

import fde_inputs as fi
import oracle as O
from gpu_util import dev, host, lib, need_gpu, params, relerr

pytestmark = pytest.mark.gpu


def _instance(nx, ny, nt, seed=3, **boxes):
    p = params(nx, ny, nt, gamma=1e-3)
    ybar = fi.desired_state_sine(p, seed)
    g = 0.05 * fi.random_field(seed + 11, (nt, nx, ny))
    return fi.FdeInstance(p, ybar, g, boxes.get("ya"), boxes.get("yb"), boxes.get("ua"), boxes.get("ub"), seed)


def _solve(F, inst, fo):
    prob = F.Problem(inst.params)
    r = prob.admm_solve(fo, dev(inst.ybar), g=None if inst.g is None else dev(inst.g), ya=inst.ya, yb=inst.yb,
                        ua=inst.ua, ub=inst.ub, allow_noconv=True)
    prob.close()
    return r


ALGS = {1: dict(delta=0.8, rho=1.618), 2: dict(delta=0.8, rho=1.0, algorithm=2, c_y=1.25, c_u=2e-3)}


@pytest.mark.parametrize("alg", [1, 2])
@pytest.mark.parametrize("boxes", [dict(ua=-0.05, ub=0.05), dict(ya=-0.1, yb=0.25, ua=-0.2, ub=0.1)])
@pytest.mark.parametrize("dims", [(5, 4, 3), (16, 12, 8), (20, 30, 5)])
def test_minres_admm_fp64(dims, boxes, alg):
    need_gpu()
    F = lib()
    inst = _instance(*dims, **boxes)
    K = 8
    ref = O.admm_direct(inst, O.AdmmOptions(**ALGS[alg]), iters=K)
    fo = F.AdmmOptions(**ALGS[alg], max_admm=K, fixed_iters=True, inner_tol_mode=1, inner_tol=1e-13,
                       precision=F.FDE_FP64, inner_solver=1, max_pcg=3000)
    r = _solve(F, inst, fo)
    assert r["stats"]["max_sub_relres"] <= 1e-13
    for k in ("y", "u", "p", "zu"):
        assert relerr(host(r[k]), getattr(ref, k)) < 1e-10, (k, relerr(host(r[k]), getattr(ref, k)))
    res = (r["stats"]["res_eq"], r["stats"]["res_y"], r["stats"]["res_u"])
    assert np.allclose(res, ref.residuals, rtol=1e-6, atol=1e-12)


@pytest.mark.parametrize("prec_name", ["FDE_MIXED", "FDE_MIXED_DF"])
@pytest.mark.parametrize("alg", [1, 2])
def test_minres_admm_mixed(prec_name, alg):
    need_gpu()
    F = lib()
    inst = _instance(24, 20, 6, ua=-0.1, ub=0.1, yb=0.3)
    K = 6
    ref = O.admm_direct(inst, O.AdmmOptions(**ALGS[alg]), iters=K)
    fo = F.AdmmOptions(**ALGS[alg], max_admm=K, fixed_iters=True, inner_tol_mode=1, inner_tol=1e-12,
                       precision=getattr(F, prec_name), inner_solver=1, max_pcg=3000, inner_tol_mixed=1e-4)
    r = _solve(F, inst, fo)
    assert r["stats"]["refine_steps"] > 0
    assert r["stats"]["max_sub_relres"] <= 1e-12
    for k in ("y", "u", "p"):
        assert relerr(host(r[k]), getattr(ref, k)) < 1e-8, (k, relerr(host(r[k]), getattr(ref, k)))


def test_minres_counts_match_oracle():
    """Same algorithm, same sub-problems: the GPU's MINRES iteration counts over K
    ADMM iterations equal the oracle's within rounding (+-1 per solve)."""
    need_gpu()
    F = lib()
    inst = _instance(12, 10, 4, ua=-0.05, ub=0.05)
    K = 5
    o = O.AdmmOptions(delta=0.9, rho=1.618)
    st = O.admm_minres(inst, o, iters=K, inner_tol=1e-8)
    fo = F.AdmmOptions(delta=0.9, rho=1.618, max_admm=K, fixed_iters=True, inner_tol_mode=1, inner_tol=1e-8,
                       precision=F.FDE_FP64, inner_solver=1, max_pcg=3000)
    r = _solve(F, inst, fo)
    assert abs(r["stats"]["pcg_iters"] - sum(st.pcg_iters)) <= K, (r["stats"]["pcg_iters"], st.pcg_iters)
    assert relerr(host(r["y"]), st.y) < 1e-7


def test_minres_converges_to_polished_kkt():
    need_gpu()
    F = lib()
    inst = _instance(8, 6, 5, ua=-0.05, ub=0.05, yb=0.3)
    o = O.AdmmOptions(delta=1.0, rho=1.618, tol=1e-11, max_iter=20000)
    sol = O.polish(inst, O.admm_direct(inst, o))
    fo = F.AdmmOptions(delta=1.0, rho=1.618, tol_admm=1e-11, max_admm=20000, inner_tol_mode=1, inner_tol=1e-13,
                       inner_solver=1, max_pcg=3000)
    r = _solve(F, inst, fo)
    assert r["status"] == F.FDE_OK
    assert relerr(host(r["y"]), sol.y) < 1e-8 and relerr(host(r["u"]), sol.u) < 1e-8
    assert abs(r["stats"]["objective"] - sol.J) <= 1e-8 * abs(sol.J)


def test_minres_rejected_in_batch_and_invalid_solver():
    need_gpu()
    F = lib()
    p = params(16, 16, 4)
    b = F.Batch([p])
    fo = F.AdmmOptions(max_admm=2, precision=F.FDE_MIXED, inner_solver=1)
    with pytest.raises(F.FdeError) as e:
        b.admm_solve(fo, [dev(np.zeros(p.nt * p.nx * p.ny))])
    assert e.value.status == F.FDE_EUNSUPPORTED
    b.close()
    prob = F.Problem(p)
    with pytest.raises(F.FdeError) as e:
        prob.admm_solve(F.AdmmOptions(max_admm=2, inner_solver=2), dev(np.zeros(prob.N)))
    assert e.value.status == F.FDE_EINVAL
    prob.close()


def test_minres_medium_workload_properties():
    """256^2 x 64 in MIXED: every saddle-point solve meets its target, the iterates
    are finite and the MINRES count per solve stays in the range of the small
    grids (the preconditioned spectrum does not depend on n)."""
    need_gpu()
    F = lib()
    inst = fi.config_medium()
    fo = F.AdmmOptions(delta=1.0, rho=1.618, max_admm=2, fixed_iters=True, inner_tol_mode=1, inner_tol=1e-8,
                       precision=F.FDE_MIXED, inner_solver=1, max_pcg=2000)
    prob = F.Problem(inst.params)
    r = prob.admm_solve(fo, dev(inst.ybar), ya=inst.ya, yb=inst.yb, ua=inst.ua, ub=inst.ub, allow_noconv=True)
    s = r["stats"]
    assert s["max_sub_relres"] <= 1e-8
    assert np.all(np.isfinite(host(r["y"]))) and np.all(np.isfinite(host(r["u"])))
    assert s["pcg_iters"] / max(1, s["refine_steps"]) < 200
    prob.close()
