"""GPU gradient of the optimal value J* with state bounds, the iterate
get/set entry points, and the differentiation workload's finite-difference
check at its own size, through the C ABI.

The adjoint equation of the envelope-theorem gradient (stationarity of the
Lagrangian of Section 3.1 in y) is B^T p = -J1 (y* - ybar) - w_y*, where w_y*
is the multiplier of y = z_y: with an active state bound it is non-zero, and
the gradient with respect to the diffusion coefficients depends on it."""
import numpy as np
import pytest
import torch

import fde_inputs as fi
import oracle as O
from gpu_util import dev, host, lib, need_gpu, params, relerr

pytestmark = pytest.mark.gpu


def _state_box_instance():
    """8x6x5 with the state bound y <= 0.3 and no control bound: the unconstrained
    state reaches 0.78, so the bound is active at 51 points (|w_y*| up to 0.64)."""
    p = params(8, 6, 5, gamma=1e-3)
    ybar = fi.desired_state_sine(p, 3)
    g = 0.05 * fi.random_field(14, (5, 8, 6))
    return fi.FdeInstance(p, ybar, g, None, 0.3, None, None, 3)


def _oracle_optimum(inst):
    st = O.admm_direct(inst, O.AdmmOptions(delta=1.0, rho=1.618, tol=1e-12, max_iter=40000))
    return O.polish(inst, st)


BOUNDS = dict(yb=0.3)
# ADMM penalty of the 256^2 x 64 differentiation solves (Section 6.1 picks delta from
# {0.1, 0.4, 2, 10, 100}); the optimum does not depend on it
DELTA_GRAD = 0.4


def test_gradient_with_active_state_bound():
    """8x6x5, y <= 0.3 active at the optimum: fde_admm_grad with the
    solve's w_y matches the oracle's KKT multiplier, adjoint p* and envelope
    gradient; without w_y the coefficient gradient is measurably wrong."""
    need_gpu()
    F = lib()
    inst = _state_box_instance()
    sol = _oracle_optimum(inst)
    assert np.count_nonzero(np.abs(sol.mu_y) > 1e-6) >= 10, "the state bound must be active for this test"
    ref = O.objective_gradient(inst, sol)
    p_dense = O.dense_adjoint(inst, sol)
    prob = F.Problem(inst.params)
    fo = F.AdmmOptions(delta=1.0, rho=1.618, tol_admm=1e-12, max_admm=40000, inner_tol_mode=1, inner_tol=1e-14)
    ybar = dev(inst.ybar)
    r = prob.admm_solve(fo, ybar, g=dev(inst.g), **BOUNDS)
    assert r["status"] == F.FDE_OK
    it = prob.iterates(("y", "wy", "p"))
    assert torch.equal(it["y"], r["y"]) and torch.equal(it["p"], r["p"])
    scale_mu = np.max(np.abs(sol.mu_y))
    assert np.max(np.abs(host(it["wy"]) - sol.mu_y.ravel())) <= 1e-8 * scale_mu
    dJ, coef, pv = prob.admm_grad(r["y"], ybar, wy=it["wy"], tol=1e-14)
    assert relerr(host(dJ), ref["ybar"]) < 1e-9
    assert relerr(host(pv), p_dense) < 1e-8
    assert relerr(host(pv), sol.p) < 1e-8
    for i, k in enumerate(("dp", "dm", "ep", "em")):
        assert abs(float(coef[i]) - ref[k]) <= 1e-7 * max(1.0, abs(ref[k])), (k, float(coef[i]), ref[k])
    # the multiplier matters: dropping it gives a different adjoint and gradient
    _, coef0, _ = prob.admm_grad(r["y"], ybar, wy=None, tol=1e-14)
    gap = max(abs(float(coef0[i]) - ref[k]) / max(1.0, abs(ref[k])) for i, k in enumerate(("dp", "dm", "ep", "em")))
    assert gap > 1e-4, gap
    prob.close()


def test_autograd_function_with_state_bound():
    """FdeAdmmFn with a state bound: J* and its gradients with respect to ybar and
    the four coefficients equal the oracle's; a second backward (retain_graph)
    gives the same gradients."""
    need_gpu()
    F = lib()
    inst = _state_box_instance()
    sol = _oracle_optimum(inst)
    ref = O.objective_gradient(inst, sol)
    p = inst.params
    ybar = dev(inst.ybar).view(p.nt, p.nx, p.ny).requires_grad_(True)
    coef = torch.tensor([p.dp, p.dm, p.ep, p.em], dtype=torch.float64, requires_grad=True)
    fo = F.AdmmOptions(delta=1.0, rho=1.618, tol_admm=1e-12, max_admm=40000, inner_tol_mode=1, inner_tol=1e-14)
    bounds = dict(g=dev(inst.g), **BOUNDS)
    J = F.solve_objective(ybar, coef, p, fo, bounds)
    assert abs(float(J.detach()) - sol.J) <= 1e-8 * abs(sol.J)
    J.backward(retain_graph=True)
    g1 = (ybar.grad.clone(), coef.grad.clone())
    assert relerr(host(ybar.grad), ref["ybar"]) < 1e-7
    for i, k in enumerate(("dp", "dm", "ep", "em")):
        assert abs(float(coef.grad[i]) - ref[k]) <= 1e-6 * max(1.0, abs(ref[k])), (k, float(coef.grad[i]), ref[k])
    ybar.grad = None
    coef.grad = None
    J.backward()
    assert torch.equal(ybar.grad, g1[0]) and torch.equal(coef.grad, g1[1])


@pytest.mark.parametrize("prec_name", ["FDE_FP64", "FDE_MIXED_DFV"])
def test_iterates_carry_a_warm_start_across_problems(prec_name):
    """K1 iterations on one problem, its iterates loaded into a second problem with
    the same parameters, K2 warm-started iterations there = K1 + K2 iterations on
    the first; get_iterates before any solve and on a failed state is rejected."""
    need_gpu()
    F = lib()
    p = params(16, 12, 6, gamma=1e-3)
    inst = fi.FdeInstance(p, fi.desired_state_sine(p, 5), None, None, 0.3, -0.05, 0.05, 5)
    prec = getattr(F, prec_name)
    base = dict(delta=0.8, rho=1.618, fixed_iters=True, inner_tol_mode=1, inner_tol=1e-12, precision=prec)
    kw = dict(yb=0.3, ua=-0.05, ub=0.05, allow_noconv=True)
    a = F.Problem(p)
    b = F.Problem(p)
    with pytest.raises(F.FdeError) as e:
        b.iterates(("y",))
    assert e.value.status == F.FDE_EINVAL
    ybar = dev(inst.ybar)
    whole = a.admm_solve(F.AdmmOptions(**base, max_admm=7), ybar, **kw)
    y7 = host(whole["y"])
    a.admm_solve(F.AdmmOptions(**base, max_admm=3), ybar, **kw)
    b.set_iterates(a.iterates())
    two = b.admm_solve(F.AdmmOptions(**base, max_admm=4, warm_start=True), ybar, **kw)
    assert relerr(host(two["y"]), y7) < 1e-11
    ref = O.admm_direct(inst, O.AdmmOptions(delta=0.8, rho=1.618), iters=7)
    tol = 1e-10 if prec_name == "FDE_FP64" else 1e-8
    assert relerr(host(two["y"]), ref.y) < tol
    # a partial set: missing iterates are zero, so loading only zeros equals a cold start
    b.set_iterates({})
    cold = b.admm_solve(F.AdmmOptions(**base, max_admm=3, warm_start=True), ybar, **kw)
    ref3 = O.admm_direct(inst, O.AdmmOptions(delta=0.8, rho=1.618), iters=3)
    assert relerr(host(cold["y"]), ref3.y) < tol
    with pytest.raises(ValueError):
        b.set_iterates({"q": ybar})
    a.close()
    b.close()


def _lagrangian_value(F, prob, st, r, psi):
    """J + p^T (B y + psi u) + w_y^T (y - z_y) + psi w_u^T (u - z_u) at the iterates
    of a solve with g = 0: the Lagrangian of Section 3.1 (psi-scaled as in Section
    6.1). Its gradient vanishes at the solution in every variable that can move
    (z sits exactly on its bound where w_u is non-zero), so at iterates within e of
    the solution it differs from J* by O(e^2), where J(y, u) alone differs by O(e)."""
    By = prob.matvec(st["y"], F.FDE_OP_B)
    extra = (torch.dot(st["p"], By + psi * st["u"]) + torch.dot(st["wy"], st["y"] - st["zy"])
             + psi * torch.dot(st["wu"], st["u"] - st["zu"]))
    return r["stats"]["objective"] + float(extra)


def test_gradient_differentiation_workload_finite_differences():
    """256x256 x 64, beta = 1.5, control box [-1, 1], FP64: the solve converged to
    1e-8 in the three residuals of Section 6.1, then dJ*/d(d+, d-, e+, e-) of
    fde_admm_grad against central differences of the GPU's own optimal value with
    h = 1e-6. The perturbed problems start from the base solution's iterates
    (fde_admm_set_iterates), so each needs only the iterations that close an
    O(h) gap. J* at each solve is the Lagrangian value at its iterates (second-order
    accurate in the iterate error); the O(h^2) truncation error is negligible, so
    the differences agree with the adjoint gradient to about 1e-6 of its size."""
    need_gpu()
    F = lib()
    inst = fi.config_grad()
    p = inst.params
    fo = F.AdmmOptions(delta=DELTA_GRAD, rho=1.618, tol_admm=1e-8, max_admm=8000, inner_tol_mode=0,
                       precision=F.FDE_FP64, max_pcg=2000)
    ybar = dev(inst.ybar)
    bounds = dict(ua=inst.ua, ub=inst.ub)
    prob = F.Problem(p)
    psi = prob.psi
    r = prob.admm_solve(fo, ybar, **bounds)
    assert r["status"] == F.FDE_OK, r["stats"]
    state = prob.iterates()
    J0 = _lagrangian_value(F, prob, state, r, psi)
    assert abs(J0 - r["stats"]["objective"]) <= 1e-6 * abs(J0)
    _, coef, _ = prob.admm_grad(r["y"], ybar, tol=1e-13)
    prob.close()
    h = 1e-6
    names = ("dp", "dm", "ep", "em")
    fd = []
    warm = F.AdmmOptions(**{**fo.__dict__, "warm_start": True})
    for i, k in enumerate(names):
        vals = []
        for sgn in (1.0, -1.0):
            q = fi.FdeParams(**{**p.__dict__, k: getattr(p, k) + sgn * h})
            pr = F.Problem(q)
            pr.set_iterates(state)
            rr = pr.admm_solve(warm, ybar, **bounds)
            assert rr["status"] == F.FDE_OK, (k, sgn, rr["stats"])
            vals.append(_lagrangian_value(F, pr, pr.iterates(), rr, psi))
            pr.close()
        fd.append((vals[0] - vals[1]) / (2 * h))
    torch.cuda.empty_cache()
    scale = max(abs(v) for v in fd)
    for i, k in enumerate(names):
        assert abs(float(coef[i]) - fd[i]) <= 1e-5 * scale, (k, float(coef[i]), fd[i], J0)
