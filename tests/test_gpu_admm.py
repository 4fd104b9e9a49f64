"""GPU parity of the ADMM solve (Algorithm 1) and of the gradient against the
FP64 oracle, through the C ABI.

Tolerances (relative, infinity norm): FP64 1e-10 and MIXED 1e-8, the targets
of the workload specification. Fixed-iteration comparisons use exact oracle
sub-solves against GPU sub-solves converged to 1e-13 (FP64) or refined to
1e-12 (MIXED), so the only differences are rounding and the sub-solve
residual, amplified by at most the condition number of S (< 1e3 here)."""
import numpy as np
import pytest
import torch

import fde_inputs as fi
import oracle as O
from gpu_util import dev, host, lib, need_gpu, params, relerr

pytestmark = pytest.mark.gpu


def _instance(nx, ny, nt, seed=3, **boxes):
    p = params(nx, ny, nt, gamma=1e-3)
    ybar = fi.desired_state_sine(p, seed)
    g = 0.05 * fi.random_field(seed + 11, (nt, nx, ny))
    return fi.FdeInstance(p, ybar, g, boxes.get("ya"), boxes.get("yb"), boxes.get("ua"), boxes.get("ub"), seed)


def _run(F, inst, opts):
    prob = F.Problem(inst.params)
    r = prob.admm_solve(opts, dev(inst.ybar), g=None if inst.g is None else dev(inst.g), ya=inst.ya, yb=inst.yb,
                        ua=inst.ua, ub=inst.ub, allow_noconv=True)
    prob.close()
    return r


BOXES = [dict(ua=-0.05, ub=0.05), dict(yb=0.3), dict(ya=-0.1, yb=0.25, ua=-0.2, ub=0.1), dict()]


@pytest.mark.parametrize("boxes", BOXES)
@pytest.mark.parametrize("dims", [(5, 4, 3), (8, 6, 5), (16, 16, 8)])
def test_admm_fixed_iterations_fp64(dims, boxes):
    need_gpu()
    F = lib()
    inst = _instance(*dims, **boxes)
    K = 12
    o = O.AdmmOptions(delta=0.8, rho=1.618)
    ref = O.admm_direct(inst, o, iters=K)
    fo = F.AdmmOptions(delta=0.8, rho=1.618, max_admm=K, fixed_iters=True, inner_tol_mode=1, inner_tol=1e-13,
                       precision=F.FDE_FP64)
    r = _run(F, inst, fo)
    assert r["stats"]["admm_iters"] == K
    assert relerr(host(r["y"]), ref.y) < 1e-10
    assert relerr(host(r["u"]), ref.u) < 1e-10
    assert relerr(host(r["p"]), ref.p) < 1e-10
    assert relerr(host(r["zu"]), ref.zu) < 1e-10
    res = (r["stats"]["res_eq"], r["stats"]["res_y"], r["stats"]["res_u"])
    assert np.allclose(res, ref.residuals, rtol=1e-6, atol=1e-12)


@pytest.mark.parametrize("prec_name", ["FDE_FP64", "FDE_MIXED_DFV"])
def test_admm_with_split_double_tiles(prec_name):
    """The double (and double-float) split-halves tiles inside the solve: K ADMM
    iterations on lines that fill the transform (32 x 64) against the oracle."""
    need_gpu()
    F = lib()
    inst = _instance(32, 64, 4, ua=-0.05, ub=0.05, yb=0.3)
    K = 6
    ref = O.admm_direct(inst, O.AdmmOptions(delta=0.8, rho=1.618), iters=K)
    fo = F.AdmmOptions(delta=0.8, rho=1.618, max_admm=K, fixed_iters=True, inner_tol_mode=1,
                       inner_tol=1e-13 if prec_name == "FDE_FP64" else 1e-12, precision=getattr(F, prec_name),
                       inner_tol_mixed=1e-4)
    prob = F.Problem(inst.params)
    prob.set_tiles(-512, -512, fp64=True)
    prob.set_tiles(-512, -512, dfloat=True)
    r = prob.admm_solve(fo, dev(inst.ybar), g=dev(inst.g), ya=inst.ya, yb=inst.yb, ua=inst.ua, ub=inst.ub,
                        allow_noconv=True)
    prob.close()
    tol = 1e-10 if prec_name == "FDE_FP64" else 1e-8
    for k in ("y", "u", "p"):
        assert relerr(host(r[k]), getattr(ref, k)) < tol, k


@pytest.mark.parametrize("boxes", BOXES[:3])
def test_admm_fixed_iterations_mixed(boxes):
    need_gpu()
    F = lib()
    inst = _instance(16, 12, 6, **boxes)
    K = 12
    o = O.AdmmOptions(delta=0.8, rho=1.618)
    ref = O.admm_direct(inst, o, iters=K)
    fo = F.AdmmOptions(delta=0.8, rho=1.618, max_admm=K, fixed_iters=True, inner_tol_mode=1, inner_tol=1e-12,
                       precision=F.FDE_MIXED, inner_tol_mixed=1e-4)
    r = _run(F, inst, fo)
    assert r["stats"]["refine_steps"] > 0
    for k in ("y", "u", "p"):
        assert relerr(host(r[k]), getattr(ref, k)) < 1e-8, k


def test_admm_converged_matches_polished_kkt():
    need_gpu()
    F = lib()
    inst = _instance(8, 6, 5, ua=-0.05, ub=0.05, yb=0.3)
    o = O.AdmmOptions(delta=1.0, rho=1.618, tol=1e-11, max_iter=20000)
    st = O.admm_direct(inst, o)
    sol = O.polish(inst, st)
    fo = F.AdmmOptions(delta=1.0, rho=1.618, tol_admm=1e-11, max_admm=20000, inner_tol_mode=1, inner_tol=1e-13)
    r = _run(F, inst, fo)
    assert r["status"] == F.FDE_OK
    y, u = host(r["y"]), host(r["u"])
    assert relerr(y, sol.y) < 1e-8 and relerr(u, sol.u) < 1e-8
    # invariants: copies inside the box, residuals below tolerance
    zu = host(r["zu"])
    assert np.all(zu >= -0.05) and np.all(zu <= 0.05)
    s = r["stats"]
    assert max(s["res_eq"], s["res_y"], s["res_u"]) <= 1e-11
    assert abs(s["objective"] - sol.J) <= 1e-8 * abs(sol.J)


def test_admm_small_workload_fp64_and_mixed():
    """32x32 x 16 workload (control box [-0.5, 0.5], tol 1e-6): GPU FP64 and MIXED
    iterates after K iterations against the oracle's exact sub-solves."""
    need_gpu()
    F = lib()
    inst = fi.config_small()
    K = 6
    o = O.AdmmOptions(delta=1.0, rho=1.618)
    ref = O.admm_direct(inst, o, iters=K)
    for prec, tol, inner in ((F.FDE_FP64, 1e-10, 1e-13), (F.FDE_MIXED, 1e-8, 1e-12)):
        fo = F.AdmmOptions(delta=1.0, rho=1.618, max_admm=K, fixed_iters=True, inner_tol_mode=1, inner_tol=inner,
                           precision=prec)
        r = _run(F, inst, fo)
        for k in ("y", "u", "p"):
            assert relerr(host(r[k]), getattr(ref, k)) < tol, (prec, k, relerr(host(r[k]), getattr(ref, k)))


def test_admm_small_workload_converges():
    need_gpu()
    F = lib()
    inst = fi.config_small()
    # ADMM needs about 2e4 iterations here (delta = 1): the residuals of the
    # oracle's exact-sub-solve iteration fall by ~8% per 100 iterations
    fo = F.AdmmOptions(delta=1.0, rho=1.618, tol_admm=1e-6, max_admm=40000, inner_tol_mode=0, precision=F.FDE_MIXED)
    r = _run(F, inst, fo)
    s = r["stats"]
    assert r["status"] == F.FDE_OK, s
    assert max(s["res_eq"], s["res_y"], s["res_u"]) <= 1e-6
    zu = host(r["zu"])
    assert zu.min() >= -0.5 and zu.max() <= 0.5


def test_gradient_matches_oracle_and_closed_form():
    need_gpu()
    F = lib()
    inst = _instance(6, 5, 4, ua=-0.05, ub=0.05)
    inst.g = None
    p = inst.params
    o = O.AdmmOptions(delta=1.0, rho=1.618, tol=1e-11, max_iter=50000)
    st = O.admm_direct(inst, o)
    sol = O.polish(inst, st)
    ref = O.objective_gradient(inst, sol)
    prob = F.Problem(p)
    dJ, coef, pv = prob.admm_grad(dev(sol.y), dev(inst.ybar), tol=1e-14)
    assert relerr(host(dJ), ref["ybar"]) < 1e-12
    assert relerr(host(pv), sol.p) < 1e-9
    for i, k in enumerate(("dp", "dm", "ep", "em")):
        assert abs(float(coef[i]) - ref[k]) <= 1e-9 * max(1.0, abs(ref[k])), (k, float(coef[i]), ref[k])
    prob.close()


def test_autograd_function_gradients():
    need_gpu()
    F = lib()
    inst = _instance(6, 5, 4, ua=-0.05, ub=0.05)
    inst.g = None
    p = inst.params
    ybar = dev(inst.ybar).view(p.nt, p.nx, p.ny).requires_grad_(True)
    coef = torch.tensor([p.dp, p.dm, p.ep, p.em], dtype=torch.float64, requires_grad=True)
    fo = F.AdmmOptions(delta=1.0, rho=1.618, tol_admm=1e-11, max_admm=50000, inner_tol_mode=1, inner_tol=1e-13)
    J = F.solve_objective(ybar, coef, p, fo, dict(ua=-0.05, ub=0.05))
    J.backward()
    st = O.admm_direct(inst, O.AdmmOptions(delta=1.0, rho=1.618, tol=1e-11, max_iter=50000))
    sol = O.polish(inst, st)
    ref = O.objective_gradient(inst, sol)
    assert abs(float(J) - sol.J) <= 1e-8 * abs(sol.J)
    assert relerr(host(ybar.grad), ref["ybar"]) < 1e-7
    for i, k in enumerate(("dp", "dm", "ep", "em")):
        assert abs(float(coef.grad[i]) - ref[k]) <= 1e-6 * max(1.0, abs(ref[k]))


def test_gradient_differentiation_workload_32x32x16():
    """Differentiation workload's operator on 32x32x16 (control box [-1, 1]):
    converged GPU solve and fde_admm_grad against the oracle's exact optimum,
    adjoint and envelope gradient stored by tests/golden/make_grad_golden.py."""
    import json
    import os
    need_gpu()
    F = lib()
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "grad_32x32x16.json")))
    inst = fi.config_grad_small()
    prob = F.Problem(inst.params)
    # delta = 0.1 converges in a few hundred iterations here; the optimum does not depend on it
    fo = F.AdmmOptions(delta=0.1, rho=1.618, tol_admm=1e-11, max_admm=50000, inner_tol_mode=1, inner_tol=1e-13)
    ybar = dev(inst.ybar)
    r = prob.admm_solve(fo, ybar, ua=inst.ua, ub=inst.ub)
    assert r["status"] == F.FDE_OK
    assert abs(r["stats"]["objective"] - g["J"]) <= 1e-8 * abs(g["J"])
    idx = np.array(g["index"])
    y = host(r["y"])[idx]
    assert np.max(np.abs(y - np.array(g["y"]))) <= 1e-8 * g["y_maxabs"]
    dJ, coef, pv = prob.admm_grad(r["y"], ybar, tol=1e-14)
    assert np.max(np.abs(host(dJ)[idx] - np.array(g["dJ_dybar"]))) <= 1e-8 * g["y_maxabs"]
    assert np.max(np.abs(host(pv)[idx] - np.array(g["p"]))) <= 1e-6 * g["p_maxabs"]
    for a, b in zip(coef.tolist(), g["dcoef"]):
        assert abs(a - b) <= 1e-6 * max(1.0, abs(b)), (a, b)
    prob.close()


def test_gradient_differentiation_workload_full_size_properties():
    """256x256x64, beta = 1.5: after a fixed-iteration solve the adjoint solve
    returns p with B^T p = -J1 (y - ybar) (checked with the library's own B^T),
    and dJ/dybar equals -J1 (y - ybar) computed on the host."""
    need_gpu()
    F = lib()
    inst = fi.config_grad()
    p = inst.params
    prob = F.Problem(p)
    fo = F.AdmmOptions(delta=1.0, rho=1.618, max_admm=3, fixed_iters=True, inner_tol_mode=1, inner_tol=1e-10,
                       precision=F.FDE_MIXED)
    ybar = dev(inst.ybar)
    r = prob.admm_solve(fo, ybar, ua=inst.ua, ub=inst.ub)
    dJ, coef, pv = prob.admm_grad(r["y"], ybar, tol=1e-11)
    w = np.ones((p.nt, p.nx, p.ny))
    w[-1] = 0.5
    expect = -(w.ravel() * (host(r["y"]) - inst.ybar.ravel()))
    assert relerr(host(dJ), expect) < 1e-14
    btp = host(prob.matvec(pv, F.FDE_OP_BT))
    assert relerr(btp, expect) < 1e-8
    assert np.all(np.isfinite(coef.numpy()))
    prob.close()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec_name,inner_solver", [("FDE_FP64", 0), ("FDE_MIXED_DFV", 0), ("FDE_FP64", 1)])
def test_warm_start_continues_the_iteration(prec_name, inner_solver):
    """K1 iterations, then K2 more with warm_start, equal K1 + K2 iterations in one
    solve; without a previous solve a warm start is rejected."""
    need_gpu()
    F = lib()
    inst = _instance(16, 12, 6, ua=-0.05, ub=0.05, yb=0.3)
    prec = getattr(F, prec_name)
    base = dict(delta=0.8, rho=1.618, fixed_iters=True, inner_tol_mode=1, inner_tol=1e-12, precision=prec,
                inner_solver=inner_solver, max_pcg=3000)
    prob = F.Problem(inst.params)
    kw = dict(g=dev(inst.g), ya=inst.ya, yb=inst.yb, ua=inst.ua, ub=inst.ub, allow_noconv=True)
    with pytest.raises(F.FdeError) as e:
        prob.admm_solve(F.AdmmOptions(**base, max_admm=2, warm_start=True), dev(inst.ybar), **kw)
    assert e.value.status == F.FDE_EINVAL
    one = prob.admm_solve(F.AdmmOptions(**base, max_admm=7), dev(inst.ybar), **kw)
    y7 = host(one["y"])
    first = prob.admm_solve(F.AdmmOptions(**base, max_admm=3), dev(inst.ybar), **kw)
    # other calls on the problem in between leave the iterates alone
    prob.admm_grad(first["y"], dev(inst.ybar))
    prob.matvec(dev(inst.ybar), F.FDE_OP_S, F.AdmmOptions(**base))
    two = prob.admm_solve(F.AdmmOptions(**base, max_admm=4, warm_start=True), dev(inst.ybar), **kw)
    assert relerr(host(two["y"]), y7) < 1e-9
    ref = O.admm_direct(inst, O.AdmmOptions(delta=0.8, rho=1.618), iters=7)
    assert relerr(host(two["y"]), ref.y) < 1e-8
    prob.close()


@pytest.mark.parametrize("prec_name,inner_solver", [("FDE_FP64", 0), ("FDE_MIXED", 0), ("FDE_MIXED_DFV", 0),
                                                    ("FDE_FP64", 1), ("FDE_MIXED_DFV", 1)])
def test_zero_data_gives_zero_solution(prec_name, inner_solver):
    """ybar = 0, g = 0 and no bounds: every right-hand side vanishes and the iterates
    stay exactly zero (the zero-norm branches of the sub-solves)."""
    need_gpu()
    F = lib()
    p = params(12, 10, 4)
    prob = F.Problem(p)
    fo = F.AdmmOptions(delta=1.0, rho=1.618, max_admm=3, fixed_iters=True, inner_tol_mode=1, inner_tol=1e-10,
                       precision=getattr(F, prec_name), inner_solver=inner_solver, max_pcg=500)
    r = prob.admm_solve(fo, dev(np.zeros(prob.N)), allow_noconv=True)
    for k in ("y", "u", "p", "zu"):
        assert float(r[k].abs().max()) == 0.0, k
    assert r["stats"]["objective"] == 0.0
    prob.close()


def test_coincident_bounds_fix_the_control():
    """u_a = u_b: the projected copy z_u is that value everywhere and the iterates
    match the oracle's (FP64, fixed iterations)."""
    need_gpu()
    F = lib()
    inst = _instance(10, 8, 4, ua=0.01, ub=0.01)
    K = 8
    ref = O.admm_direct(inst, O.AdmmOptions(delta=0.8, rho=1.618), iters=K)
    fo = F.AdmmOptions(delta=0.8, rho=1.618, max_admm=K, fixed_iters=True, inner_tol_mode=1, inner_tol=1e-13,
                       precision=F.FDE_FP64)
    r = _run(F, inst, fo)
    assert float((r["zu"] - 0.01).abs().max()) == 0.0
    for k in ("y", "u", "p"):
        assert relerr(host(r[k]), getattr(ref, k)) < 1e-10, k


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("prec_name", ["FDE_FP64", "FDE_MIXED_DFV"])
def test_host_buffer_solve_matches_device_solve(prec_name, pinned):
    """fde_admm_solve_host (inputs and outputs in host memory; pinned buffers moved by
    the copy kernel, pageable ones by cudaMemcpyAsync) returns exactly what
    fde_admm_solve returns on device copies of the same arrays, with array and
    scalar bounds, and matches the oracle."""
    need_gpu()
    F = lib()
    inst = _instance(20, 36, 5, ua=-0.05, ub=0.05)
    yb = 0.3 + 0.05 * fi.random_field(71, (5, 20, 36))
    K = 5
    fo = F.AdmmOptions(delta=0.8, rho=1.618, max_admm=K, fixed_iters=True, inner_tol_mode=1, inner_tol=1e-12,
                       precision=getattr(F, prec_name), inner_tol_mixed=1e-4)

    def host(a):
        t = torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel())
        return t.pin_memory() if pinned else t.clone()

    prob = F.Problem(inst.params)
    d = prob.admm_solve(fo, dev(inst.ybar), g=dev(inst.g), yb=dev(yb), ua=inst.ua, ub=inst.ub, allow_noconv=True)
    d = {k: d[k].cpu() for k in ("y", "u", "p", "zu")}
    out = None if pinned else {k: torch.empty(inst.params.N, dtype=torch.float64) for k in ("y", "u", "p", "zu")}
    h = prob.admm_solve_host(fo, host(inst.ybar), g=host(inst.g), yb=host(yb), ua=inst.ua, ub=inst.ub,
                             allow_noconv=True, out=out, want_p=True, want_zu=True)
    prob.close()
    for k in ("y", "u", "p", "zu"):
        assert not h[k].is_cuda and torch.equal(h[k], d[k]), k
    assert h["stats"]["copy_in_ms"] > 0 and h["stats"]["copy_out_ms"] > 0
    ref = O.admm_direct(fi.FdeInstance(inst.params, inst.ybar, inst.g, None, yb, inst.ua, inst.ub, inst.seed),
                        O.AdmmOptions(delta=0.8, rho=1.618), iters=K)
    tol = 1e-10 if prec_name == "FDE_FP64" else 1e-8
    assert relerr(h["y"].numpy(), ref.y) < tol and relerr(h["u"].numpy(), ref.u) < tol


def test_host_buffer_solve_rejects_bad_buffers():
    need_gpu()
    F = lib()
    p = params(8, 8, 2)
    prob = F.Problem(p)
    fo = F.AdmmOptions(max_admm=2, precision=F.FDE_FP64)
    with pytest.raises(F.FdeError) as e:
        prob.admm_solve_host(fo, None)
    assert e.value.status == F.FDE_EINVAL
    with pytest.raises(ValueError):
        prob.admm_solve_host(fo, torch.zeros(prob.N, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        prob.admm_solve_host(fo, torch.zeros(prob.N + 1, dtype=torch.float64))
    r = prob.admm_solve_host(fo, torch.zeros(prob.N, dtype=torch.float64), allow_noconv=True)
    assert float(r["y"].abs().max()) == 0.0 and float(r["u"].abs().max()) == 0.0
    prob.close()
