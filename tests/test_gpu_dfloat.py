"""Double-float products (FDE_MIXED_DF): B and B^T on double vectors with the
FFTs in pairs of floats, and the mixed ADMM solve whose refinement residuals
use them.

Tolerance of a product: a double-float operation rounds to about 2^-46
relative (the sum is the fast "sloppy" variant), the tables carry 2^-48, and a
transform of length 2L <= 8192 takes 13 passes, so the norm-wise error is a
few 1e-13; 1e-11 relative (infinity norm) leaves a factor of 20 for the
operator's dynamic range. The solves keep the MIXED target of 1e-8."""
import numpy as np
import pytest
import torch

import fde_inputs as fi
import oracle as O
from gpu_util import dev, host, lib, need_gpu, params, relerr

pytestmark = pytest.mark.gpu

SIZES = [(1, 1, 1), (3, 5, 2), (7, 8, 3), (16, 12, 5), (17, 33, 6), (64, 64, 4), (100, 50, 3), (31, 200, 2),
         (1100, 20, 1)]


@pytest.mark.parametrize("alpha", [1.0, 0.6])
@pytest.mark.parametrize("dims", SIZES)
def test_matvec_dfloat_against_oracle(dims, alpha):
    need_gpu()
    F = lib()
    nx, ny, nt = dims
    p = params(nx, ny, nt, alpha_t=alpha)
    prob = F.Problem(p)
    x = fi.random_field(23, (nt, nx, ny))
    xd = dev(x)
    for op, tr in ((F.FDE_OP_B, False), (F.FDE_OP_BT, True)):
        ref = O.apply_B(p, x, transpose=tr)
        got = host(prob.matvec(xd, op, dfloat=True))
        assert relerr(got, ref) < 1e-11, (op, relerr(got, ref))
        # and it is not the float product: far closer than float rounding allows
        g32 = host(prob.matvec(xd.float(), op))
        if np.max(np.abs(ref)) > 0 and nx * ny * nt > 8:
            assert relerr(got, ref) < 1e-3 * max(relerr(g32, ref), 1e-9)
    prob.close()


@pytest.mark.parametrize("dims", [(7, 5, 3), (33, 17, 4), (64, 128, 2), (1024, 40, 2)])
def test_apply_factor_dfloat(dims):
    """One Kronecker factor in double-float arithmetic (one launch)."""
    need_gpu()
    F = lib()
    nx, ny, nt = dims
    p = params(nx, ny, nt)
    prob = F.Problem(p)
    x = fi.random_field(41, (nt, nx, ny))
    X, Y = O.space_matrices(p)
    psi = O.psi_scale(p)
    for axis, M, along in ((1, X, O.along_x1), (2, Y, O.along_x2)):
        for op, Mt in ((F.FDE_OP_B, M), (F.FDE_OP_BT, M.T)):
            ref = -psi * along(Mt, x)
            assert relerr(host(prob.apply_factor(dev(x), axis, op, dfloat=True)), ref) < 1e-11
    prob.close()


def test_matvec_dfloat_full_size_sampled():
    """1024^2 x 128: double-float B and B^T at sampled points against the
    oracle's one-by-one evaluation and against the double product."""
    need_gpu()
    F = lib()
    inst = fi.config_large()
    p = inst.params
    prob = F.Problem(p)
    x = inst.ybar
    xd = dev(x)
    rng = np.random.default_rng(8)
    pts = [(0, 0, 0), (p.nt - 1, p.nx - 1, p.ny - 1)]
    pts += [tuple(int(rng.integers(0, m)) for m in (p.nt, p.nx, p.ny)) for _ in range(20)]
    for op, tr in ((F.FDE_OP_B, False), (F.FDE_OP_BT, True)):
        full = prob.matvec(xd, op, dfloat=True)
        d64 = prob.matvec(xd, op)
        scale = float(torch.max(torch.abs(d64)))
        assert float(torch.max(torch.abs(full - d64))) / scale < 1e-11
        fh = host(full).reshape(p.nt, p.nx, p.ny)
        ref = O.apply_B_at(p, x, pts, transpose=tr)
        got = np.array([fh[q] for q in pts])
        assert np.max(np.abs(got - ref)) / scale < 1e-11
        del full, d64, fh
    prob.close()
    torch.cuda.empty_cache()


def test_dfloat_rejects_S_and_float_arrays():
    need_gpu()
    F = lib()
    prob = F.Problem(params(8, 8, 4))
    x = dev(np.ones(prob.N))
    with pytest.raises(F.FdeError) as e:
        prob.matvec(x, F.FDE_OP_S, F.AdmmOptions(), dfloat=True)
    assert e.value.status == F.FDE_EINVAL
    with pytest.raises(ValueError):
        prob.matvec(x.float(), dfloat=True)
    prob.close()


def _instance(nx, ny, nt, seed=3, **boxes):
    p = params(nx, ny, nt, gamma=1e-3)
    ybar = fi.desired_state_sine(p, seed)
    g = 0.05 * fi.random_field(seed + 11, (nt, nx, ny))
    return fi.FdeInstance(p, ybar, g, boxes.get("ya"), boxes.get("yb"), boxes.get("ua"), boxes.get("ub"), seed)


@pytest.mark.parametrize("boxes", [dict(ua=-0.05, ub=0.05), dict(ya=-0.1, yb=0.25, ua=-0.2, ub=0.1)])
@pytest.mark.parametrize("dims", [(16, 12, 6), (40, 24, 5)])
def test_admm_mixed_df_fixed_iterations(dims, boxes):
    need_gpu()
    F = lib()
    inst = _instance(*dims, **boxes)
    K = 10
    ref = O.admm_direct(inst, O.AdmmOptions(delta=0.8, rho=1.618), iters=K)
    fo = F.AdmmOptions(delta=0.8, rho=1.618, max_admm=K, fixed_iters=True, inner_tol_mode=1, inner_tol=1e-12,
                       precision=F.FDE_MIXED_DF, inner_tol_mixed=1e-4)
    prob = F.Problem(inst.params)
    r = prob.admm_solve(fo, dev(inst.ybar), g=dev(inst.g), ya=inst.ya, yb=inst.yb, ua=inst.ua, ub=inst.ub,
                        allow_noconv=True)
    prob.close()
    assert r["stats"]["refine_steps"] > 0
    assert r["stats"]["max_sub_relres"] <= 1e-12
    for k in ("y", "u", "p"):
        assert relerr(host(r[k]), getattr(ref, k)) < 1e-8, (k, relerr(host(r[k]), getattr(ref, k)))


def test_admm_mixed_df_small_workload():
    """32x32 x 16 workload: MIXED_DF iterates after K iterations against the
    oracle's exact sub-solves, and against the MIXED (double residual) solve."""
    need_gpu()
    F = lib()
    inst = fi.config_small()
    K = 6
    ref = O.admm_direct(inst, O.AdmmOptions(delta=1.0, rho=1.618), iters=K)
    out = {}
    for prec in (F.FDE_MIXED, F.FDE_MIXED_DF):
        fo = F.AdmmOptions(delta=1.0, rho=1.618, max_admm=K, fixed_iters=True, inner_tol_mode=1, inner_tol=1e-12,
                           precision=prec)
        prob = F.Problem(inst.params)
        r = prob.admm_solve(fo, dev(inst.ybar), ya=inst.ya, yb=inst.yb, ua=inst.ua, ub=inst.ub, allow_noconv=True)
        prob.close()
        for k in ("y", "u", "p"):
            assert relerr(host(r[k]), getattr(ref, k)) < 1e-8, (prec, k)
        out[prec] = host(r["y"])
    assert relerr(out[F.FDE_MIXED_DF], out[F.FDE_MIXED]) < 1e-9


def test_batch_mixed_df_matches_oracle():
    need_gpu()
    F = lib()
    insts = []
    for k, (nx, ny, nt) in enumerate([(16, 16, 4), (24, 20, 3), (30, 18, 5)]):
        p = fi.FdeParams(nx=nx, ny=ny, nt=nt, T=1.0, beta_x=1.4, beta_y=1.7, alpha_t=1.0, dp=1.0, dm=0.5, ep=0.8,
                         em=0.3, gamma=1e-3)
        insts.append(fi.FdeInstance(p, fi.desired_state_sine(p, 700 + k), None, None, None, -0.05, 0.05, 700 + k))
    K = 4
    b = F.Batch([i.params for i in insts])
    fo = F.AdmmOptions(delta=0.9, rho=1.618, max_admm=K, inner_tol=1e-12, precision=F.FDE_MIXED_DF,
                       inner_tol_mixed=1e-5, max_refine=5, max_pcg=40)
    ys, us, stats = b.admm_solve(fo, [dev(i.ybar) for i in insts], ua=[i.ua for i in insts],
                                 ub=[i.ub for i in insts])
    for inst, y, u, s in zip(insts, ys, us, stats):
        ref = O.admm_direct(inst, O.AdmmOptions(delta=0.9, rho=1.618), iters=K)
        assert s["max_sub_relres"] <= 1e-12, s
        assert relerr(host(y), ref.y) < 1e-8
        assert relerr(host(u), ref.u) < 1e-8
    b.close()


@pytest.mark.parametrize("inner_solver", [0, 1])
def test_admm_mixed_dfv_fixed_iterations(inner_solver):
    """FDE_MIXED_DFV: double-float products for the evaluations that cannot be the
    last one, double for the accepted ones; parity with the oracle at 1e-8 and
    every sub-problem's accepted residual below its target."""
    need_gpu()
    F = lib()
    inst = _instance(40, 24, 5, ua=-0.05, ub=0.05)
    K = 8
    ref = O.admm_direct(inst, O.AdmmOptions(delta=0.8, rho=1.618), iters=K)
    fo = F.AdmmOptions(delta=0.8, rho=1.618, max_admm=K, fixed_iters=True, inner_tol_mode=1, inner_tol=1e-10,
                       precision=F.FDE_MIXED_DFV, inner_tol_mixed=1e-4, inner_solver=inner_solver, max_pcg=3000)
    prob = F.Problem(inst.params)
    r = prob.admm_solve(fo, dev(inst.ybar), g=dev(inst.g), ua=inst.ua, ub=inst.ub, allow_noconv=True)
    prob.close()
    assert r["stats"]["refine_steps"] > 0
    assert r["stats"]["max_sub_relres"] <= 1e-10
    for k in ("y", "u", "p"):
        assert relerr(host(r[k]), getattr(ref, k)) < 1e-8, (k, relerr(host(r[k]), getattr(ref, k)))


def test_admm_mixed_dfv_equals_mixed_small_workload():
    need_gpu()
    F = lib()
    inst = fi.config_small()
    K = 6
    out = {}
    for prec in (F.FDE_MIXED, F.FDE_MIXED_DFV):
        fo = F.AdmmOptions(delta=1.0, rho=1.618, max_admm=K, fixed_iters=True, inner_tol_mode=1, inner_tol=1e-12,
                           precision=prec)
        prob = F.Problem(inst.params)
        r = prob.admm_solve(fo, dev(inst.ybar), ya=inst.ya, yb=inst.yb, ua=inst.ua, ub=inst.ub, allow_noconv=True)
        prob.close()
        assert r["stats"]["max_sub_relres"] <= 1e-12
        out[prec] = host(r["y"])
    assert relerr(out[F.FDE_MIXED_DFV], out[F.FDE_MIXED]) < 1e-9


def test_batch_mixed_dfv_matches_oracle():
    need_gpu()
    F = lib()
    insts = []
    for k, (nx, ny, nt) in enumerate([(16, 16, 4), (24, 20, 3), (30, 18, 5)]):
        p = fi.FdeParams(nx=nx, ny=ny, nt=nt, T=1.0, beta_x=1.4, beta_y=1.7, alpha_t=1.0, dp=1.0, dm=0.5, ep=0.8,
                         em=0.3, gamma=1e-3)
        insts.append(fi.FdeInstance(p, fi.desired_state_sine(p, 800 + k), None, None, None, -0.05, 0.05, 800 + k))
    K = 4
    b = F.Batch([i.params for i in insts])
    fo = F.AdmmOptions(delta=0.9, rho=1.618, max_admm=K, inner_tol=1e-12, precision=F.FDE_MIXED_DFV,
                       inner_tol_mixed=1e-5, max_refine=5, max_pcg=40)
    ys, us, stats = b.admm_solve(fo, [dev(i.ybar) for i in insts], ua=[i.ua for i in insts],
                                 ub=[i.ub for i in insts])
    for inst, y, u, s in zip(insts, ys, us, stats):
        ref = O.admm_direct(inst, O.AdmmOptions(delta=0.9, rho=1.618), iters=K)
        assert s["max_sub_relres"] <= 1e-12, s
        assert relerr(host(y), ref.y) < 1e-8
        assert relerr(host(u), ref.u) < 1e-8
    b.close()


@pytest.mark.parametrize("tiles", [(256, 256), (-512, -512), (-256, -512), (128, 128)])
@pytest.mark.parametrize("dims", [(17, 33, 6), (64, 64, 4), (100, 50, 3), (31, 200, 2), (2, 1100, 2)])
def test_every_dfloat_tile_matches_oracle(dims, tiles):
    """Both double-float tile variants (both halves per thread, split halves) of
    the x2 and x1 passes, with the epilogue, against the oracle."""
    need_gpu()
    F = lib()
    nx, ny, nt = dims
    p = params(nx, ny, nt)
    prob = F.Problem(p)
    rows, axis = tiles
    if ny > 2048 and rows in (-256, 128):
        rows = 0
    prob.set_tiles(rows, axis, dfloat=True)
    assert prob.tiles(dfloat=True)[1] == axis
    x = fi.random_field(47, (nt, nx, ny))
    for op, tr in ((F.FDE_OP_B, False), (F.FDE_OP_BT, True)):
        got = host(prob.matvec(dev(x), op, dfloat=True))
        assert relerr(got, O.apply_B(p, x, transpose=tr)) < 1e-11
    prob.close()


def test_dfv_full_size_against_mixed_and_fp64():
    """1024^2 x 128, the benchmark's configuration (one ADMM iteration, sub-solves
    to 1e-8): the FDE_MIXED_DFV solve meets every sub-problem target with a double
    residual, keeps the box, and agrees with the all-double refinement and with the
    all-FP64 solve to the accuracy the 1e-8 sub-solve tolerance allows."""
    need_gpu()
    F = lib()
    inst = fi.config_large()
    prob = F.Problem(inst.params)
    ybar = dev(inst.ybar)
    base = dict(delta=1.0, rho=1.618, max_admm=1, fixed_iters=True, inner_tol_mode=1, inner_tol=1e-8,
                inner_tol_mixed=1e-4, max_pcg=500, max_refine=30)
    ys = {}
    for prec in (F.FDE_MIXED_DFV, F.FDE_MIXED, F.FDE_FP64):
        r = prob.admm_solve(F.AdmmOptions(**base, precision=prec), ybar, ua=inst.ua, ub=inst.ub, allow_noconv=True)
        assert r["stats"]["max_sub_relres"] <= 1e-8, (prec, r["stats"])
        ys[prec] = r["y"].clone()
        if prec == F.FDE_MIXED_DFV:
            zu = r["zu"]
            assert bool(torch.all(zu >= inst.ua)) and bool(torch.all(zu <= inst.ub))
            assert bool(torch.all(torch.isfinite(r["y"])))
        del r
    scale = float(ys[F.FDE_FP64].abs().max())
    assert float((ys[F.FDE_MIXED_DFV] - ys[F.FDE_MIXED]).abs().max()) / scale < 1e-6
    assert float((ys[F.FDE_MIXED_DFV] - ys[F.FDE_FP64]).abs().max()) / scale < 1e-6
    del ys
    prob.close()
    torch.cuda.empty_cache()


def test_dfv_recursive_steering_in_a_converged_run():
    """A long FDE_MIXED_DFV run: once the warm starts are good, corrections are
    steered by the float PCG's recursive residual (counted in the stats); every
    accepted sub-problem residual is still a double evaluation below its target,
    and the run reaches the polished KKT point."""
    need_gpu()
    F = lib()
    inst = _instance(8, 6, 5, ua=-0.05, ub=0.05)
    sol = O.polish(inst, O.admm_direct(inst, O.AdmmOptions(delta=1.0, rho=1.618, tol=1e-11, max_iter=20000)))
    prob = F.Problem(inst.params)
    fo = F.AdmmOptions(delta=1.0, rho=1.618, tol_admm=1e-8, max_admm=20000, inner_tol_mode=1, inner_tol=1e-8,
                       precision=F.FDE_MIXED_DFV, inner_tol_mixed=1e-4)
    r = prob.admm_solve(fo, dev(inst.ybar), g=dev(inst.g), ua=inst.ua, ub=inst.ub)
    prob.close()
    s = r["stats"]
    assert s["recursive_steers"] > 0, s
    assert s["max_sub_relres"] <= 1e-8
    assert relerr(host(r["y"]), sol.y) < 1e-6 and relerr(host(r["u"]), sol.u) < 1e-6
