"""The matching Schur complement approximation S-hat (Section 3.2.2, Eq. second
schur complement preconditioner) with D-tilde = C_3(B) on the GPU: the
preconditioner element by element against the oracle (FP64 1e-12, FP32 2e-5),
and PCG-ADMM with it against the oracle's exact sub-solves (1e-10 / 1e-8) with
the oracle's own PCG counts."""
import numpy as np
import pytest
import torch

import fde_inputs as fi
import oracle as O
from gpu_util import dev, host, lib, need_gpu, params, relerr

pytestmark = pytest.mark.gpu

PSIZES = [(1, 1, 1), (3, 5, 2), (6, 10, 9), (8, 8, 8), (12, 15, 7), (20, 16, 5), (64, 32, 16), (50, 100, 4)]


@pytest.mark.parametrize("alg", [1, 2])
@pytest.mark.parametrize("dims", PSIZES)
def test_matching_preconditioner(dims, alg):
    need_gpu()
    F = lib()
    nx, ny, nt = dims
    p = params(nx, ny, nt, gamma=1e-3)
    kw = dict(delta=0.5, rho=1.4) if alg == 1 else dict(delta=0.5, rho=0.9, algorithm=2, c_y=1.2, c_u=2e-3)
    o = O.AdmmOptions(**kw, precond=1)
    fo = F.AdmmOptions(**kw, precond=1)
    prob = F.Problem(p)
    r = fi.random_field(19, (nt, nx, ny))
    ref = O.apply_preconditioner(p, o, r)
    assert relerr(host(prob.precond(dev(r), fo)), ref) < 1e-12
    assert relerr(host(prob.precond(dev(r, torch.float32), fo)), ref) < 2e-5
    # and it is not S-tilde
    ref0 = O.apply_preconditioner(p, O.AdmmOptions(**kw), r)
    if nx * ny * nt > 1:
        assert relerr(ref, ref0) > 1e-6
    prob.close()


def _instance(nx, ny, nt, seed=3, **boxes):
    p = params(nx, ny, nt, gamma=1e-3)
    ybar = fi.desired_state_sine(p, seed)
    g = 0.05 * fi.random_field(seed + 11, (nt, nx, ny))
    return fi.FdeInstance(p, ybar, g, boxes.get("ya"), boxes.get("yb"), boxes.get("ua"), boxes.get("ub"), seed)


@pytest.mark.parametrize("dims", [(8, 6, 5), (20, 16, 6)])
def test_admm_with_matching_preconditioner_fp64(dims):
    need_gpu()
    F = lib()
    inst = _instance(*dims, ua=-0.05, ub=0.05)
    K = 6
    o = O.AdmmOptions(delta=0.8, rho=1.618, precond=1)
    ref = O.admm_direct(inst, o, iters=K)
    st = O.admm_pcg(inst, o, iters=K, inner_tol=1e-8)
    prob = F.Problem(inst.params)
    fo = F.AdmmOptions(delta=0.8, rho=1.618, max_admm=K, fixed_iters=True, inner_tol_mode=1, inner_tol=1e-13,
                       precision=F.FDE_FP64, precond=1)
    r = prob.admm_solve(fo, dev(inst.ybar), g=dev(inst.g), ua=inst.ua, ub=inst.ub, allow_noconv=True)
    for k in ("y", "u", "p"):
        assert relerr(host(r[k]), getattr(ref, k)) < 1e-10, k
    # PCG counts with S-hat equal the oracle's PCG with S-hat (same recurrence), within one per solve
    fo8 = F.AdmmOptions(**{**fo.__dict__, "inner_tol": 1e-8})
    r8 = prob.admm_solve(fo8, dev(inst.ybar), g=dev(inst.g), ua=inst.ua, ub=inst.ub, allow_noconv=True)
    assert abs(r8["stats"]["pcg_iters"] - sum(st.pcg_iters)) <= K, (r8["stats"]["pcg_iters"], st.pcg_iters)
    prob.close()


def test_batch_with_matching_preconditioner():
    need_gpu()
    F = lib()
    insts = []
    for k, (nx, ny, nt) in enumerate([(16, 16, 4), (24, 20, 3)]):
        p = fi.FdeParams(nx=nx, ny=ny, nt=nt, T=1.0, beta_x=1.4, beta_y=1.7, alpha_t=1.0, dp=1.0, dm=0.5, ep=0.8,
                         em=0.3, gamma=1e-3)
        insts.append(fi.FdeInstance(p, fi.desired_state_sine(p, 950 + k), None, None, None, -0.05, 0.05, 950 + k))
    K = 4
    b = F.Batch([i.params for i in insts])
    fo = F.AdmmOptions(delta=0.9, rho=1.618, max_admm=K, inner_tol=1e-12, precision=F.FDE_MIXED,
                       inner_tol_mixed=1e-5, max_refine=5, max_pcg=40, precond=1)
    ys, us, stats = b.admm_solve(fo, [dev(i.ybar) for i in insts], ua=[i.ua for i in insts],
                                 ub=[i.ub for i in insts])
    for inst, y, u, s in zip(insts, ys, us, stats):
        ref = O.admm_direct(inst, O.AdmmOptions(delta=0.9, rho=1.618), iters=K)
        assert s["max_sub_relres"] <= 1e-12, s
        assert relerr(host(y), ref.y) < 1e-8
    b.close()
