"""The batch solve run by one persistent cooperative kernel
(fde_batch_admm_solve_persistent).

The executor replays the launches the batch solve records, so its reference is
the same launches issued one by one (replay=True): the results must agree bit
for bit, whatever the split of the CTAs into instance groups. The results are
also checked against the oracle's ADMM after K iterations (1e-8, every
sub-problem solved tightly on both sides), and the bounded waits are exercised
in both schedules (lockstep, instance groups): a CTA that never arrives at its
barrier ends the kernel with FDE_ETIMEOUT, and the context stays usable for the
next solve."""
import numpy as np
import pytest
import torch

import fde_inputs as fi
import oracle as O
from gpu_util import dev, host, lib, need_gpu, relerr

pytestmark = pytest.mark.gpu


def _pow2_batch():
    out = []
    shapes = [(16, 16, 4), (32, 16, 8), (8, 32, 16), (64, 32, 2), (32, 32, 16), (4, 8, 8)]
    rng = fi.uniform01(91, 4 * len(shapes))
    for k, (nx, ny, nt) in enumerate(shapes):
        p = fi.FdeParams(nx=nx, ny=ny, nt=nt, T=1.0, beta_x=1.1 + 0.8 * rng[4 * k], beta_y=1.1 + 0.8 * rng[4 * k + 1],
                         alpha_t=1.0, dp=1.0, dm=0.5, ep=0.8, em=0.3, gamma=10 ** (-4 + 2 * rng[4 * k + 2]))
        ub = 0.02 + 0.2 * rng[4 * k + 3]
        out.append(fi.FdeInstance(p, fi.desired_state_sine(p, 700 + k), None, None, None, -ub, ub, 700 + k))
    return out


def _solve(b, fo, insts, **kw):
    ys, us, stats, info, status = b.admm_solve_persistent(
        fo, [dev(i.ybar) for i in insts], ua=[i.ua for i in insts], ub=[i.ub for i in insts], **kw)
    return [host(y).copy() for y in ys], [host(u).copy() for u in us], stats, info, status


def test_persistent_equals_stream_replay_bitwise():
    need_gpu()
    F = lib()
    insts = _pow2_batch()
    b = F.Batch([i.params for i in insts])
    fo = F.AdmmOptions(delta=1.0, rho=1.618, max_admm=3, inner_tol=1e-10, precision=F.FDE_MIXED,
                       inner_tol_mixed=1e-5, max_refine=3, max_pcg=20)
    yr, ur, sr, _, _ = _solve(b, fo, insts, replay=True)
    # lockstep; instance groups: default split, one CTA per group, 7 CTAs, one group of all CTAs
    for sched, gc in ((0, 0), (1, 0), (1, 1), (1, 7), (1, 100000)):
        yp, up, sp, info, st = _solve(b, fo, insts, group_ctas=gc, schedule=sched)
        assert st == F.FDE_OK
        assert info["schedule"] == sched and info["groups"] >= 1 and info["commands"] > 0
        for a, c in zip(yr + ur, yp + up):
            assert np.array_equal(a, c), (sched, gc)
        for a, c in zip(sr, sp):
            assert a["pcg_iters"] == c["pcg_iters"] and a["max_sub_relres"] == c["max_sub_relres"]
    b.close()


def test_persistent_matches_oracle_after_fixed_iterations():
    need_gpu()
    F = lib()
    insts = _pow2_batch()
    K = 4
    b = F.Batch([i.params for i in insts])
    fo = F.AdmmOptions(delta=0.9, rho=1.618, max_admm=K, inner_tol=1e-12, precision=F.FDE_MIXED,
                       inner_tol_mixed=1e-5, max_refine=5, max_pcg=40)
    ys, us, stats, info, _ = _solve(b, fo, insts)
    for inst, y, u, s in zip(insts, ys, us, stats):
        ref = O.admm_direct(inst, O.AdmmOptions(delta=0.9, rho=1.618), iters=K)
        assert s["max_sub_relres"] <= 1e-12, s
        assert relerr(y, ref.y) < 1e-8, (inst.params.nx, relerr(y, ref.y))
        assert relerr(u, ref.u) < 1e-8
        assert np.allclose([s["res_eq"], s["res_y"], s["res_u"]], ref.residuals, rtol=1e-6, atol=1e-10)
    # the graph solve of the same batch (register-resident transforms) agrees
    yg, ug, _ = b.admm_solve(fo, [dev(i.ybar) for i in insts], ua=[i.ua for i in insts], ub=[i.ub for i in insts])
    for a, g in zip(ys, yg):
        assert relerr(a, host(g)) < 1e-9
    b.close()


def test_persistent_bounded_wait_returns_timeout():
    need_gpu()
    F = lib()
    insts = _pow2_batch()[:3]
    b = F.Batch([i.params for i in insts])
    fo = F.AdmmOptions(delta=1.0, rho=1.618, max_admm=2, inner_tol=1e-10, precision=F.FDE_MIXED,
                       inner_tol_mixed=1e-5, max_refine=2, max_pcg=10)
    yr, _, _, _, _ = _solve(b, fo, insts, replay=True)
    # instance groups: group 0's first CTA never arrives at the barrier after its
    # claim, so every wait of group 0 runs out after 50 ms
    _, _, _, info, st = _solve(b, fo, insts, group_ctas=4, schedule=1, timeout_s=0.05, stall_group=1, check=False)
    assert st == F.FDE_ETIMEOUT
    assert info["timeout_group"] == 0 and info["timeout_command"] == -1
    # lockstep: the first CTA runs step 0 and never arrives at its barrier
    _, _, _, info, st = _solve(b, fo, insts, timeout_s=0.05, stall_group=1, check=False)
    assert st == F.FDE_ETIMEOUT
    assert info["schedule"] == 0 and info["timeout_group"] == 0 and info["timeout_command"] == 0
    # the context is usable: the next solves run and equal the reference executor
    for sched in (0, 1):
        yp, _, _, _, st = _solve(b, fo, insts, group_ctas=4, schedule=sched)
        assert st == F.FDE_OK
        for a, c in zip(yp, yr):
            assert np.array_equal(a, c)
    torch.cuda.synchronize()
    b.close()


def test_persistent_rejects_what_it_cannot_run():
    need_gpu()
    F = lib()
    odd = _pow2_batch()[:1] + [fi.FdeInstance(fi.FdeParams(nx=12, ny=8, nt=4, T=1.0, beta_x=1.5, beta_y=1.5,
                                                         alpha_t=1.0, dp=1.0, dm=0.5, ep=0.8, em=0.3, gamma=1e-4),
                                              np.zeros(12 * 8 * 4), None, None, None, -0.1, 0.1, 0)]
    b = F.Batch([i.params for i in odd])
    fo = F.AdmmOptions(delta=1.0, rho=1.618, max_admm=1, inner_tol=1e-8, precision=F.FDE_MIXED, max_pcg=4)
    _, _, _, _, st = _solve(b, fo, odd, check=False)
    assert st == F.FDE_EUNSUPPORTED
    b.close()
    insts = _pow2_batch()[:2]
    b = F.Batch([i.params for i in insts])
    for prec in (F.FDE_MIXED_DF, F.FDE_MIXED_DFV, F.FDE_FP64):
        fo = F.AdmmOptions(delta=1.0, rho=1.618, max_admm=1, inner_tol=1e-8, precision=prec, max_pcg=4)
        _, _, _, _, st = _solve(b, fo, insts, check=False)
        assert st == F.FDE_EINVAL
    b.close()


def test_persistent_batch_workload_64_uneven_instances():
    """The 64-instance workload: bit-identical to the reference executor, every
    sub-problem at its target."""
    need_gpu()
    F = lib()
    insts = fi.config_batch()
    b = F.Batch([i.params for i in insts])
    fo = F.AdmmOptions(delta=1.0, rho=1.618, max_admm=2, inner_tol=1e-8, precision=F.FDE_MIXED,
                       inner_tol_mixed=1e-4, max_refine=2, max_pcg=12)
    ybars = [dev(i.ybar) for i in insts]
    kw = dict(ua=[i.ua for i in insts], ub=[i.ub for i in insts])
    ys, us, stats, info, st = b.admm_solve_persistent(fo, ybars, **kw)
    assert st == F.FDE_OK
    yp = [host(y).copy() for y in ys]
    for s, y, u in zip(stats, ys, us):
        assert s["max_sub_relres"] <= 1e-8, s
        assert torch.isfinite(y).all() and torch.isfinite(u).all()
    assert info["schedule"] == 0  # the fixed budgets make every instance's launch sequence alike
    ys, _, _, _, _ = b.admm_solve_persistent(fo, ybars, replay=True, **kw)
    for a, y in zip(yp, ys):
        assert np.array_equal(a, host(y))
    b.close()
    torch.cuda.empty_cache()
