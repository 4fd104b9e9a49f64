"""GPU parity of the operator and preconditioner kernels against the FP64 oracle,
through the C ABI. FP64 tolerance: 1e-12 relative (infinity norm) for products
whose rounding error is a few hundred ulps; FP32: 2e-5 (float eps 6e-8 times
the log-depth of the transforms and the operator's dynamic range)."""
import numpy as np
import pytest
import torch

import fde_inputs as fi
import oracle as O
from gpu_util import dev, host, lib, need_gpu, params, relerr

pytestmark = pytest.mark.gpu

SIZES = [(1, 1, 1), (2, 3, 1), (3, 5, 2), (5, 7, 4), (7, 8, 3), (8, 8, 8), (16, 12, 5), (33, 17, 6), (64, 64, 4),
         (100, 50, 3)]


@pytest.mark.parametrize("alpha", [1.0, 0.6])
@pytest.mark.parametrize("dims", SIZES)
def test_matvec_B_BT_fp64(dims, alpha):
    need_gpu()
    F = lib()
    nx, ny, nt = dims
    p = params(nx, ny, nt, alpha_t=alpha)
    prob = F.Problem(p)
    x = fi.random_field(17, (nt, nx, ny))
    xd = dev(x)
    for op, tr in ((F.FDE_OP_B, False), (F.FDE_OP_BT, True)):
        got = host(prob.matvec(xd, op))
        ref = O.apply_B(p, x, transpose=tr)
        assert relerr(got, ref) < 1e-12, (op, relerr(got, ref))
    prob.close()


@pytest.mark.parametrize("dims", SIZES[:8])
def test_matvec_S_fp64_and_fp32(dims):
    need_gpu()
    F = lib()
    nx, ny, nt = dims
    p = params(nx, ny, nt)
    o = O.AdmmOptions(delta=0.7, rho=1.4)
    prob = F.Problem(p)
    x = fi.random_field(5, (nt, nx, ny))
    fo = F.AdmmOptions(delta=0.7, rho=1.4)
    got = host(prob.matvec(dev(x), F.FDE_OP_S, fo))
    ref = O.apply_S(p, o, x)
    assert relerr(got, ref) < 1e-12
    got32 = host(prob.matvec(dev(x, torch.float32), F.FDE_OP_S, fo))
    assert relerr(got32, ref) < 2e-5
    for op, tr in ((F.FDE_OP_B, False), (F.FDE_OP_BT, True)):
        g32 = host(prob.matvec(dev(x, torch.float32), op))
        assert relerr(g32, O.apply_B(p, x, transpose=tr)) < 2e-5
    prob.close()


PSIZES = [(1, 1, 1), (2, 3, 1), (3, 5, 2), (5, 7, 4), (6, 10, 9), (8, 8, 8), (12, 15, 7), (20, 16, 5),
          (64, 32, 16), (50, 100, 4)]


@pytest.mark.parametrize("dims", PSIZES)
def test_preconditioner_fp64_fp32(dims):
    need_gpu()
    F = lib()
    nx, ny, nt = dims
    p = params(nx, ny, nt, gamma=1e-4)
    o = O.AdmmOptions(delta=0.4, rho=1.618)
    fo = F.AdmmOptions(delta=0.4, rho=1.618)
    prob = F.Problem(p)
    r = fi.random_field(9, (nt, nx, ny))
    ref = O.apply_preconditioner(p, o, r)
    got = host(prob.precond(dev(r), fo))
    assert relerr(got, ref) < 1e-12
    got32 = host(prob.precond(dev(r, torch.float32), fo))
    assert relerr(got32, ref) < 2e-5
    # in place
    rd = dev(r)
    prob.precond(rd, fo, out=rd)
    assert relerr(host(rd), ref) < 1e-12
    prob.close()


def test_unsupported_preconditioner_length_is_reported():
    need_gpu()
    F = lib()
    prob = F.Problem(params(11, 4, 2))
    r = dev(np.ones(prob.N))
    with pytest.raises(F.FdeError) as e:
        prob.precond(r, F.AdmmOptions())
    assert e.value.status == F.FDE_EUNSUPPORTED
    # the matvec supports every length
    x = fi.random_field(1, prob.shape)
    assert relerr(host(prob.matvec(dev(x))), O.apply_B(prob.params, x)) < 1e-12


def test_invalid_parameters_rejected():
    need_gpu()
    F = lib()
    for bad in (dict(beta_x=2.0), dict(beta_y=1.0), dict(alpha_t=0.0), dict(alpha_t=1.2), dict(gamma=0.0),
                dict(dp=-1.0)):
        with pytest.raises(F.FdeError) as e:
            F.Problem(params(4, 4, 4, **bad))
        assert e.value.status == F.FDE_EINVAL
    with pytest.raises(F.FdeError) as e:
        F.Problem(params(4097, 4, 4))
    assert e.value.status == F.FDE_EUNSUPPORTED
    prob = F.Problem(params(4, 4, 4))
    x = dev(np.zeros(prob.N))
    with pytest.raises(F.FdeError):
        prob.matvec(x, op=7)
    with pytest.raises(F.FdeError):
        prob.matvec(x, op=F.FDE_OP_S, opts=F.AdmmOptions(rho=1.7))
    prob.close()


@pytest.mark.parametrize("cfg", ["medium", "large"])
def test_matvec_full_size_sampled(cfg):
    """B x and B^T x at the 256^2 x 64 and 1024^2 x 128 workloads, FP64 and FP32,
    checked at sampled points that the oracle evaluates one by one."""
    need_gpu()
    F = lib()
    inst = fi.config_medium() if cfg == "medium" else fi.config_large()
    p = inst.params
    prob = F.Problem(p)
    x = inst.ybar
    rng = np.random.default_rng(4)
    pts = [(0, 0, 0), (p.nt - 1, p.nx - 1, p.ny - 1), (p.nt - 1, 0, p.ny - 1)]
    pts += [tuple(int(rng.integers(0, m)) for m in (p.nt, p.nx, p.ny)) for _ in range(24)]
    xd = dev(x)
    for op, tr in ((F.FDE_OP_B, False), (F.FDE_OP_BT, True)):
        full = host(prob.matvec(xd, op)).reshape(p.nt, p.nx, p.ny)
        ref = O.apply_B_at(p, x, pts, transpose=tr)
        got = np.array([full[q] for q in pts])
        scale = np.max(np.abs(full))
        assert np.max(np.abs(got - ref)) / scale < 1e-12
        full32 = host(prob.matvec(xd.float(), op)).reshape(p.nt, p.nx, p.ny)
        got32 = np.array([full32[q] for q in pts])
        assert np.max(np.abs(got32 - ref)) / scale < 2e-5
        del full, full32
    prob.close()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dims", [(7, 5, 3), (33, 17, 4), (64, 128, 2)])
def test_apply_factor_single_axis(dims):
    """fde_apply_factor: one Kronecker factor, -psi X along x1 or -psi Y along x2."""
    need_gpu()
    F = lib()
    nx, ny, nt = dims
    p = params(nx, ny, nt)
    prob = F.Problem(p)
    x = fi.random_field(21, (nt, nx, ny))
    X, Y = O.space_matrices(p)
    psi = O.psi_scale(p)
    for axis, M, along in ((1, X, O.along_x1), (2, Y, O.along_x2)):
        for op, Mt in ((F.FDE_OP_B, M), (F.FDE_OP_BT, M.T)):
            ref = -psi * along(Mt, x)
            assert relerr(host(prob.apply_factor(dev(x), axis, op)), ref) < 1e-12
            assert relerr(host(prob.apply_factor(dev(x, torch.float32), axis, op)), ref) < 2e-5
    prob.close()


def test_alu_peak_probe_is_plausible():
    need_gpu()
    F = lib()
    f64 = F.alu_peak(F.FDE_FP64)
    f32 = F.alu_peak(F.FDE_FP32)
    assert 0.1 < f64 < 200 and 1 < f32 < 500 and f32 > f64


@pytest.mark.parametrize("dims", [(64, 64, 8), (128, 256, 4), (33, 1024, 2)])
def test_autotuned_tiles_keep_parity(dims):
    """fde_autotune picks valid tiles; products with every tile choice match the oracle."""
    need_gpu()
    F = lib()
    nx, ny, nt = dims
    p = params(nx, ny, nt)
    prob = F.Problem(p)
    rows, axis = prob.autotune()
    assert rows in (128, 256, 512) and axis in (256, 512)
    rd, ad = prob.tiles(dfloat=True)
    assert rd in (128, 256, -256, -512) and ad in (128, 256, -512)
    r64, a64 = prob.tiles(fp64=True)
    assert r64 in (128, 256, -256, -512) and a64 in (128, 256, -512)
    assert relerr(host(prob.matvec(dev(fi.random_field(3, (nt, nx, ny))), dfloat=True)),
                  O.apply_B(p, fi.random_field(3, (nt, nx, ny)))) < 1e-11
    x = fi.random_field(31, (nt, nx, ny))
    ref = O.apply_B(p, x)
    assert relerr(host(prob.matvec(dev(x, torch.float32))), ref) < 2e-5
    assert relerr(host(prob.matvec(dev(x))), ref) < 1e-12
    prob.close()


@pytest.mark.parametrize("tiles", [(128, 256), (256, 512), (128, 512), (256, 256), (512, 512)])
@pytest.mark.parametrize("dims", [(7, 5, 3), (33, 17, 6), (64, 64, 4), (100, 50, 3), (17, 300, 2), (2, 1100, 2)])
def test_every_float_tile_matches_oracle(dims, tiles):
    """Each float tile of the x2 and x1 passes: B, B^T and S against the oracle,
    with the epilogue."""
    need_gpu()
    F = lib()
    nx, ny, nt = dims
    p = params(nx, ny, nt)
    prob = F.Problem(p)
    rows, axis = tiles
    if ny > 2048 and rows == 128:
        rows = 0
    prob.set_tiles(rows, axis)
    x = fi.random_field(37, (nt, nx, ny))
    for op, tr in ((F.FDE_OP_B, False), (F.FDE_OP_BT, True)):
        assert relerr(host(prob.matvec(dev(x, torch.float32), op)), O.apply_B(p, x, transpose=tr)) < 2e-5
    fo = F.AdmmOptions(delta=0.7, rho=1.4)
    got = host(prob.matvec(dev(x, torch.float32), F.FDE_OP_S, fo))
    assert relerr(got, O.apply_S(p, O.AdmmOptions(delta=0.7, rho=1.4), x)) < 2e-5
    for axis_ in (1, 2):
        X, Y = O.space_matrices(p)
        M, along = (X, O.along_x1) if axis_ == 1 else (Y, O.along_x2)
        ref = -O.psi_scale(p) * along(M, x)
        assert relerr(host(prob.apply_factor(dev(x, torch.float32), axis_)), ref) < 2e-5
    prob.close()


def test_set_tiles_rejects_unknown_values():
    need_gpu()
    F = lib()
    prob = F.Problem(params(8, 8, 2))
    for bad in ((64, 0), (0, 1000), (-128, 0), (-256, 0), (0, -512)):
        with pytest.raises(F.FdeError) as e:
            prob.set_tiles(*bad)
        assert e.value.status == F.FDE_EINVAL
    for bad in ((64, 0), (512, 0), (0, 512), (-128, 0), (0, -256)):
        for kw in (dict(dfloat=True), dict(fp64=True)):
            with pytest.raises(F.FdeError) as e:
                prob.set_tiles(*bad, **kw)
            assert e.value.status == F.FDE_EINVAL
    prob.close()


@pytest.mark.parametrize("tiles", [(256, 256), (-512, -512), (-256, -512), (256, -512), (128, 128)])
@pytest.mark.parametrize("dims", [(7, 5, 3), (17, 33, 6), (64, 64, 4), (100, 50, 3), (31, 200, 2), (2, 1100, 2)])
def test_every_fp64_tile_matches_oracle(dims, tiles):
    """Each double tile of the x2 and x1 passes (both halves per thread, split
    halves): B, B^T and S with the epilogue, and the single factors, against the
    oracle; lines that fill the transform (64) and ragged ones."""
    need_gpu()
    F = lib()
    nx, ny, nt = dims
    p = params(nx, ny, nt)
    prob = F.Problem(p)
    rows, axis = tiles
    if ny > 2048 and rows in (-256, 128):
        rows = 0
    prob.set_tiles(rows, axis, fp64=True)
    assert prob.tiles(fp64=True) == (rows or 256, axis)
    x = fi.random_field(41, (nt, nx, ny))
    for op, tr in ((F.FDE_OP_B, False), (F.FDE_OP_BT, True)):
        assert relerr(host(prob.matvec(dev(x), op)), O.apply_B(p, x, transpose=tr)) < 1e-12
    fo = F.AdmmOptions(delta=0.7, rho=1.4)
    got = host(prob.matvec(dev(x), F.FDE_OP_S, fo))
    assert relerr(got, O.apply_S(p, O.AdmmOptions(delta=0.7, rho=1.4), x)) < 1e-12
    for axis_ in (1, 2):
        X, Y = O.space_matrices(p)
        M, along = (X, O.along_x1) if axis_ == 1 else (Y, O.along_x2)
        ref = -O.psi_scale(p) * along(M, x)
        assert relerr(host(prob.apply_factor(dev(x), axis_)), ref) < 1e-12
    prob.close()


@pytest.mark.parametrize("dims,alpha", [((4096, 3, 2), 1.0), ((2, 4096, 2), 1.0), ((3, 5, 4096), 0.6),
                                        ((2, 4095, 3), 1.0)])
def test_largest_axis_length(dims, alpha):
    """Axes of the largest supported length (4096: the 4096-point register FFT,
    three radix-16/16/16 passes) and a ragged 4095, in double, float and
    double-float (every double-float tile), against the oracle."""
    need_gpu()
    F = lib()
    nx, ny, nt = dims
    p = params(nx, ny, nt, alpha_t=alpha)
    prob = F.Problem(p)
    x = fi.random_field(53, (nt, nx, ny))
    xd = dev(x)
    for op, tr in ((F.FDE_OP_B, False), (F.FDE_OP_BT, True)):
        ref = O.apply_B(p, x, transpose=tr)
        assert relerr(host(prob.matvec(xd, op)), ref) < 1e-12
        assert relerr(host(prob.matvec(xd.float(), op)), ref) < 5e-5
        for rows, axis in ((256, 256), (-512, -512), (256, 128)):
            prob.set_tiles(rows, axis, dfloat=True)
            assert relerr(host(prob.matvec(xd, op, dfloat=True)), ref) < 1e-11, (rows, axis)
            prob.set_tiles(rows, axis, fp64=True)
            assert relerr(host(prob.matvec(xd, op)), ref) < 1e-12, (rows, axis)
        prob.set_tiles(256, 256, fp64=True)
    prob.close()


@pytest.mark.parametrize("precond", [0, 1])
def test_preconditioner_full_size_properties(precond):
    """1024^2 x 128 (the benchmark's grid): S-tilde^-1 (and the matching S-hat^-1)
    is symmetric and positive definite, <M x, w> = <x, M w> and <M x, x> > 0, and the
    float application agrees with the double one."""
    need_gpu()
    F = lib()
    inst = fi.config_large()
    prob = F.Problem(inst.params)
    fo = F.AdmmOptions(delta=1.0, rho=1.618, precond=precond)
    x = dev(inst.ybar)
    w = dev(fi.random_field(61, prob.shape))
    mx = prob.precond(x, fo)
    mw = prob.precond(w, fo)
    a = float(torch.dot(mx, w))
    b = float(torch.dot(x, mw))
    assert abs(a - b) <= 1e-10 * max(abs(a), abs(b)), (a, b)
    assert float(torch.dot(mx, x)) > 0 and float(torch.dot(mw, w)) > 0
    m32 = prob.precond(x.float(), fo)
    scale = float(mx.abs().max())
    assert float((m32.double() - mx).abs().max()) / scale < 1e-4
    del mx, mw, m32, x, w
    prob.close()
    torch.cuda.empty_cache()
