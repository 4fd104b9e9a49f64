"""The allocation-free Toeplitz product (fde_matvec_noalloc) against fde_matvec.

fde_matvec_noalloc serves callers that cannot call cudaMalloc (a plug-in whose
host framework owns the device memory, a serving path that must not allocate):
it keeps its intermediates and tables in one fixed device array instead of a
workspace from fde_setup. This file is collected last so that a run stopping
at its first failure has already run every other test; it must pass alone in
a fresh process and after the rest of the suite."""
import ctypes

import numpy as np
import pytest
import torch

import fde_inputs as fi
import oracle as O
from gpu_util import dev, host, lib, need_gpu, params, relerr

pytestmark = pytest.mark.gpu


def _noalloc(F, p, op, x, y):
    ps = F.params_struct(p)
    return F.lib().fde_matvec_noalloc(ctypes.byref(ps), op, ctypes.c_void_p(x.data_ptr()),
                                      ctypes.c_void_p(y.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("dims,alpha", [((64, 48, 16), 1.0), ((33, 17, 6), 0.6), ((128, 128, 64), 1.0)])
def test_noalloc_matches_fde_matvec_on_two_calls(dims, alpha):
    need_gpu()
    F = lib()
    nx, ny, nt = dims
    p = params(nx, ny, nt, alpha_t=alpha)
    prob = F.Problem(p)
    for call in range(2):  # two calls in a row share the fixed array
        x = dev(fi.random_field(100 + call, (nt, nx, ny)))
        for op in (F.FDE_OP_B, F.FDE_OP_BT):
            ref = host(prob.matvec(x, op))
            y = torch.full_like(x, float("nan"))
            assert _noalloc(F, p, op, x, y) == F.FDE_OK
            torch.cuda.synchronize()
            assert relerr(host(y), ref) < 1e-12, (call, op, relerr(host(y), ref))
    prob.close()


@pytest.mark.parametrize("dims,alpha", [((8, 6, 20), 0.6), ((5, 19, 3), 1.0)])
def test_noalloc_matches_the_oracle(dims, alpha):
    """Independently of fde_matvec (which shares the transform kernels): B x and
    B^T x against the FP64 oracle's per-axis dense products, including a time
    axis of 20 steps with alpha_t = 0.6 (the embedded time transform of length 32)."""
    need_gpu()
    F = lib()
    nx, ny, nt = dims
    p = params(nx, ny, nt, alpha_t=alpha)
    x = fi.random_field(7, (nt, nx, ny))
    for op, tr in ((F.FDE_OP_B, False), (F.FDE_OP_BT, True)):
        y = torch.full((p.N,), float("nan"), dtype=torch.float64, device="cuda")
        assert _noalloc(F, p, op, dev(x), y) == F.FDE_OK
        torch.cuda.synchronize()
        assert relerr(host(y), O.apply_B(p, x, transpose=tr)) < 1e-12, (dims, op)


def test_noalloc_rejects_sizes_beyond_its_array():
    need_gpu()
    F = lib()
    p = params(1024, 1024, 2)  # 2M points > 1M
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    y = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert _noalloc(F, p, F.FDE_OP_B, x, y) == F.FDE_EUNSUPPORTED
    assert _noalloc(F, params(4, 4, 4), 5, x, y) == F.FDE_EINVAL
