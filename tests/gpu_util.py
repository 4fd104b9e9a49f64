"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest
import torch

import fde_inputs as fi


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def lib():
    import paper_1907_13428_gb300 as F
    F.lib()  # raises if the library was not built: the CUDA path is mandatory
    return F


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a).ravel(), dtype=dtype, device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


def relerr(got, ref):
    got = np.asarray(got, float).ravel()
    ref = np.asarray(ref, float).ravel()
    scale = max(np.max(np.abs(ref)), 1e-300)
    return float(np.max(np.abs(got - ref)) / scale)


def params(nx, ny, nt, **kw):
    base = dict(T=1.0, beta_x=1.45, beta_y=1.7, alpha_t=1.0, dp=1.0, dm=0.5, ep=0.8, em=0.3, gamma=1e-3)
    base.update(kw)
    return fi.FdeParams(nx=nx, ny=ny, nt=nt, **base)
