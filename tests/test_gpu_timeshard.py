"""The library side of the time-slice partition on one GPU: every block of a
split of the time axis, extended by its one-slice halo and applied as a
problem of its own (timeshard.LibraryBackend), reproduces its rows of the
full problem's B and B^T (the exchanges themselves are tested on CPU ranks)."""
import numpy as np
import pytest
import torch

import fde_inputs as fi
from gpu_util import dev, lib, need_gpu, params, relerr

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,world", [((12, 10, 7), 2), ((32, 64, 9), 3), ((20, 36, 5), 5)])
def test_extended_blocks_reproduce_the_full_operator(dims, world):
    need_gpu()
    F = lib()
    from paper_1907_13428_gb300 import timeshard
    nx, ny, nt = dims
    p = params(nx, ny, nt)
    prob = F.Problem(p)
    x = dev(fi.random_field(21, (nt, nx, ny))).view(nt, nx, ny)
    be = timeshard.LibraryBackend(p)
    for op, transpose in ((F.FDE_OP_B, False), (F.FDE_OP_BT, True)):
        full = prob.matvec(x.reshape(-1), op).view(nt, nx, ny)
        rows = []
        for t0, t1 in timeshard.block_ranges(nt, world):
            if not transpose:
                prev = x[t0 - 1:t0] if t0 > 0 else torch.zeros_like(x[:1])
                rows.append(be.apply_B(torch.cat([prev, x[t0:t1]], 0), False)[1:])
            else:
                nxt = x[t1:t1 + 1] if t1 < nt else torch.zeros_like(x[:1])
                rows.append(be.apply_B(torch.cat([x[t0:t1], nxt], 0), True)[:-1])
        got = torch.cat(rows, 0)
        assert relerr(got.cpu().numpy(), full.cpu().numpy()) < 1e-13, (op, dims, world)
    be.close()
    prob.close()
