"""Time-slice partition of one instance across CPU ranks (gloo, world sizes 2
and 3): B, B^T (implicit Euler with the one-slice halo, and alpha_t < 1 with
t-pencil transposes), the multilevel circulant preconditioner (spatial DFTs
on time blocks, time solve on t-pencils) and a PCG solve of S y = b with
all-reduced FP64 inner products, each equal to the oracle's single-process
result. The local arithmetic of every rank is the oracle's, applied to the
rank's block: the test checks the partition, the halos, the transposes and
the reductions."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import fde_inputs as fi
import oracle as O
from paper_1907_13428_gb300 import timeshard


class OracleBackend:
    """Rank-local arithmetic from the oracle (test infrastructure)."""

    def __init__(self, p, o):
        self.p, self.o = p, o

    def _block(self, n):
        _, _, ht = O.mesh(self.p)
        return fi.FdeParams(**{**self.p.__dict__, "nt": n, "T": ht * n})

    def apply_B(self, x, transpose):
        q = self._block(x.shape[0])
        return torch.as_tensor(O.apply_B(q, x.numpy(), transpose=transpose))

    def apply_space(self, x, transpose):
        X, Y = O.space_matrices(self.p)
        if transpose:
            X, Y = X.T, Y.T
        v = x.numpy()
        return torch.as_tensor(-O.psi_scale(self.p) * (O.along_x1(X, v) + O.along_x2(Y, v)))

    def apply_time(self, pencil, transpose):
        C = O.caputo_matrix(self.p)
        if transpose:
            C = C.T
        v = pencil.numpy()
        return torch.as_tensor(O.psi_scale(self.p) * (C @ v.reshape(v.shape[0], -1)).reshape(v.shape))

    def spatial_dft(self, x, inverse):
        v = x.numpy()
        if inverse:
            return torch.as_tensor(np.fft.ifft2(v, axes=(1, 2)).real.copy())
        return torch.as_tensor(np.fft.fft2(v, axes=(1, 2)))

    def time_solve(self, pencil, k1):
        sigma = O.preconditioner_symbol(self.p, self.o)[:, k1[0]:k1[1], :]
        v = np.fft.ifft(np.fft.fft(pencil.numpy(), axis=0) / sigma, axis=0)
        return torch.as_tensor(v)


def _problem(alpha_t):
    return fi.FdeParams(nx=7, ny=6, nt=9, T=1.0, beta_x=1.45, beta_y=1.7, alpha_t=alpha_t, dp=1.0, dm=0.5, ep=0.8,
                        em=0.3, gamma=1e-3)


def test_block_ranges_partition_and_balance():
    for n in (1, 5, 9, 128):
        for world in range(1, min(n, 8) + 1):
            blocks = timeshard.block_ranges(n, world)
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            assert all(a < b for a, b in blocks)
            assert all(blocks[i][1] == blocks[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        timeshard.block_ranges(3, 4)


def test_single_rank_view_without_process_group():
    p = _problem(1.0)
    o = O.AdmmOptions(delta=1.0, rho=1.618)
    sh = timeshard.TimeShard(p.nt, p.nx, p.ny)
    assert (sh.rank, sh.world, sh.t0, sh.t1) == (0, 1, 0, p.nt)
    x = fi.random_field(5, (p.nt, p.nx, p.ny))
    be = OracleBackend(p, o)
    got = sh.apply_B(be, torch.as_tensor(x)).numpy()
    assert np.max(np.abs(got - O.apply_B(p, x))) <= 1e-13 * np.max(np.abs(got))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _relerr(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.set_num_threads(1)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out = {}
    try:
        o = O.AdmmOptions(delta=1.0, rho=1.618)
        for alpha_t in (1.0, 0.6):
            p = _problem(alpha_t)
            be = OracleBackend(p, o)
            sh = timeshard.TimeShard(p.nt, p.nx, p.ny)
            x = fi.random_field(11, (p.nt, p.nx, p.ny))
            xl = torch.as_tensor(sh.local(torch.as_tensor(x)).numpy())
            euler = alpha_t == 1.0
            for tr in (False, True):
                got = sh.gather(sh.apply_B(be, xl, transpose=tr, euler=euler)).numpy()
                out[("B", alpha_t, tr)] = _relerr(got, O.apply_B(p, x, transpose=tr))
            if not euler:
                continue
            r = fi.random_field(12, (p.nt, p.nx, p.ny))
            rl = sh.local(torch.as_tensor(r))
            z = sh.gather(sh.apply_precond(be, rl)).numpy()
            out["precond"] = _relerr(z, O.apply_preconditioner(p, o, r))
            # PCG on S y = b with S = M1 + B^T M2^-1 B, rank-local diagonals
            M1, _, M2 = O.admm_diagonals(p, o)
            M1l, M2l = sh.local(torch.as_tensor(M1)), sh.local(torch.as_tensor(M2))

            def A(v):
                return M1l * v + sh.apply_B(be, sh.apply_B(be, v) / M2l, transpose=True)

            b = fi.random_field(13, (p.nt, p.nx, p.ny))
            y, it = sh.pcg(A, lambda v: sh.apply_precond(be, v), sh.local(torch.as_tensor(b)),
                           torch.zeros(sh.nloc, p.nx, p.ny, dtype=torch.float64), 1e-12, 500)
            yref, itref = O.pcg(lambda v: O.apply_S(p, o, v), lambda v: O.apply_preconditioner(p, o, v), b,
                                np.zeros_like(b), 1e-12, 500)
            out["pcg"] = _relerr(sh.gather(y).numpy(), yref)
            out["pcg_iters"] = (it, itref)
            # infinity norms and sums over ranks
            res = timeshard.residual_norms(sh, [xl, torch.zeros(0)])
            out["maxnorm"] = (res[0], float(np.max(np.abs(x))), res[1])
            out["sum"] = (sh.allreduce_sum(float(xl.sum())), float(x.sum()))
        q.put((rank, out))
    except Exception as e:  # report to the parent instead of hanging it
        q.put((rank, repr(e)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_time_partition_matches_single_process_oracle(world):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, out in res:
        assert isinstance(out, dict), out
        for key in (("B", 1.0, False), ("B", 1.0, True), ("B", 0.6, False), ("B", 0.6, True)):
            assert out[key] < 1e-13, (rank, key, out[key])
        assert out["precond"] < 1e-13, out["precond"]
        assert out["pcg"] < 1e-10, out["pcg"]
        it, itref = out["pcg_iters"]
        assert abs(it - itref) <= 1, (it, itref)
        assert out["maxnorm"][0] == out["maxnorm"][1] and out["maxnorm"][2] == 0.0
        s, sref = out["sum"]
        assert abs(s - sref) <= 1e-12 * max(1.0, abs(sref))
