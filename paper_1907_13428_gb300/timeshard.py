"""One problem instance across ranks: the [t][x1][x2] vectors partitioned by
time slices (host-side exchange logic; one process per GPU).

The operator B = psi (C_t (x) I - I (x) X (x) I - I (x) I (x) Y) of
Eq. (FDE constraint matrix) acts slice by slice in space, so a rank holding
the slices [t0, t1) applies the two spatial Toeplitz factors on its own data.
The time term couples slices:
  * implicit Euler (alpha_t = 1): B's row block t needs x_{t-1}, B^T's needs
    x_{t+1}. A rank sends its last slice to the next rank and its first slice
    to the previous one (a one-slice halo), then applies the operator to the
    extended block [x_{t0-1}, x_{t0..t1-1}] (or [x_{t0..t1-1}, x_{t1}]) and
    drops the halo's own output row: the extended block's backward difference
    at its first interior slice is exactly the global one.
  * alpha_t < 1 (the Gruenwald-Letnikov time matrix, lower triangular in t,
    Eq. (Caputo matrix)): every slice depends on all earlier ones, so the time
    term is applied on t-pencils: an all-to-all gives each rank all nt slices
    of a band of x1 rows, the time Toeplitz acts along t there, and a second
    all-to-all brings the result back.
The multilevel circulant preconditioner of Section 5 is a three-level DFT, a
divide by sigma and the inverse DFT. Its two spatial levels are local to a
time slice; the time level needs whole t-lines. With a pencil transpose (one
all-to-all each way) every rank applies the time DFT, the divide and the
inverse time DFT to all nt entries of its band of x1 frequencies.
PCG and ADMM scalars (inner products, objective) are all-reduced sums in FP64;
the ADMM residual infinity norms are all-reduced maxima.

The local arithmetic comes from a backend (an object with the methods named
in `Backend`); this module only partitions, exchanges and assembles.
Collectives go through torch.distributed (NCCL between GPUs, gloo on CPU).
"""
from __future__ import annotations

from typing import Callable, List, Optional, Protocol, Sequence, Tuple

import torch
import torch.distributed as dist


def block_ranges(n: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous, balanced [start, stop) blocks of n items over `world` ranks:
    the first n % world ranks get one item more. Every rank gets at least one
    item (n >= world is required)."""
    if world < 1 or n < world:
        raise ValueError(f"cannot split {n} items over {world} ranks")
    base, extra = divmod(n, world)
    out, s = [], 0
    for r in range(world):
        c = base + (1 if r < extra else 0)
        out.append((s, s + c))
        s += c
    return out


class Backend(Protocol):
    """Local arithmetic on one rank's data (tensors of float64)."""

    def apply_B(self, x: torch.Tensor, transpose: bool) -> torch.Tensor:
        """B (or B^T) of a standalone block of x.shape[0] consecutive time slices,
        with the block's own zero history (x_{-1} = 0 for B, x_{n} = 0 for B^T);
        implicit Euler only."""

    def apply_space(self, x: torch.Tensor, transpose: bool) -> torch.Tensor:
        """-psi (X (x) I + I (x) Y) (or its transpose) on every slice of x."""

    def apply_time(self, pencil: torch.Tensor, transpose: bool) -> torch.Tensor:
        """psi C_t (or psi C_t^T) along axis 0 of a t-pencil (nt, ...)."""

    def spatial_dft(self, x: torch.Tensor, inverse: bool) -> torch.Tensor:
        """Two-level DFT over (x1, x2) of every slice: real slices to complex
        spectra, or (inverse) complex spectra back to real slices."""

    def time_solve(self, pencil: torch.Tensor, k1: Tuple[int, int]) -> torch.Tensor:
        """Time DFT, divide by sigma(k_t, k1, k2) for the x1 frequencies
        k1[0] <= k1 < k1[1], inverse time DFT, on a complex t-pencil
        (nt, k1[1] - k1[0], ny). Together with spatial_dft the three steps give
        F^-1 diag(1/sigma) F with the normalisation of the inverse included once."""


class TimeShard:
    """Rank-local view of an nt x nx x ny problem partitioned by time slices.
    Without an initialised process group it is the single-rank case."""

    def __init__(self, nt: int, nx: int, ny: int, rank: Optional[int] = None, world: Optional[int] = None,
                 group=None):
        self.group = group
        if world is None:
            world = dist.get_world_size(group) if dist.is_available() and dist.is_initialized() else 1
        if rank is None:
            rank = dist.get_rank(group) if world > 1 else 0
        self.nt, self.nx, self.ny = nt, nx, ny
        self.rank, self.world = rank, world
        self.t_blocks = block_ranges(nt, world)
        self.x1_blocks = block_ranges(nx, world)
        self.t0, self.t1 = self.t_blocks[rank]
        self.nloc = self.t1 - self.t0

    # ---- partition ----------------------------------------------------------
    def local(self, full: torch.Tensor) -> torch.Tensor:
        """This rank's slices of a full (nt, nx, ny) array."""
        return full.reshape(self.nt, self.nx, self.ny)[self.t0:self.t1].contiguous()

    def gather(self, x_local: torch.Tensor) -> torch.Tensor:
        """The full (nt, ...) array from every rank's slices (for checks and output)."""
        if self.world == 1:
            return x_local
        # blocks differ by at most one slice: gather padded blocks of equal size, then trim
        sizes = [b - a for a, b in self.t_blocks]
        m = max(sizes)
        rest = tuple(x_local.shape[1:])
        pad = torch.zeros((m,) + rest, dtype=x_local.dtype, device=x_local.device)
        pad[:self.nloc] = x_local
        parts = [torch.empty((m,) + rest, dtype=x_local.dtype, device=x_local.device) for _ in sizes]
        dist.all_gather(parts, pad, group=self.group)
        return torch.cat([p[:s] for p, s in zip(parts, sizes)], 0)

    # ---- halo exchange (implicit Euler) --------------------------------------
    def _shift(self, send: torch.Tensor, to_next: bool) -> torch.Tensor:
        """Send `send` to the next (to_next) or previous rank and receive the
        matching slice from the other side; zeros at the ends of the time axis."""
        recv = torch.zeros_like(send)
        if self.world == 1:
            return recv
        dst = self.rank + 1 if to_next else self.rank - 1
        src = self.rank - 1 if to_next else self.rank + 1
        ops = []
        if 0 <= dst < self.world:
            ops.append(dist.P2POp(dist.isend, send.contiguous(), self._global(dst), group=self.group))
        if 0 <= src < self.world:
            ops.append(dist.P2POp(dist.irecv, recv, self._global(src), group=self.group))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        return recv

    def _global(self, r: int) -> int:
        return r if self.group is None else dist.get_global_rank(self.group, r)

    def halo_prev(self, x_local: torch.Tensor) -> torch.Tensor:
        """x_{t0-1}: the previous rank's last slice (zero on rank 0)."""
        return self._shift(x_local[-1], to_next=True)

    def halo_next(self, x_local: torch.Tensor) -> torch.Tensor:
        """x_{t1}: the next rank's first slice (zero on the last rank)."""
        return self._shift(x_local[0], to_next=False)

    # ---- t-pencil transposes -------------------------------------------------
    def to_pencils(self, x_local: torch.Tensor) -> torch.Tensor:
        """(nloc, nx, ny) time block -> (nt, nx_band, ny) pencil of this rank's
        band of x1 rows (all-to-all)."""
        a, b = self.x1_blocks[self.rank]
        if self.world == 1:
            return x_local.contiguous()
        send = [x_local[:, s:e].contiguous() for s, e in self.x1_blocks]
        recv = [torch.empty((t1 - t0, b - a) + tuple(x_local.shape[2:]), dtype=x_local.dtype,
                            device=x_local.device) for t0, t1 in self.t_blocks]
        self._all_to_all(recv, send)
        return torch.cat(recv, 0)

    def from_pencils(self, pencil: torch.Tensor) -> torch.Tensor:
        """Inverse of to_pencils: (nt, nx_band, ny) -> (nloc, nx, ny)."""
        if self.world == 1:
            return pencil.contiguous()
        send = [pencil[t0:t1].contiguous() for t0, t1 in self.t_blocks]
        recv = [torch.empty((self.nloc, e - s) + tuple(pencil.shape[2:]), dtype=pencil.dtype,
                            device=pencil.device) for s, e in self.x1_blocks]
        self._all_to_all(recv, send)
        return torch.cat(recv, 1)

    def _all_to_all(self, recv: List[torch.Tensor], send: List[torch.Tensor]):
        """All-to-all of tensor lists; gloo has no all_to_all, so it is built from
        point-to-point messages there. Complex tensors travel as real views."""
        def real(t):
            return torch.view_as_real(t) if t.is_complex() else t
        if dist.get_backend(self.group) == "nccl":
            dist.all_to_all([real(t) for t in recv], [real(t) for t in send], group=self.group)
            return
        ops = []
        for r in range(self.world):
            if r == self.rank:
                recv[r].copy_(send[r])
                continue
            ops.append(dist.P2POp(dist.isend, real(send[r]), self._global(r), group=self.group))
            ops.append(dist.P2POp(dist.irecv, real(recv[r]), self._global(r), group=self.group))
        for req in dist.batch_isend_irecv(ops):
            req.wait()

    # ---- scalars -------------------------------------------------------------
    def allreduce_sum(self, v: float) -> float:
        """Sum over ranks in FP64 (inner products, objective)."""
        if self.world == 1:
            return float(v)
        t = torch.tensor([float(v)], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return float(t.item())

    def allreduce_max(self, v: float) -> float:
        """Maximum over ranks (ADMM residual infinity norms)."""
        if self.world == 1:
            return float(v)
        t = torch.tensor([float(v)], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=self.group)
        return float(t.item())

    def dot(self, a: torch.Tensor, b: torch.Tensor) -> float:
        return self.allreduce_sum(float(torch.sum(a * b)))

    # ---- operators -----------------------------------------------------------
    def apply_B(self, be: Backend, x_local: torch.Tensor, transpose: bool = False, euler: bool = True
                ) -> torch.Tensor:
        """B x (or B^T x) of the full problem, rank-local rows."""
        if euler:
            if not transpose:
                ext = torch.cat([self.halo_prev(x_local)[None], x_local], 0)
                return be.apply_B(ext, False)[1:]
            ext = torch.cat([x_local, self.halo_next(x_local)[None]], 0)
            return be.apply_B(ext, True)[:-1]
        space = be.apply_space(x_local, transpose)
        time = self.from_pencils(be.apply_time(self.to_pencils(x_local), transpose))
        return space + time

    def apply_precond(self, be: Backend, r_local: torch.Tensor) -> torch.Tensor:
        """S-tilde^-1 r: spatial DFTs on the time block, time solve on t-pencils of
        the x1 frequency bands, inverse spatial DFTs."""
        spec = be.spatial_dft(r_local, inverse=False)
        pencil = be.time_solve(self.to_pencils(spec), self.x1_blocks[self.rank])
        return be.spatial_dft(self.from_pencils(pencil), inverse=True)

    def pcg(self, apply_A: Callable[[torch.Tensor], torch.Tensor], apply_M: Callable[[torch.Tensor], torch.Tensor],
            b: torch.Tensor, x0: torch.Tensor, tol: float, max_iter: int) -> Tuple[torch.Tensor, int]:
        """Preconditioned CG on rank-local blocks: the operators exchange what they
        need, every inner product is an FP64 all-reduced sum, so all ranks take
        the same decisions. Stops when ||b - A x|| <= tol ||b|| (recursive residual)."""
        x = x0.clone()
        r = b - apply_A(x)
        bb = self.dot(b, b)
        if bb == 0.0:
            return torch.zeros_like(b), 0
        thr = tol * tol * bb
        if self.dot(r, r) <= thr:
            return x, 0
        z = apply_M(r)
        d = z.clone()
        rz = self.dot(r, z)
        for it in range(1, max_iter + 1):
            q = apply_A(d)
            alpha = rz / self.dot(d, q)
            x += alpha * d
            r -= alpha * q
            if self.dot(r, r) <= thr:
                return x, it
            z = apply_M(r)
            rz_new = self.dot(r, z)
            d = z + (rz_new / rz) * d
            rz = rz_new
        return x, max_iter


def residual_norms(shard: TimeShard, parts: Sequence[torch.Tensor]) -> List[float]:
    """Infinity norms of rank-local residual blocks, maximised over ranks."""
    return [shard.allreduce_max(float(p.abs().max())) if p.numel() else shard.allreduce_max(0.0) for p in parts]


class LibraryBackend:
    """Rank-local B and B^T through the library (implicit Euler, the halo path):
    a block of n consecutive slices is a problem of its own with the same
    spatial grid, orders, coefficients and time step (T = n h_t), whose
    fde_matvec starts from a zero history, so TimeShard.apply_B on the extended
    block gives the global rows. One problem handle per block length is kept.
    The preconditioner stages and the alpha_t < 1 pencil path have no library
    backend (their exchange logic is exercised with a host backend)."""

    def __init__(self, params):
        import dataclasses
        if params.alpha_t != 1.0:
            raise ValueError("the library backend covers implicit Euler (alpha_t = 1)")
        self.params = params
        hx = 1.0 / (params.nx + 1)
        self.ht = params.T / params.nt if params.time_step_mode == 0 else hx
        self._replace = dataclasses.replace
        self._probs = {}

    def _problem(self, n):
        from . import Problem
        if n not in self._probs:
            q = self._replace(self.params, nt=n, T=self.ht * n)
            self._probs[n] = Problem(q)
        return self._probs[n]

    def apply_B(self, x: torch.Tensor, transpose: bool) -> torch.Tensor:
        from . import FDE_OP_B, FDE_OP_BT
        prob = self._problem(x.shape[0])
        y = prob.matvec(x.contiguous().view(-1), FDE_OP_BT if transpose else FDE_OP_B)
        return y.view(x.shape)

    def close(self):
        for p in self._probs.values():
            p.close()
        self._probs.clear()
