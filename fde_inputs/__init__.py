"""Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.

This module holds only input construction: a counter-based generator
(splitmix64, Steele/Lea/Flood 2014), Box-Muller normals, the interior grid
coordinates and the desired-state fields of the five workloads. It holds none
of the method's arithmetic (no weights, operators, projections or solves), so
that the oracle and the CUDA path can both use it without sharing code.

Layout of every field: C-order ``[t][x1][x2]`` (x2 fastest), interior points
x1_i = i*h_x (i = 1..nx), x2_j = j*h_y (j = 1..ny), times t_k = k*h_t
(k = 1..nt); t = 0 is excluded because the initial state is zero.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

_MASK = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def splitmix64(seed: int, count: int) -> np.ndarray:
    """``count`` outputs of splitmix64 started from ``seed`` (uint64 array).

    Output i is the finaliser applied to ``seed + (i+1)*golden`` (mod 2^64),
    which is the published sequential definition written counter-wise.
    """
    i = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK) + i * np.uint64(_GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of splitmix64."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller on pairs of uniforms (u1 in (0, 1])."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m)
    u1 = 1.0 - u[0::2]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * math.pi * u2)
    z[1::2] = r * np.sin(2.0 * math.pi * u2)
    return z[:count]


@dataclasses.dataclass
class FdeParams:
    """Problem description; mirrors the C struct ``fde_params``.

    beta_x, beta_y: spatial orders in (1, 2); alpha_t: time order in (0, 1]
    (1 = implicit Euler). dp/dm and ep/em: coefficients of the left/right
    shifted Gruenwald-Letnikov matrices along x1 and x2. gamma: control
    regularisation. weights: 0 = trapezoid in time (last slice 1/2), 1 =
    uniform. time_step_mode: 0 -> h_t = T/nt, 1 -> h_t = h_x (paper grids).
    """
    nx: int
    ny: int
    nt: int
    T: float = 1.0
    beta_x: float = 1.5
    beta_y: float = 1.5
    alpha_t: float = 1.0
    dp: float = 1.0
    dm: float = 1.0
    ep: float = 1.0
    em: float = 1.0
    gamma: float = 1e-4
    weights: int = 0
    time_step_mode: int = 0

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nt


@dataclasses.dataclass
class FdeInstance:
    """Inputs of one solve: parameters, desired state, forcing and box bounds.

    Bounds are scalars (broadcast) or None (unbounded).
    """
    params: FdeParams
    ybar: np.ndarray
    g: Optional[np.ndarray]
    ya: Optional[float]
    yb: Optional[float]
    ua: Optional[float]
    ub: Optional[float]
    seed: int


def grid(p: FdeParams):
    """Interior coordinates (x1, x2, t) as 1-D arrays."""
    hx = 1.0 / (p.nx + 1)
    hy = 1.0 / (p.ny + 1)
    ht = p.T / p.nt if p.time_step_mode == 0 else hx
    x1 = hx * np.arange(1, p.nx + 1)
    x2 = hy * np.arange(1, p.ny + 1)
    t = ht * np.arange(1, p.nt + 1)
    return x1, x2, t


def desired_state_sine(p: FdeParams, seed: int, sigma: float = 0.1) -> np.ndarray:
    """ybar = sin(pi x1) sin(pi x2) t + N(0, sigma^2) noise, layout [t][x1][x2]."""
    x1, x2, t = grid(p)
    base = t[:, None, None] * np.sin(np.pi * x1)[None, :, None] * np.sin(np.pi * x2)[None, None, :]
    noise = normal(seed, p.N).reshape(p.nt, p.nx, p.ny)
    return base + sigma * noise


def desired_state_paper(p: FdeParams) -> np.ndarray:
    """Section 6.1 test state 10 cos(10 x1) sin(x1 x2) (1 - exp(-5 t))."""
    x1, x2, t = grid(p)
    X1 = x1[None, :, None]
    X2 = x2[None, None, :]
    tt = t[:, None, None]
    return 10.0 * np.cos(10.0 * X1) * np.sin(X1 * X2) * (1.0 - np.exp(-5.0 * tt))


def random_field(seed: int, shape, scale: float = 1.0) -> np.ndarray:
    """Standard-normal test vector of the given shape."""
    n = int(np.prod(shape))
    return scale * normal(seed, n).reshape(shape)


MASTER_SEED = 1907


def config_small() -> FdeInstance:
    """32x32 interior grid, 16 implicit-Euler steps, control box [-0.5, 0.5]."""
    p = FdeParams(nx=32, ny=32, nt=16, T=1.0, beta_x=1.5, beta_y=1.7, alpha_t=1.0,
                  dp=1.0, dm=0.5, ep=0.8, em=0.3, gamma=1e-4)
    return FdeInstance(p, desired_state_sine(p, MASTER_SEED), None, None, None, -0.5, 0.5, MASTER_SEED)


def config_medium() -> FdeInstance:
    """256x256 x 64 steps, state box y <= 0.8 and control box [-1, 1]."""
    p = FdeParams(nx=256, ny=256, nt=64, T=1.0, beta_x=1.3, beta_y=1.8, alpha_t=1.0,
                  dp=1.0, dm=0.5, ep=0.8, em=0.3, gamma=1e-4)
    return FdeInstance(p, desired_state_sine(p, MASTER_SEED), None, None, 0.8, -1.0, 1.0, MASTER_SEED)


def config_large() -> FdeInstance:
    """1024x1024 x 128 steps, anisotropic coefficients, control box [-1, 1]."""
    p = FdeParams(nx=1024, ny=1024, nt=128, T=1.0, beta_x=1.7, beta_y=1.2, alpha_t=1.0,
                  dp=2.0, dm=0.1, ep=0.5, em=0.5, gamma=1e-6)
    return FdeInstance(p, desired_state_sine(p, MASTER_SEED), None, None, None, -1.0, 1.0, MASTER_SEED)


def config_large_slab() -> FdeInstance:
    """The 1024x1024 operator of config_large on 16 time steps (profiling case:
    the same transform lengths, vectors larger than L2, a few GB on the device)."""
    inst = config_large()
    p = FdeParams(**{**inst.params.__dict__, "nt": 16})
    return FdeInstance(p, desired_state_sine(p, MASTER_SEED), None, None, None, -1.0, 1.0, MASTER_SEED)


def config_grad() -> FdeInstance:
    """256x256 x 64 steps, beta = 1.5 on both axes, control box [-1, 1]."""
    p = FdeParams(nx=256, ny=256, nt=64, T=1.0, beta_x=1.5, beta_y=1.5, alpha_t=1.0,
                  dp=1.0, dm=0.5, ep=0.8, em=0.3, gamma=1e-4)
    return FdeInstance(p, desired_state_sine(p, MASTER_SEED), None, None, None, -1.0, 1.0, MASTER_SEED)


def config_grad_small() -> FdeInstance:
    """The differentiation workload's operator on the 32x32 x 16 grid."""
    p = FdeParams(nx=32, ny=32, nt=16, T=1.0, beta_x=1.5, beta_y=1.5, alpha_t=1.0,
                  dp=1.0, dm=0.5, ep=0.8, em=0.3, gamma=1e-4)
    return FdeInstance(p, desired_state_sine(p, MASTER_SEED), None, None, None, -1.0, 1.0, MASTER_SEED)


def config_batch_params(count: int = 64, seed0: int = MASTER_SEED):
    """Parameters and control bounds of the uneven batch: grids {64^2,128^2,256^2,512^2},
    nt {16,32,64}, orders U(1.1,1.9), gamma log-uniform in [1e-6, 1e-2],
    u_b ~ U(0.25, 2), u_a = -U(0.25, 2). Returns [(params, ua, ub, seed)]."""
    out = []
    for k in range(count):
        s = seed0 + k
        u = uniform01(s ^ 0x5EED, 8)
        n = (64, 128, 256, 512)[int(u[0] * 4)]
        nt = (16, 32, 64)[int(u[1] * 3)]
        bx = 1.1 + 0.8 * u[2]
        by = 1.1 + 0.8 * u[3]
        gamma = 10.0 ** (-6.0 + 4.0 * u[4])
        ub = 0.25 + 1.75 * u[5]
        ua = -(0.25 + 1.75 * u[6])
        p = FdeParams(nx=n, ny=n, nt=nt, T=1.0, beta_x=bx, beta_y=by, alpha_t=1.0,
                      dp=1.0, dm=0.5, ep=0.8, em=0.3, gamma=gamma)
        out.append((p, ua, ub, s))
    return out


def config_batch(count: int = 64, seed0: int = MASTER_SEED):
    """The uneven batch with desired states (see config_batch_params)."""
    return [FdeInstance(p, desired_state_sine(p, s), None, None, None, ua, ub, s)
            for p, ua, ub, s in config_batch_params(count, seed0)]
