"""FP64 CPU oracle for the ADMM / Toeplitz hot path.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import or call this module.
The CUDA library never calls it and shares no code with it; the only common
code is ``fde_inputs`` (seeded inputs, no method arithmetic).

Everything here is plain NumPy/SciPy in float64, written from Pougkakiotis,
Pearson, Leveque and Gondzio, "Fast Solution Methods for Convex Fractional
Differential Equation Optimization" (arXiv:1907.13428). Citations name the
paper's section and equation labels.

Layout: vectors are arrays of shape (nt, nx, ny) in C order, i.e. the
lexicographic ordering of Section 2 with x2 fastest and time slowest, which is
the ordering the Kronecker form of Eq. (FDE constraint matrix) implies.

Readings of the paper used here (every one is also listed in the design notes):
  * time order alpha_t in (0, 1]; alpha_t = 1 gives the weights [1, -1, 0, ...]
    (implicit Euler), the workloads' time scheme;
  * the spatial operator generalises the Riesz matrix of Eq. (Riesz matrix) to
    X = d+ L + d- L^T (left/right coefficients), the Riesz case being
    d+ = d- = -1/(2 cos(beta pi / 2));
  * h_x = 1/(nx+1), h_y = 1/(ny+1); h_t = T/nt, or h_t = h_x in paper mode;
  * the psi-scaled ADMM of Section 6.1: constraints B y + psi u = psi g,
    y = z_y, psi u = psi z_u, all with penalty 1/(2 delta);
  * J1 = diag(w), J2 = gamma diag(w), w = 1 except 1/2 on the last time slice
    (trapezoid, Eq. (discretized Objective function)), or w = 1;
  * preconditioner scalars use J ~ I: m1 = rho (1 + 1/delta),
    m2 = psi^2 / (rho (gamma + psi^2/delta)) + delta/rho;
  * matching Schur approximation (Eq. (second schur complement preconditioner)) with
    the circulant approximations D-tilde = C_3(B), J1-tilde = J2-tilde = I (Algorithm 1)
    or the exact scalars (Algorithm 2); it is FFT-diagonal like S-tilde;
  * generalized ADMM (Algorithm 2): both proximal terms carry the factor 1/2
    (the coefficient matrix printed for R_y = c_y I - J1, R_u = c_u I - J2
    needs it on the u term too); R_y, R_u positive semi-definite is accepted
    (c_y >= max w, c_u >= gamma max w), R = 0 being Algorithm 1; the psi-scaled
    u block is rho (c_u + psi^2/delta); its preconditioner scalars are exact;
  * DFT convention lambda_k = sum_j c_j exp(-2 pi i j k / n) (unnormalised).

Parity status: every function below is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_pins.py``; nothing here is parity-unpinned.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

# --------------------------------------------------------------------------
# Discretisation (Section 4)
# --------------------------------------------------------------------------


def gl_weights(order: float, count: int) -> np.ndarray:
    """Gruenwald-Letnikov weights g_0..g_{count-1} by the recurrence of Eq. (C_GL):
    g_0 = 1, g_k = (1 - (order+1)/k) g_{k-1}."""
    g = np.zeros(count)
    if count == 0:
        return g
    g[0] = 1.0
    for k in range(1, count):
        g[k] = (1.0 - (order + 1.0) / k) * g[k - 1]
    return g


def mesh(p):
    """(h_x, h_y, h_t): interior spacing 1/(n+1) in space (Section 6.1);
    h_t = T/nt, or h_t = h_x when time_step_mode == 1."""
    hx = 1.0 / (p.nx + 1)
    hy = 1.0 / (p.ny + 1)
    ht = p.T / p.nt if p.time_step_mode == 0 else hx
    return hx, hy, ht


def psi_scale(p) -> float:
    """psi = min{h_t^alpha, h_x^beta1, h_y^beta2} (Section 5, scaling before Eq.
    (multilevel circulant preconditioner))."""
    hx, hy, ht = mesh(p)
    return min(ht ** p.alpha_t, hx ** p.beta_x, hy ** p.beta_y)


def caputo_matrix(p) -> np.ndarray:
    """Eq. (Caputo matrix): lower-triangular Toeplitz, entry (i, j) = g_{i-j}/h_t^alpha."""
    _, _, ht = mesh(p)
    g = gl_weights(p.alpha_t, p.nt)
    C = np.zeros((p.nt, p.nt))
    for i in range(p.nt):
        for j in range(i + 1):
            C[i, j] = g[i - j]
    return C / ht ** p.alpha_t


def shifted_gl_matrix(beta: float, n: int, h: float) -> np.ndarray:
    """Shifted GL matrix of Eq. (RL_GL) with shift 1: entry (i, j) = g_{i-j+1}/h^beta
    for 0 <= i-j+1 <= n, zero otherwise (one super-diagonal)."""
    g = gl_weights(beta, n + 1)
    L = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            k = i - j + 1
            if 0 <= k <= n:
                L[i, j] = g[k]
    return L / h ** beta


def space_matrices(p):
    """X = d+ L_x + d- L_x^T (x1 axis) and Y = e+ L_y + e- L_y^T (x2 axis):
    the two-sided generalisation of Eq. (Riesz matrix)."""
    hx, hy, _ = mesh(p)
    Lx = shifted_gl_matrix(p.beta_x, p.nx, hx)
    Ly = shifted_gl_matrix(p.beta_y, p.ny, hy)
    X = p.dp * Lx + p.dm * Lx.T
    Y = p.ep * Ly + p.em * Ly.T
    return X, Y


def assemble_B_sparse(p) -> sp.csr_matrix:
    """B = psi D with D = C_t (x) I - I (x) (X (x) I + I (x) Y) (Eq. (FDE constraint
    matrix), scaled as in Section 5), assembled with Kronecker products."""
    C = caputo_matrix(p)
    X, Y = space_matrices(p)
    It, Ix, Iy = sp.identity(p.nt), sp.identity(p.nx), sp.identity(p.ny)
    D = (sp.kron(sp.csr_matrix(C), sp.kron(Ix, Iy))
         - sp.kron(It, sp.kron(sp.csr_matrix(X), Iy))
         - sp.kron(It, sp.kron(Ix, sp.csr_matrix(Y))))
    return (psi_scale(p) * D).tocsr()


def assemble_B(p) -> np.ndarray:
    """Dense B (tiny grids only)."""
    return assemble_B_sparse(p).toarray()


def objective_weights(p) -> np.ndarray:
    """Diagonal of J1 (Eq. (discretized Objective function)): ones, with 1/2 on the
    last time slice for the trapezoid rule; all ones when weights == 1."""
    w = np.ones((p.nt, p.nx, p.ny))
    if p.weights == 0:
        w[-1] = 0.5
    return w


# --------------------------------------------------------------------------
# Structured (per-axis) operator application: Tier-S
# --------------------------------------------------------------------------


def along_t(M: np.ndarray, x: np.ndarray) -> np.ndarray:
    """out[k, i, j] = sum_l M[k, l] x[l, i, j] (matrix acting on the time axis)."""
    nt, nx, ny = x.shape
    return (M @ x.reshape(nt, nx * ny)).reshape(M.shape[0], nx, ny)


def along_x1(M: np.ndarray, x: np.ndarray) -> np.ndarray:
    """out[k, i, j] = sum_l M[i, l] x[k, l, j] (matrix acting on the x1 axis)."""
    return np.matmul(M, x)


def along_x2(M: np.ndarray, x: np.ndarray) -> np.ndarray:
    """out[k, i, j] = sum_l M[j, l] x[k, i, l] (matrix acting on the x2 axis)."""
    return np.matmul(x, M.T)


def apply_B(p, x: np.ndarray, transpose: bool = False) -> np.ndarray:
    """B x (or B^T x) applied axis by axis: the Kronecker sum of Eq. (FDE constraint
    matrix) means the time matrix acts on axis 0, X on axis 1 and Y on axis 2."""
    C = caputo_matrix(p)
    X, Y = space_matrices(p)
    if transpose:
        C, X, Y = C.T, X.T, Y.T
    x = x.reshape(p.nt, p.nx, p.ny)
    return psi_scale(p) * (along_t(C, x) - along_x1(X, x) - along_x2(Y, x))


def apply_B_at(p, x: np.ndarray, points, transpose: bool = False) -> np.ndarray:
    """Entries (k, i, j) of B x for a list of points, one at a time from the rows of
    the three 1-D matrices (for sampled checks on grids too large for apply_B)."""
    C = caputo_matrix(p)
    X, Y = space_matrices(p)
    if transpose:
        C, X, Y = C.T, X.T, Y.T
    x = x.reshape(p.nt, p.nx, p.ny)
    psi = psi_scale(p)
    out = []
    for (k, i, j) in points:
        v = C[k] @ x[:, i, j] - X[i] @ x[k, :, j] - Y[j] @ x[k, i, :]
        out.append(psi * v)
    return np.array(out)


# --------------------------------------------------------------------------
# ADMM diagonals and the normal equations (Section 3.1, Eq. (generic ADMM normal
# equations)) with the psi scaling of Section 6.1
# --------------------------------------------------------------------------


@dataclasses.dataclass
class AdmmOptions:
    """delta: penalty parameter (penalty 1/delta); rho: dual step length in
    (0, (1+sqrt 5)/2) (Algorithm 1) or (0, 1] (Algorithm 2); tol: infinity-norm
    tolerance on the three residuals. algorithm 2: generalized ADMM with the
    proximal matrices R_y = c_y I - J1 and R_u = c_u I - J2 (Section 3.3.2)."""
    delta: float = 1.0
    rho: float = 1.618
    tol: float = 1e-6
    max_iter: int = 1000
    algorithm: int = 1
    c_y: float = 0.0
    c_u: float = 0.0
    precond: int = 0        # 0: S-tilde (first Schur complement approximation), 1: S-hat (matching)


def check_generalized(p, o: AdmmOptions):
    """Algorithm 2 needs rho in (0, 1] and R_y, R_u positive semi-definite."""
    w = objective_weights(p)
    if not (0.0 < o.rho <= 1.0):
        raise ValueError("generalized ADMM needs rho in (0, 1]")
    if o.c_y < np.max(w) or o.c_u < p.gamma * np.max(w):
        raise ValueError("c_y >= max J1 and c_u >= max J2 are required")


def admm_diagonals(p, o: AdmmOptions):
    """M1 = rho (J1 + I/delta), Q = rho (J2 + psi^2 I/delta), M2 = psi^2 Q^-1 + (delta/rho) I.
    Algorithm 2: J1 + R_y = c_y I and J2 + R_u = c_u I replace J1 and J2
    (Eq. (generic generalized ADMM subproblems 1and3 optimality operator)), so all
    three are multiples of the identity."""
    w = objective_weights(p)
    psi = psi_scale(p)
    if o.algorithm == 2:
        check_generalized(p, o)
        one = np.ones_like(w)
        M1 = o.rho * (o.c_y + 1.0 / o.delta) * one
        Q = o.rho * (o.c_u + psi * psi / o.delta) * one
    else:
        M1 = o.rho * (w + 1.0 / o.delta)
        Q = o.rho * (p.gamma * w + psi * psi / o.delta)
    M2 = psi * psi / Q + o.delta / o.rho
    return M1, Q, M2


def apply_S(p, o: AdmmOptions, v: np.ndarray) -> np.ndarray:
    """S v = M1 v + B^T (M2^-1 (B v)) (Eq. (generic ADMM normal equations))."""
    M1, _, M2 = admm_diagonals(p, o)
    v = v.reshape(p.nt, p.nx, p.ny)
    return M1 * v + apply_B(p, apply_B(p, v) / M2, transpose=True)


def assemble_S(p, o: AdmmOptions) -> np.ndarray:
    """Dense S = M1 + B^T M2^-1 B."""
    B = assemble_B_sparse(p)
    M1, _, M2 = admm_diagonals(p, o)
    S = (B.T @ sp.diags(1.0 / M2.ravel()) @ B).toarray()
    S[np.diag_indices_from(S)] += M1.ravel()
    return S


# --------------------------------------------------------------------------
# T. Chan circulant preconditioner (Section 5, Eq. (level 1 circulant
# optimization problem), Eq. (multilevel circulant preconditioner)) and the
# Schur approximation of Eq. (first schur complement preconditioner)
# --------------------------------------------------------------------------


def tchan_column(T: np.ndarray) -> np.ndarray:
    """First column of the T. Chan circulant of a Toeplitz matrix T:
    c_i = ((n - i) t_i + i t_{i-n}) / n, with t_k = T[k, 0] and t_{-k} = T[0, k]."""
    n = T.shape[0]
    c = np.zeros(n)
    for i in range(n):
        t_i = T[i, 0]
        t_im = T[0, n - i] if i > 0 else 0.0
        c[i] = ((n - i) * t_i + i * t_im) / n
    return c


def circulant(c: np.ndarray) -> np.ndarray:
    """Dense circulant matrix with first column c: entry (i, j) = c[(i - j) mod n]."""
    n = len(c)
    return np.array([[c[(i - j) % n] for j in range(n)] for i in range(n)])


def dft_matrix(n: int) -> np.ndarray:
    """F[k, j] = exp(-2 pi i j k / n) (unnormalised DFT)."""
    k = np.arange(n)
    return np.exp(-2j * np.pi * np.outer(k, k) / n)


def circulant_eigenvalues(c: np.ndarray) -> np.ndarray:
    """Eigenvalues of circulant(c) in DFT order: Lambda = F c (Section 2, Theorem on
    circulant matrices)."""
    return dft_matrix(len(c)) @ c


def preconditioner_axis_eigenvalues(p):
    """(lambda_t, lambda_x, lambda_y): eigenvalues of the T. Chan circulants of
    C_t, X and Y."""
    C = caputo_matrix(p)
    X, Y = space_matrices(p)
    return (circulant_eigenvalues(tchan_column(C)),
            circulant_eigenvalues(tchan_column(X)),
            circulant_eigenvalues(tchan_column(Y)))


def preconditioner_scalars(p, o: AdmmOptions):
    """m1, m2: the scalar (J ~ I) versions of M1 and M2 used in S-tilde; for
    Algorithm 2, M1 and M2 themselves (already scalar)."""
    psi = psi_scale(p)
    if o.algorithm == 2:
        M1, _, M2 = admm_diagonals(p, o)
        return float(M1.flat[0]), float(M2.flat[0])
    m1 = o.rho * (1.0 + 1.0 / o.delta)
    m2 = psi * psi / (o.rho * (p.gamma + psi * psi / o.delta)) + o.delta / o.rho
    return m1, m2


def preconditioner_symbol(p, o: AdmmOptions) -> np.ndarray:
    """sigma[k, i, j] = m1 + |Lambda|^2 / m2 with Lambda = psi (lambda_t[k] - lambda_x[i]
    - lambda_y[j]), the eigenvalues of C_3(B) (Kronecker sum after Eq. (multilevel
    circulant preconditioner)).
    Matching variant (o.precond = 1, Eq. (second schur complement preconditioner)) with
    the circulant D-tilde = C_3(B) and scalar M1, M2: D-hat = C_3^T + sqrt(m1 m2) I is
    circulant too, so S-hat = D-hat D-hat^T / m2 has the eigenvalues
    |conj(Lambda) + sqrt(m1 m2)|^2 / m2 = m1 + |Lambda|^2 / m2 + 2 sqrt(m1/m2) Re(Lambda)."""
    lt, lx, ly = preconditioner_axis_eigenvalues(p)
    psi = psi_scale(p)
    Lam = psi * (lt[:, None, None] - lx[None, :, None] - ly[None, None, :])
    m1, m2 = preconditioner_scalars(p, o)
    sigma = m1 + np.abs(Lam) ** 2 / m2
    if o.precond == 1:
        sigma = sigma + 2.0 * math.sqrt(m1 / m2) * Lam.real
    return sigma


def apply_preconditioner(p, o: AdmmOptions, r: np.ndarray) -> np.ndarray:
    """z = S-tilde^-1 r = F^-1 diag(1/sigma) F r with F the 3-level DFT, applied as
    a dense DFT matrix along each axis."""
    r = r.reshape(p.nt, p.nx, p.ny).astype(complex)
    Ft, Fx, Fy = dft_matrix(p.nt), dft_matrix(p.nx), dft_matrix(p.ny)
    R = along_x2(Fy, along_x1(Fx, along_t(Ft, r)))
    Z = R / preconditioner_symbol(p, o)
    Z = along_x2(Fy.conj(), along_x1(Fx.conj(), along_t(Ft.conj(), Z))) / p.N
    return Z.real


def dense_matching_preconditioner(p, o: AdmmOptions) -> np.ndarray:
    """Dense S-hat = D-hat M2^-1 D-hat^T, D-hat = C_3^T + (m1 m2)^(1/2) I (Eq. (second
    schur complement preconditioner) with D-tilde = C_3 and the scalar M1, M2)."""
    C = caputo_matrix(p)
    X, Y = space_matrices(p)
    Ct, Cx, Cy = (circulant(tchan_column(M)) for M in (C, X, Y))
    It, Ix, Iy = np.eye(p.nt), np.eye(p.nx), np.eye(p.ny)
    C3 = psi_scale(p) * (np.kron(Ct, np.kron(Ix, Iy)) - np.kron(It, np.kron(Cx, Iy))
                         - np.kron(It, np.kron(Ix, Cy)))
    m1, m2 = preconditioner_scalars(p, o)
    Dh = C3.T + math.sqrt(m1 * m2) * np.eye(p.N)
    return Dh @ Dh.T / m2


def dense_preconditioner(p, o: AdmmOptions) -> np.ndarray:
    """Dense S-tilde = m1 I + C_3^T C_3 / m2 with C_3 assembled from dense T. Chan
    circulants (tiny grids)."""
    C = caputo_matrix(p)
    X, Y = space_matrices(p)
    Ct, Cx, Cy = (circulant(tchan_column(M)) for M in (C, X, Y))
    It, Ix, Iy = np.eye(p.nt), np.eye(p.nx), np.eye(p.ny)
    C3 = psi_scale(p) * (np.kron(Ct, np.kron(Ix, Iy)) - np.kron(It, np.kron(Cx, Iy))
                         - np.kron(It, np.kron(Ix, Cy)))
    m1, m2 = preconditioner_scalars(p, o)
    return m1 * np.eye(p.N) + C3.T @ C3 / m2


# --------------------------------------------------------------------------
# ADMM, Algorithm 1 with the sub-problem merged with the p-update
# --------------------------------------------------------------------------


@dataclasses.dataclass
class AdmmState:
    y: np.ndarray
    u: np.ndarray
    zy: np.ndarray
    zu: np.ndarray
    p: np.ndarray
    wy: np.ndarray
    wu: np.ndarray
    iters: int = 0
    residuals: tuple = (np.inf, np.inf, np.inf)
    pcg_iters: list = dataclasses.field(default_factory=list)


def zero_state(p) -> AdmmState:
    z = lambda: np.zeros((p.nt, p.nx, p.ny))
    return AdmmState(z(), z(), z(), z(), z(), z(), z())


def box_bounds(p, lo, hi):
    shape = (p.nt, p.nx, p.ny)
    lo = np.full(shape, -np.inf) if lo is None else np.broadcast_to(np.asarray(lo, float), shape)
    hi = np.full(shape, np.inf) if hi is None else np.broadcast_to(np.asarray(hi, float), shape)
    return lo, hi


def admm_block_rhs(p, o, ybar, g, st: AdmmState):
    """Right-hand sides of the three block rows of the merged system (the psi-scaled
    form of Eq. (generic ADMM subproblems 1and3 optimality conditions)):
    b_y = rho (J1 ybar - w_y + z_y/delta) + (1-rho) B^T p,
    b_u = rho (-psi w_u + psi^2 z_u/delta) + (1-rho) psi p,
    f_p = psi g - (delta/rho) p.
    Algorithm 2 adds the proximal pulls rho R_y y^j to b_y and rho R_u u^j to b_u."""
    psi = psi_scale(p)
    w = objective_weights(p)
    by = o.rho * (w * ybar - st.wy + st.zy / o.delta) + (1.0 - o.rho) * apply_B(p, st.p, True)
    bu = o.rho * (-psi * st.wu + psi * psi * st.zu / o.delta) + (1.0 - o.rho) * psi * st.p
    if o.algorithm == 2:
        by = by + o.rho * (o.c_y - w) * st.y
        bu = bu + o.rho * (o.c_u - p.gamma * w) * st.u
    fp = psi * g - (o.delta / o.rho) * st.p
    return by, bu, fp


def admm_rhs(p, o, ybar, g, st: AdmmState):
    """Pivoting the u and p rows of the merged system (Section 3.1):
    r0  = psi Q^-1 b_u - psi g + (delta/rho) p,
    rhs = b_y - B^T (M2^-1 r0)   (right-hand side of S y = rhs)."""
    psi = psi_scale(p)
    _, Q, M2 = admm_diagonals(p, o)
    by, bu, _ = admm_block_rhs(p, o, ybar, g, st)
    r0 = psi * bu / Q - psi * g + (o.delta / o.rho) * st.p
    rhs = by - apply_B(p, r0 / M2, True)
    return rhs, bu, r0


def admm_after_solve(p, o, g, lo_y, hi_y, lo_u, hi_u, st: AdmmState, y, bu, r0):
    """Pivots and the remaining steps of Algorithm 1 given the sub-problem solution y:
    p = M2^-1 (B y + r0), u = Q^-1 (b_u - psi p); z-step = projection onto the box
    of y + delta w_y and u + delta w_u / psi; multiplier steps with rho/delta."""
    psi = psi_scale(p)
    _, Q, M2 = admm_diagonals(p, o)
    By = apply_B(p, y)
    pn = (By + r0) / M2
    u = (bu - psi * pn) / Q
    zy = np.clip(y + o.delta * st.wy, lo_y, hi_y)
    zu = np.clip(u + o.delta * st.wu / psi, lo_u, hi_u)
    wy = st.wy + (o.rho / o.delta) * (y - zy)
    wu = st.wu + (o.rho / o.delta) * psi * (u - zu)
    res = (np.max(np.abs(By + psi * (u - g))), np.max(np.abs(y - zy)), np.max(np.abs(u - zu)))
    return AdmmState(y, u, zy, zu, pn, wy, wu, st.iters + 1, res, st.pcg_iters)


def factor_S(p, o: AdmmOptions):
    """Cholesky factor of S (lower), kept in Fortran order so that every solve
    reads it in place."""
    c, lower = sla.cho_factor(np.asfortranarray(assemble_S(p, o)), lower=True, overwrite_a=True,
                              check_finite=False)
    return np.asfortranarray(c), lower


def admm_direct(inst, o: AdmmOptions, iters: Optional[int] = None, state: Optional[AdmmState] = None,
                factor=None) -> AdmmState:
    """Algorithm 1 with each sub-problem solved exactly: S is factored once by
    Cholesky (the sub-problem matrix never changes) and every iteration does two
    triangular solves. Runs ``iters`` iterations if given, else until the three
    infinity-norm residuals of Section 6.1 are <= o.tol."""
    p = inst.params
    g = np.zeros((p.nt, p.nx, p.ny)) if inst.g is None else inst.g
    lo_y, hi_y = box_bounds(p, inst.ya, inst.yb)
    lo_u, hi_u = box_bounds(p, inst.ua, inst.ub)
    st = zero_state(p) if state is None else state
    cho = factor if factor is not None else factor_S(p, o)
    n = iters if iters is not None else o.max_iter
    for _ in range(n):
        rhs, bu, r0 = admm_rhs(p, o, inst.ybar, g, st)
        y = sla.cho_solve(cho, rhs.ravel(), check_finite=False).reshape(rhs.shape)
        st = admm_after_solve(p, o, g, lo_y, hi_y, lo_u, hi_u, st, y, bu, r0)
        if iters is None and max(st.residuals) <= o.tol:
            break
    return st


def pcg(apply_A, apply_M, b, x0, tol, max_iter):
    """Preconditioned conjugate gradients (Hestenes-Stiefel form). Stops when
    ||b - A x||_2 <= tol ||b||_2 (the recursive residual). Returns (x, iterations)."""
    x = x0.copy()
    r = b - apply_A(x)
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return np.zeros_like(b), 0
    if np.linalg.norm(r) <= tol * bn:
        return x, 0
    z = apply_M(r)
    d = z.copy()
    rz = np.vdot(r, z).real
    for it in range(1, max_iter + 1):
        q = apply_A(d)
        a = rz / np.vdot(d, q).real
        x += a * d
        r -= a * q
        if np.linalg.norm(r) <= tol * bn:
            return x, it
        z = apply_M(r)
        rz_new = np.vdot(r, z).real
        d = z + (rz_new / rz) * d
        rz = rz_new
    return x, max_iter


def admm_pcg(inst, o: AdmmOptions, iters: Optional[int] = None, inner_tol: float = 1e-10,
             max_pcg: int = 500, paper_inner_rule: bool = False, x0_zero: bool = False) -> AdmmState:
    """Algorithm 1 with each sub-problem solved by PCG preconditioned with S-tilde
    (Section 6.1), warm-started from the previous y (x0_zero: from zero, the default
    initial guess of MATLAB's pcg). With paper_inner_rule the PCG tolerance is
    0.05 max{min{residuals}, tol} (Section 6.1); else inner_tol."""
    p = inst.params
    g = np.zeros((p.nt, p.nx, p.ny)) if inst.g is None else inst.g
    lo_y, hi_y = box_bounds(p, inst.ya, inst.yb)
    lo_u, hi_u = box_bounds(p, inst.ua, inst.ub)
    st = zero_state(p)
    A = lambda v: apply_S(p, o, v)
    M = lambda r: apply_preconditioner(p, o, r)
    n = iters if iters is not None else o.max_iter
    for _ in range(n):
        rhs, bu, r0 = admm_rhs(p, o, inst.ybar, g, st)
        if paper_inner_rule:
            tol = 0.05 * max(min(st.residuals), o.tol) if st.iters > 0 else 0.05
        else:
            tol = inner_tol
        y, k = pcg(A, M, rhs, np.zeros_like(st.y) if x0_zero else st.y, tol, max_pcg)
        pcg_hist = st.pcg_iters + [k]
        st = admm_after_solve(p, o, g, lo_y, hi_y, lo_u, hi_u, st, y, bu, r0)
        st.pcg_iters = pcg_hist
        if iters is None and max(st.residuals) <= o.tol:
            break
    return st


# --------------------------------------------------------------------------
# Saddle-point sub-problem solved by MINRES with the block-diagonal
# preconditioner K-tilde (Section 3.3.1, Eq. (generic block-diagonal
# preconditioner)). Vectors of the 3N system are arrays (3, nt, nx, ny):
# blocks y, u, p.
# --------------------------------------------------------------------------


def apply_K(p, o: AdmmOptions, x: np.ndarray) -> np.ndarray:
    """K [y; u; p] with the psi-scaled coefficient matrix of Eq. (generic ADMM
    subproblems 1and3 optimality conditions):
    [[M1, 0, B^T], [0, Q, psi I], [B, psi I, -(delta/rho) I]]."""
    M1, Q, _ = admm_diagonals(p, o)
    psi = psi_scale(p)
    y, u, q = (x[k].reshape(p.nt, p.nx, p.ny) for k in range(3))
    return np.stack([M1 * y + apply_B(p, q, transpose=True),
                     Q * u + psi * q,
                     apply_B(p, y) + psi * u - (o.delta / o.rho) * q])


def assemble_K(p, o: AdmmOptions) -> np.ndarray:
    """Dense K (tiny grids)."""
    M1, Q, _ = admm_diagonals(p, o)
    B = assemble_B(p)
    N, psi = p.N, psi_scale(p)
    Z = np.zeros((N, N))
    return np.block([[np.diag(M1.ravel()), Z, B.T],
                     [Z, np.diag(Q.ravel()), psi * np.eye(N)],
                     [B, psi * np.eye(N), -(o.delta / o.rho) * np.eye(N)]])


def schur_p_symbol(p, o: AdmmOptions) -> np.ndarray:
    """Eigenvalues of Sigma-tilde = m2 I + C_3 C_3^T / m1, the circulant stand-in for
    the Schur complement (delta/rho) I + B M1^-1 B^T + psi^2 Q^-1 = M2 + B M1^-1 B^T
    of the p block (m1, m2 as in S-tilde): m2 + |Lambda|^2 / m1."""
    lt, lx, ly = preconditioner_axis_eigenvalues(p)
    psi = psi_scale(p)
    Lam = psi * (lt[:, None, None] - lx[None, :, None] - ly[None, None, :])
    m1, m2 = preconditioner_scalars(p, o)
    return m2 + np.abs(Lam) ** 2 / m1


def apply_block_preconditioner(p, o: AdmmOptions, r: np.ndarray) -> np.ndarray:
    """K-tilde^-1 r with K-tilde = blkdiag(M1, Q, Sigma-tilde): J1 and J2 are
    diagonal, so their blocks are used exactly; Sigma-tilde^-1 by the 3-level DFT."""
    M1, Q, _ = admm_diagonals(p, o)
    ry, ru, rq = (r[k].reshape(p.nt, p.nx, p.ny) for k in range(3))
    Ft, Fx, Fy = dft_matrix(p.nt), dft_matrix(p.nx), dft_matrix(p.ny)
    R = along_x2(Fy, along_x1(Fx, along_t(Ft, rq.astype(complex))))
    Z = along_x2(Fy.conj(), along_x1(Fx.conj(), along_t(Ft.conj(), R / schur_p_symbol(p, o)))) / p.N
    return np.stack([ry / M1, ru / Q, Z.real])


def dense_block_preconditioner(p, o: AdmmOptions) -> np.ndarray:
    """Dense K-tilde with Sigma-tilde assembled from dense T. Chan circulants."""
    M1, Q, _ = admm_diagonals(p, o)
    C = caputo_matrix(p)
    X, Y = space_matrices(p)
    Ct, Cx, Cy = (circulant(tchan_column(M)) for M in (C, X, Y))
    It, Ix, Iy = np.eye(p.nt), np.eye(p.nx), np.eye(p.ny)
    C3 = psi_scale(p) * (np.kron(Ct, np.kron(Ix, Iy)) - np.kron(It, np.kron(Cx, Iy))
                         - np.kron(It, np.kron(Ix, Cy)))
    m1, m2 = preconditioner_scalars(p, o)
    N = p.N
    Z = np.zeros((N, N))
    Sig = m2 * np.eye(N) + C3 @ C3.T / m1
    return np.block([[np.diag(M1.ravel()), Z, Z], [Z, np.diag(Q.ravel()), Z], [Z, Z, Sig]])


def minres(apply_A, apply_M, b, x0, tol, max_iter):
    """Preconditioned MINRES (Paige and Saunders) for symmetric A and symmetric
    positive definite M: the Lanczos process in the M^-1 inner product builds a
    tridiagonal T_k, whose QR factorisation by Givens rotations updates x so that
    ||b - A x||_{M^-1} is minimal over x0 + K_k(M^-1 A, M^-1 r0). The rotations
    also give that norm, |eta|, at no cost. Stops when |eta| <= tol ||b||_{M^-1}.
    Returns (x, iterations, |eta| / ||b||_{M^-1})."""
    x = x0.copy()
    bn = math.sqrt(max(float(np.vdot(b, apply_M(b)).real), 0.0))
    if bn == 0.0:
        return np.zeros_like(b), 0, 0.0
    v = b - apply_A(x)                      # v_1 (the Lanczos vectors are v_k / beta_k)
    z = apply_M(v)
    beta = math.sqrt(max(float(np.vdot(v, z).real), 0.0))
    eta = beta
    if eta <= tol * bn:
        return x, 0, eta / bn
    v_prev = np.zeros_like(b)
    beta_prev = 1.0
    w_prev = np.zeros_like(b)
    w = np.zeros_like(b)
    c_prev, c = 1.0, 1.0                    # the two previous rotations
    s_prev, s = 0.0, 0.0
    for k in range(1, max_iter + 1):
        z = z / beta
        q = apply_A(z)
        alpha = float(np.vdot(q, z).real)
        v_next = q - (alpha / beta) * v - (beta / beta_prev) * v_prev
        z_next = apply_M(v_next)
        beta_next = math.sqrt(max(float(np.vdot(v_next, z_next).real), 0.0))
        # column k of T_k: beta_k above the diagonal, alpha_k on it, beta_{k+1} below;
        # the rotations k-2 and k-1 act on it, a new rotation removes beta_{k+1}
        e3 = s_prev * beta
        e2 = s * alpha + c_prev * c * beta
        e0 = c * alpha - c_prev * s * beta
        e1 = math.hypot(e0, beta_next)
        c_new, s_new = e0 / e1, beta_next / e1
        w_next = (z - e3 * w_prev - e2 * w) / e1
        x += c_new * eta * w_next
        eta = -s_new * eta
        if abs(eta) <= tol * bn:
            return x, k, abs(eta) / bn
        v_prev, v = v, v_next
        beta_prev, beta = beta, beta_next
        w_prev, w = w, w_next
        z = z_next
        c_prev, c = c, c_new
        s_prev, s = s, s_new
        if beta == 0.0:                     # invariant subspace: x is exact
            return x, k, abs(eta) / bn
    return x, max_iter, abs(eta) / bn


def admm_after_saddle(p, o, g, lo_y, hi_y, lo_u, hi_u, st: AdmmState, y, u, pn):
    """Remaining steps of Algorithm 1 (or 2) given the sub-problem solution (y, u, p)
    of the saddle-point system: projections and multiplier steps as in admm_after_solve."""
    psi = psi_scale(p)
    By = apply_B(p, y)
    zy = np.clip(y + o.delta * st.wy, lo_y, hi_y)
    zu = np.clip(u + o.delta * st.wu / psi, lo_u, hi_u)
    wy = st.wy + (o.rho / o.delta) * (y - zy)
    wu = st.wu + (o.rho / o.delta) * psi * (u - zu)
    res = (np.max(np.abs(By + psi * (u - g))), np.max(np.abs(y - zy)), np.max(np.abs(u - zu)))
    return AdmmState(y, u, zy, zu, pn, wy, wu, st.iters + 1, res, st.pcg_iters)


def admm_minres(inst, o: AdmmOptions, iters: Optional[int] = None, inner_tol: float = 1e-10,
                max_minres: int = 2000) -> AdmmState:
    """Algorithm 1 (or 2) whose joint (y, u, p) step is the saddle-point system of
    Eq. (generic ADMM subproblems 1and3 optimality conditions) solved by MINRES with
    K-tilde (Section 3.3.1), warm-started from the previous (y, u, p)."""
    p = inst.params
    g = np.zeros((p.nt, p.nx, p.ny)) if inst.g is None else inst.g
    lo_y, hi_y = box_bounds(p, inst.ya, inst.yb)
    lo_u, hi_u = box_bounds(p, inst.ua, inst.ub)
    st = zero_state(p)
    A = lambda v: apply_K(p, o, v)
    M = lambda r: apply_block_preconditioner(p, o, r)
    n = iters if iters is not None else o.max_iter
    for _ in range(n):
        f = np.stack(admm_block_rhs(p, o, inst.ybar, g, st))
        x0 = np.stack([st.y, st.u, st.p])
        x, k, _ = minres(A, M, f, x0, inner_tol, max_minres)
        hist = st.pcg_iters + [k]
        st = admm_after_saddle(p, o, g, lo_y, hi_y, lo_u, hi_u, st, x[0], x[1], x[2])
        st.pcg_iters = hist
        if iters is None and max(st.residuals) <= o.tol:
            break
    return st


def objective(p, ybar, y, u) -> float:
    """J = 1/2 (y - ybar)^T J1 (y - ybar) + 1/2 u^T J2 u (Eq. (discretized generic
    inverse problem) with J2 = gamma J1)."""
    w = objective_weights(p)
    d = y - ybar
    return 0.5 * float(np.sum(w * d * d)) + 0.5 * p.gamma * float(np.sum(w * u * u))


# --------------------------------------------------------------------------
# Polish: exact solution on a fixed active set, and the gradient of J*
# --------------------------------------------------------------------------


@dataclasses.dataclass
class KktSolution:
    y: np.ndarray
    u: np.ndarray
    p: np.ndarray
    mu_y: np.ndarray   # box multiplier of y: J1 (y - ybar) + B^T p + mu_y = 0
    mu_u: np.ndarray   # box multiplier of psi u: J2 u + psi p + psi mu_u = 0
    J: float


def kkt_solve(inst, act_y_lo, act_y_hi, act_u_lo, act_u_hi, B=None) -> KktSolution:
    """Solve the equality-constrained QP with the given components of y and u fixed at
    their bounds (the optimality conditions of Eq. (discretized generic inverse
    problem) on an active set). With y_F, u_F the free parts, eliminating them
    gives (B_F J1_F^-1 B_F^T + psi^2 P_uF J2^-1) p = B_F ybar_F + B_A y_A
    + psi u_A - psi g, then y_F = ybar_F - J1_F^-1 (B^T p)_F, u_F = -psi J2_F^-1 p_F."""
    p = inst.params
    shape = (p.nt, p.nx, p.ny)
    N = p.N
    psi = psi_scale(p)
    w = objective_weights(p).ravel()
    g = np.zeros(N) if inst.g is None else inst.g.ravel()
    ybar = inst.ybar.ravel()
    lo_y, hi_y = (a.ravel() for a in box_bounds(p, inst.ya, inst.yb))
    lo_u, hi_u = (a.ravel() for a in box_bounds(p, inst.ua, inst.ub))
    ay = (act_y_lo | act_y_hi).ravel()
    au = (act_u_lo | act_u_hi).ravel()
    yA = np.where(act_y_lo.ravel(), lo_y, np.where(act_y_hi.ravel(), hi_y, 0.0))
    uA = np.where(act_u_lo.ravel(), lo_u, np.where(act_u_hi.ravel(), hi_u, 0.0))
    if B is None:
        B = assemble_B_sparse(p)
    B = sp.csc_matrix(B)
    fy = ~ay
    BF = B[:, np.flatnonzero(fy)]
    K = (BF @ sp.diags(1.0 / w[fy]) @ BF.T).toarray()
    K[np.diag_indices(N)] += np.where(au, 0.0, psi * psi / (p.gamma * w))
    rhs = BF @ ybar[fy] + B[:, np.flatnonzero(ay)] @ yA[ay] + psi * np.where(au, uA, 0.0) - psi * g
    try:
        pv = sla.solve(K, rhs, assume_a="pos")
    except (np.linalg.LinAlgError, sla.LinAlgError):
        # an intermediate active set of active_set_solve can make K singular
        pv = sla.lstsq(K, rhs)[0]
    BTp = B.T @ pv
    y = np.where(ay, yA, ybar - BTp / w)
    u = np.where(au, uA, -psi * pv / (p.gamma * w))
    mu_y = -(w * (y - ybar) + BTp)
    mu_u = -(p.gamma * w * u + psi * pv) / psi
    sol = KktSolution(y.reshape(shape), u.reshape(shape), pv.reshape(shape), mu_y.reshape(shape),
                      mu_u.reshape(shape), 0.0)
    sol.J = objective(p, inst.ybar, sol.y, sol.u)
    return sol


def polish(inst, st: AdmmState) -> KktSolution:
    """Active set read off the converged copies z (components sitting exactly on a
    bound, Eq. (ADMM subproblem 2) being a projection), then kkt_solve."""
    p = inst.params
    lo_y, hi_y = box_bounds(p, inst.ya, inst.yb)
    lo_u, hi_u = box_bounds(p, inst.ua, inst.ub)
    return kkt_solve(inst, st.zy == lo_y, st.zy == hi_y, st.zu == lo_u, st.zu == hi_u)


def kkt_violation(inst, sol: KktSolution) -> dict:
    """Primal feasibility, multiplier signs and complementarity at a KKT point."""
    p = inst.params
    lo_y, hi_y = box_bounds(p, inst.ya, inst.yb)
    lo_u, hi_u = box_bounds(p, inst.ua, inst.ub)
    B = assemble_B_sparse(p)
    psi = psi_scale(p)
    g = np.zeros(p.N) if inst.g is None else inst.g.ravel()
    eq = np.max(np.abs(B @ sol.y.ravel() + psi * (sol.u.ravel() - g)))
    box = max(np.max(np.maximum(lo_y - sol.y, 0)), np.max(np.maximum(sol.y - hi_y, 0)),
              np.max(np.maximum(lo_u - sol.u, 0)), np.max(np.maximum(sol.u - hi_u, 0)))
    # mu > 0 only at an upper bound, mu < 0 only at a lower bound
    sign = 0.0
    for mu, x, lo, hi in ((sol.mu_y, sol.y, lo_y, hi_y), (sol.mu_u, sol.u, lo_u, hi_u)):
        at_hi = np.isclose(x, hi)
        at_lo = np.isclose(x, lo)
        sign = max(sign, np.max(np.where(at_hi, np.maximum(-mu, 0), 0)),
                   np.max(np.where(at_lo, np.maximum(mu, 0), 0)),
                   np.max(np.where(~(at_hi | at_lo), np.abs(mu), 0)))
    return {"equality": eq, "box": box, "sign_complementarity": sign}


def objective_gradient(inst, sol: KktSolution) -> dict:
    """Gradient of the optimal value J* (envelope theorem on the Lagrangian
    J + p^T (B y + psi u - psi g)): dJ*/dybar = -J1 (y* - ybar);
    dJ*/dd+ = p*^T (dB/dd+) y* = -psi p*^T (I (x) L_x (x) I) y*, dd- with L_x^T,
    and de+/de- with L_y, L_y^T on the x2 axis."""
    p = inst.params
    hx, hy, _ = mesh(p)
    psi = psi_scale(p)
    Lx = shifted_gl_matrix(p.beta_x, p.nx, hx)
    Ly = shifted_gl_matrix(p.beta_y, p.ny, hy)
    y, pv = sol.y, sol.p
    w = objective_weights(p)
    out = {"ybar": -w * (sol.y - inst.ybar)}
    for name, M, axis in (("dp", Lx, 1), ("dm", Lx.T, 1), ("ep", Ly, 2), ("em", Ly.T, 2)):
        My = along_x1(M, y) if axis == 1 else along_x2(M, y)
        out[name] = -psi * float(np.sum(pv * My))
    return out


def dense_adjoint(inst, sol: KktSolution) -> np.ndarray:
    """p* from the adjoint equation B^T p = -J1 (y* - ybar) - mu_y (dense solve of the
    transposed operator)."""
    p = inst.params
    B = assemble_B(p)
    w = objective_weights(p)
    rhs = -(w * (sol.y - inst.ybar)) - sol.mu_y
    return np.linalg.solve(B.T, rhs.ravel()).reshape(sol.y.shape)


def l2_misfit(p, y, ybar) -> float:
    """Discrete L2 misfit sqrt(h_x h_y h_t sum w (y - ybar)^2) (Section 6.1)."""
    hx, hy, ht = mesh(p)
    w = objective_weights(p)
    return math.sqrt(hx * hy * ht * float(np.sum(w * (y - ybar) ** 2)))


def active_set_solve(inst, max_iter: int = 50) -> KktSolution:
    """Exact optimum of the box-constrained QP by a primal-dual active-set
    iteration: starting from the unconstrained solution, a component is taken as
    active at its upper (lower) bound when mu + c (x - bound) > 0 (< 0), with c
    the curvature of the objective in that variable (c_y = w, c_u = gamma w /
    psi for the psi-scaled multiplier of u), and kkt_solve is repeated until the
    active sets repeat. The KKT conditions of the result are checked by
    kkt_violation in the tests. Control bounds only (state bounds: use polish)."""
    if inst.ya is not None or inst.yb is not None:
        raise NotImplementedError("active_set_solve handles control bounds only")
    p = inst.params
    psi = psi_scale(p)
    w = objective_weights(p)
    lo_y, hi_y = box_bounds(p, inst.ya, inst.yb)
    lo_u, hi_u = box_bounds(p, inst.ua, inst.ub)
    B = assemble_B_sparse(p)
    none = np.zeros(w.shape, bool)
    sol = kkt_solve(inst, none, none, none, none, B=B)
    sets = None
    for _ in range(max_iter):
        ay_hi = sol.mu_y + w * (sol.y - hi_y) > 0
        ay_lo = sol.mu_y + w * (sol.y - lo_y) < 0
        cu = p.gamma * w / psi
        au_hi = sol.mu_u + cu * (sol.u - hi_u) > 0
        au_lo = sol.mu_u + cu * (sol.u - lo_u) < 0
        new = (ay_lo, ay_hi, au_lo, au_hi)
        if sets is not None and all(np.array_equal(a, b) for a, b in zip(new, sets)):
            return sol
        sets = new
        sol = kkt_solve(inst, ay_lo, ay_hi, au_lo, au_hi, B=B)
    return sol


def equality_constrained_solve(inst, tol: float = 1e-12, max_iter: int = 5000) -> KktSolution:
    """Exact optimum of the problem without box constraints (Eq. (discretized generic
    inverse problem) with only B y + psi u = psi g), for grids too large for the
    dense kkt_solve. Stationarity gives y = ybar - J1^-1 B^T p and
    u = -psi J2^-1 p, and the constraint then reads
    (B J1^-1 B^T + psi^2 J2^-1) p = B ybar - psi g, an SPD system solved by
    preconditioned CG (the pcg above) with the FFT-diagonal stand-in
    |Lambda|^2 + psi^2/gamma of the multilevel circulant approximation (J1 ~ I)."""
    p = inst.params
    psi = psi_scale(p)
    w = objective_weights(p)
    g = np.zeros((p.nt, p.nx, p.ny)) if inst.g is None else inst.g
    lt, lx, ly = preconditioner_axis_eigenvalues(p)
    lam = psi * (lt[:, None, None] - lx[None, :, None] - ly[None, None, :])
    sig = np.abs(lam) ** 2 + psi * psi / p.gamma
    A = lambda v: apply_B(p, apply_B(p, v, transpose=True) / w) + (psi * psi / p.gamma) * v / w
    M = lambda r: np.fft.ifftn(np.fft.fftn(r) / sig).real
    rhs = apply_B(p, inst.ybar) - psi * g
    pv, _ = pcg(A, M, rhs, np.zeros_like(rhs), tol, max_iter)
    y = inst.ybar - apply_B(p, pv, transpose=True) / w
    u = -psi * pv / (p.gamma * w)
    zero = np.zeros_like(y)
    return KktSolution(y, u, pv, zero, zero, objective(p, inst.ybar, y, u))
