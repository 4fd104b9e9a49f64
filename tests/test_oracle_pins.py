"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed form
(Gamma-function weights, fractional power-rule derivatives), an identity of the
generating function, a library eigen-solver, brute-force minimisation, or a
direct solve of a differently arranged system. A dropped term, a wrong sign or
index, or a transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import fde_inputs as fi
import oracle as O

# --------------------------------------------------------------------------
# P1: Gruenwald-Letnikov weights (Eq. (C_GL), Proposition gamma prop)
# --------------------------------------------------------------------------


def _gamma_ratio_weight(a, k):
    """g_k = Gamma(k - a) / (Gamma(-a) Gamma(k + 1)) through log-gamma and signs."""
    if float(a).is_integer():
        return math.comb(int(a), k) * (-1) ** k if k <= a else 0.0
    s1, l1 = math.copysign(1, math.gamma(k - a)), math.lgamma(k - a)
    s2, l2 = math.copysign(1, math.gamma(-a)), math.lgamma(-a)
    return s1 * s2 * math.exp(l1 - l2 - math.lgamma(k + 1))


@pytest.mark.parametrize("a", [0.3, 0.7, 1.2, 1.5, 1.8])
def test_gl_weights_match_gamma_form(a):
    g = O.gl_weights(a, 40)
    ref = np.array([_gamma_ratio_weight(a, k) for k in range(40)])
    assert np.allclose(g, ref, rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("a,expect", [(1.0, [1, -1, 0, 0, 0]), (2.0, [1, -2, 1, 0, 0]),
                                      (0.0, [1, 0, 0, 0, 0])])
def test_gl_weights_integer_orders_are_binomial(a, expect):
    assert np.array_equal(O.gl_weights(a, 5), np.array(expect, float))


@pytest.mark.parametrize("b", [1.1, 1.3, 1.5, 1.7, 1.9])
def test_gl_weight_properties_space(b):
    g = O.gl_weights(b, 3000)
    assert g[0] == 1.0 and abs(g[1] + b) < 1e-15
    assert np.all(g[2:] > 0) and np.all(np.diff(g[2:]) < 0)
    partial = np.cumsum(g)
    assert np.all(partial[1:] < 0)
    # sum_{k<=K} g_k^(b) = g_K^(b-1): coefficients of (1-z)^b / (1-z) = (1-z)^(b-1)
    assert np.allclose(partial[:50], O.gl_weights(b - 1.0, 50), rtol=1e-12, atol=1e-15)
    assert abs(partial[-1]) < 1e-2  # sum -> 0 as K -> infinity


@pytest.mark.parametrize("a", [0.1, 0.5, 0.9])
def test_gl_weight_properties_time(a):
    g = O.gl_weights(a, 500)
    assert g[0] > 0 and np.all(g[1:] < 0)
    assert np.all(np.cumsum(g)[1:] > 0)


# --------------------------------------------------------------------------
# P7: discretisation correctness by manufactured solutions (first order in h)
# --------------------------------------------------------------------------


def _rl_left_poly(coeffs, beta, x):
    """Left Riemann-Liouville derivative on [0, x] of sum c_p x^p by the power rule
    D^beta x^p = Gamma(p+1)/Gamma(p+1-beta) x^(p-beta)."""
    return sum(c * math.gamma(pw + 1) / math.gamma(pw + 1 - beta) * x ** (pw - beta)
               for pw, c in coeffs.items())


# s(x) = x^2 (1-x)^3 vanishes at both ends; its reflection s(1-x) = x^3 (1-x)^2.
S_POLY = {2: 1.0, 3: -3.0, 4: 3.0, 5: -1.0}
S_REFL = {3: 1.0, 4: -2.0, 5: 1.0}


def _s(x):
    return x ** 2 * (1 - x) ** 3


@pytest.mark.parametrize("beta", [1.3, 1.7])
def test_shifted_gl_is_first_order_left_and_right(beta):
    errs_l, errs_r = [], []
    for n in (63, 127, 255, 511):
        h = 1.0 / (n + 1)
        x = h * np.arange(1, n + 1)
        L = O.shifted_gl_matrix(beta, n, h)
        exact_left = _rl_left_poly(S_POLY, beta, x)
        exact_right = _rl_left_poly(S_REFL, beta, 1.0 - x)  # right derivative by reflection
        # interior window away from the end-point singular layers
        m = (x > 0.25) & (x < 0.75)
        errs_l.append(np.max(np.abs(L @ _s(x) - exact_left)[m]))
        errs_r.append(np.max(np.abs(L.T @ _s(x) - exact_right)[m]))
    for errs in (errs_l, errs_r):
        ratios = np.array(errs[:-1]) / np.array(errs[1:])
        assert np.all(ratios > 1.7) and np.all(ratios < 2.4), (errs, ratios)
    # left and right differ: a transposed L would fail one of the two sequences
    assert errs_l[-1] < 0.05 * np.max(np.abs(_rl_left_poly(S_POLY, beta, 0.5) -
                                               _rl_left_poly(S_REFL, beta, 0.5)))


@pytest.mark.parametrize("alpha", [0.4, 0.8])
def test_caputo_is_first_order(alpha):
    errs = []
    for nt in (64, 128, 256, 512):
        p = fi.FdeParams(nx=1, ny=1, nt=nt, alpha_t=alpha, T=1.0)
        _, _, ht = O.mesh(p)
        t = ht * np.arange(1, nt + 1)
        exact = math.gamma(3) / math.gamma(3 - alpha) * t ** (2 - alpha)  # Caputo of t^2
        errs.append(np.max(np.abs(O.caputo_matrix(p) @ t ** 2 - exact)))
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(ratios > 1.6) and np.all(ratios < 2.4), (errs, ratios)


def test_implicit_euler_is_backward_difference():
    p = fi.FdeParams(nx=1, ny=1, nt=6, alpha_t=1.0, T=3.0)
    C = O.caputo_matrix(p)
    ref = (np.eye(6) - np.eye(6, k=-1)) / 0.5
    assert np.allclose(C, ref, rtol=0, atol=1e-15)


def test_full_operator_manufactured_solution():
    """B/psi applied to y = t^2 s(x1) s(x2) approaches the continuous operator
    d^alpha_t y - (d+ D_left + d- D_right)_x1 y - (e+ D_left + e- D_right)_x2 y."""
    errs = []
    for n in (31, 63, 127):
        p = fi.FdeParams(nx=n, ny=n, nt=n, T=1.0, beta_x=1.4, beta_y=1.8, alpha_t=0.6,
                         dp=1.0, dm=0.4, ep=0.7, em=1.3)
        x1, x2, t = fi.grid(p)
        sx1, sx2 = _s(x1), _s(x2)
        y = t[:, None, None] ** 2 * sx1[None, :, None] * sx2[None, None, :]
        dt = math.gamma(3) / math.gamma(3 - p.alpha_t) * t ** (2 - p.alpha_t)
        dx1 = p.dp * _rl_left_poly(S_POLY, p.beta_x, x1) + p.dm * _rl_left_poly(S_REFL, p.beta_x, 1 - x1)
        dx2 = p.ep * _rl_left_poly(S_POLY, p.beta_y, x2) + p.em * _rl_left_poly(S_REFL, p.beta_y, 1 - x2)
        exact = (dt[:, None, None] * sx1[None, :, None] * sx2[None, None, :]
                 - t[:, None, None] ** 2 * dx1[None, :, None] * sx2[None, None, :]
                 - t[:, None, None] ** 2 * sx1[None, :, None] * dx2[None, None, :])
        got = O.apply_B(p, y) / O.psi_scale(p)
        m = ((x1 > 0.25) & (x1 < 0.75))[None, :, None] & ((x2 > 0.25) & (x2 < 0.75))[None, None, :]
        m = m & (t > 0.3)[:, None, None]
        errs.append(np.max(np.abs(got - exact)[np.broadcast_to(m, got.shape)]))
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(ratios > 1.6), (errs, ratios)


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 3, 1), (3, 2, 4), (5, 7, 2), (4, 4, 3)])
def test_structured_apply_matches_kronecker_assembly(dims):
    nx, ny, nt = dims
    p = fi.FdeParams(nx=nx, ny=ny, nt=nt, beta_x=1.35, beta_y=1.75, alpha_t=0.7,
                     dp=1.0, dm=0.5, ep=0.8, em=0.3)
    x = fi.random_field(7, (nt, nx, ny))
    B = O.assemble_B(p)
    assert np.allclose(O.apply_B(p, x).ravel(), B @ x.ravel(), rtol=1e-13, atol=1e-13)
    assert np.allclose(O.apply_B(p, x, True).ravel(), B.T @ x.ravel(), rtol=1e-13, atol=1e-13)
    pts = [(0, 0, 0), (nt - 1, nx - 1, ny - 1), (nt // 2, nx // 2, ny // 3)]
    full = O.apply_B(p, x)
    assert np.allclose(O.apply_B_at(p, x, pts), [full[q] for q in pts], rtol=1e-13, atol=1e-13)


def test_psi_and_riesz_special_case():
    p = fi.FdeParams(nx=9, ny=9, nt=9, T=1.0, beta_x=1.3, beta_y=1.6, alpha_t=0.7, time_step_mode=1)
    h = 0.1
    assert math.isclose(O.psi_scale(p), min(h ** 0.7, h ** 1.3, h ** 1.6), rel_tol=1e-15)
    # Riesz coefficients make X symmetric (Eq. (Riesz matrix))
    c = -1.0 / (2.0 * math.cos(p.beta_x * math.pi / 2.0))
    p.dp = p.dm = c
    X, _ = O.space_matrices(p)
    assert np.allclose(X, X.T, atol=0)
    assert c > 0


# --------------------------------------------------------------------------
# P3/P4: T. Chan circulant, eigenvalues, preconditioner apply
# --------------------------------------------------------------------------


@pytest.mark.parametrize("n", [1, 2, 5, 8, 13])
def test_circulant_eigenvalues_are_dft_of_first_column(n):
    c = fi.random_field(3, (n,))
    lam = O.circulant_eigenvalues(c)
    ev = np.linalg.eigvals(O.circulant(c))
    # match as multisets
    for v in lam:
        assert np.min(np.abs(ev - v)) < 1e-10 * max(1, np.max(np.abs(ev)))
    # and the DFT convention: C = F^-1 diag(lambda) F
    F = np.exp(-2j * np.pi * np.outer(np.arange(n), np.arange(n)) / n)
    assert np.allclose(np.linalg.inv(F) @ np.diag(lam) @ F, O.circulant(c), atol=1e-12)


@pytest.mark.parametrize("n", [3, 7, 16])
def test_tchan_is_frobenius_optimal(n):
    p = fi.FdeParams(nx=n, ny=n, nt=n, beta_x=1.6, dp=1.0, dm=0.3)
    X, _ = O.space_matrices(p)
    c = O.tchan_column(X)
    best = np.linalg.norm(O.circulant(c) - X)
    # least squares over the circulant basis gives the same minimiser
    basis = np.stack([O.circulant(np.eye(n)[k]).ravel() for k in range(n)], axis=1)
    c_ls = np.linalg.lstsq(basis, X.ravel(), rcond=None)[0]
    assert np.allclose(c, c_ls, rtol=1e-12, atol=1e-12)
    rng = np.random.default_rng(0)
    for _ in range(20):
        assert np.linalg.norm(O.circulant(c + 1e-3 * rng.standard_normal(n)) - X) >= best


def test_tchan_of_implicit_euler_closed_form():
    p = fi.FdeParams(nx=1, ny=1, nt=8, alpha_t=1.0, T=1.0)
    c = O.tchan_column(O.caputo_matrix(p))
    ref = np.zeros(8)
    ref[0] = 8.0
    ref[1] = -8.0 * 7 / 8
    assert np.allclose(c, ref, atol=1e-14)


@pytest.mark.parametrize("dims", [(3, 2, 2), (4, 5, 3), (2, 2, 5)])
def test_three_level_symbol_is_spectrum_of_dense_preconditioner(dims):
    nx, ny, nt = dims
    p = fi.FdeParams(nx=nx, ny=ny, nt=nt, beta_x=1.4, beta_y=1.7, alpha_t=1.0,
                     dp=1.0, dm=0.5, ep=0.8, em=0.3, gamma=1e-3)
    o = O.AdmmOptions(delta=0.7, rho=1.3)
    St = O.dense_preconditioner(p, o)
    ev = np.sort(np.linalg.eigvalsh(St))
    sig = np.sort(O.preconditioner_symbol(p, o).ravel())
    assert np.allclose(ev, sig, rtol=1e-10)
    r = fi.random_field(11, (nt, nx, ny))
    z = O.apply_preconditioner(p, o, r)
    assert np.allclose(St @ z.ravel(), r.ravel(), rtol=1e-11, atol=1e-11)


# --------------------------------------------------------------------------
# P5/P6: normal equations
# --------------------------------------------------------------------------


def _tiny_instance(nx=4, ny=3, nt=3, ya=None, yb=None, ua=None, ub=None, seed=5, alpha=1.0):
    p = fi.FdeParams(nx=nx, ny=ny, nt=nt, T=1.0, beta_x=1.45, beta_y=1.65, alpha_t=alpha,
                     dp=1.0, dm=0.5, ep=0.8, em=0.3, gamma=1e-2)
    ybar = fi.desired_state_sine(p, seed)
    g = 0.1 * fi.random_field(seed + 1, (nt, nx, ny))
    return fi.FdeInstance(p, ybar, g, ya, yb, ua, ub, seed)


def test_normal_equations_equal_merged_saddle_system():
    inst = _tiny_instance()
    p = inst.params
    o = O.AdmmOptions(delta=0.6, rho=1.4)
    st = O.zero_state(p)
    for name in ("zy", "zu", "p", "wy", "wu"):
        setattr(st, name, fi.random_field(hash(name) % 1000, (p.nt, p.nx, p.ny)))
    rhs, bu, r0 = O.admm_rhs(p, o, inst.ybar, inst.g, st)
    y = np.linalg.solve(O.assemble_S(p, o), rhs.ravel())
    # the psi-scaled merged 3x3 block system, written out independently
    N, psi = p.N, O.psi_scale(p)
    B = O.assemble_B(p)
    w = O.objective_weights(p).ravel()
    I = np.eye(N)
    K = np.block([[o.rho * np.diag(w + 1 / o.delta), np.zeros((N, N)), B.T],
                  [np.zeros((N, N)), o.rho * np.diag(p.gamma * w + psi ** 2 / o.delta), psi * I],
                  [B, psi * I, -(o.delta / o.rho) * I]])
    f = np.concatenate([
        o.rho * (w * inst.ybar.ravel() - st.wy.ravel() + st.zy.ravel() / o.delta) + (1 - o.rho) * B.T @ st.p.ravel(),
        o.rho * (-psi * st.wu.ravel() + psi ** 2 * st.zu.ravel() / o.delta) + (1 - o.rho) * psi * st.p.ravel(),
        psi * inst.g.ravel() - (o.delta / o.rho) * st.p.ravel()])
    sol = np.linalg.solve(K, f)
    assert np.allclose(y, sol[:N], rtol=1e-10, atol=1e-12)
    _, Q, M2 = O.admm_diagonals(p, o)
    pn = (B @ y + r0.ravel()) / M2.ravel()
    u = (bu.ravel() - psi * pn) / Q.ravel()
    assert np.allclose(pn, sol[2 * N:], rtol=1e-10, atol=1e-12)
    assert np.allclose(u, sol[N:2 * N], rtol=1e-10, atol=1e-12)


def test_substep_is_minimiser_of_augmented_lagrangian():
    """(y, u) of one iteration makes the gradient of L_delta (Eq. (Generic ADMM aug
    Lagrangian), psi-scaled) vanish, and p follows Eq. (ADMM dual update 1)."""
    inst = _tiny_instance(ua=-0.3, ub=0.3, yb=0.5)
    p = inst.params
    o = O.AdmmOptions(delta=0.9, rho=1.618)
    st = O.admm_direct(inst, o, iters=3)
    st1 = O.admm_direct(inst, o, iters=1, state=st)
    psi = psi_scale = O.psi_scale(p)
    B = O.assemble_B(p)
    w = O.objective_weights(p).ravel()
    y, u = st1.y.ravel(), st1.u.ravel()
    g = inst.g.ravel()
    e = B @ y + psi * u - psi * g
    gy = w * (y - inst.ybar.ravel()) + B.T @ st.p.ravel() + st.wy.ravel() + (B.T @ e + y - st.zy.ravel()) / o.delta
    gu = p.gamma * w * u + psi * st.p.ravel() + psi * st.wu.ravel() + (psi * e + psi ** 2 * (u - st.zu.ravel())) / o.delta
    assert np.max(np.abs(gy)) < 1e-10 and np.max(np.abs(gu)) < 1e-10
    assert np.allclose(st1.p.ravel(), st.p.ravel() + (o.rho / o.delta) * e, atol=1e-11)
    # z-step: brute-force 1-D minimisation of L over each box coordinate
    grid = np.linspace(-2, 2, 40001)
    for idx in (0, 5, 17):
        a, b = y[idx], st.wy.ravel()[idx]
        vals = -b * grid + (a - grid) ** 2 / (2 * o.delta)
        vals[(grid > 0.5)] = np.inf
        assert abs(grid[np.argmin(vals)] - st1.zy.ravel()[idx]) < 2e-4
    assert psi_scale > 0


def test_S_is_spd_with_lower_bound():
    inst = _tiny_instance(nx=5, ny=4, nt=3)
    p = inst.params
    o = O.AdmmOptions(delta=2.0, rho=1.2)
    S = O.assemble_S(p, o)
    assert np.allclose(S, S.T, atol=1e-12)
    assert np.linalg.eigvalsh(S)[0] >= o.rho / o.delta - 1e-12
    v = fi.random_field(2, (p.nt, p.nx, p.ny))
    assert np.allclose(O.apply_S(p, o, v).ravel(), S @ v.ravel(), rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------------------
# P8/P9: ADMM behaviour
# --------------------------------------------------------------------------


def test_admm_with_inactive_box_equals_equality_constrained_solution():
    inst = _tiny_instance(ya=-1e3, yb=1e3, ua=-1e3, ub=1e3)
    p = inst.params
    o = O.AdmmOptions(delta=1.0, rho=1.618, tol=1e-12, max_iter=5000)
    st = O.admm_direct(inst, o)
    assert max(st.residuals) <= 1e-12
    # equality-constrained KKT written out as one dense block solve
    N, psi = p.N, O.psi_scale(p)
    B = O.assemble_B(p)
    w = O.objective_weights(p).ravel()
    K = np.block([[np.diag(w), np.zeros((N, N)), B.T],
                  [np.zeros((N, N)), np.diag(p.gamma * w), psi * np.eye(N)],
                  [B, psi * np.eye(N), np.zeros((N, N))]])
    f = np.concatenate([w * inst.ybar.ravel(), np.zeros(N), psi * inst.g.ravel()])
    sol = np.linalg.solve(K, f)
    assert np.allclose(st.y.ravel(), sol[:N], atol=1e-9)
    assert np.allclose(st.u.ravel(), sol[N:2 * N], atol=1e-9)
    assert np.allclose(st.p.ravel(), sol[2 * N:], atol=1e-9)


@pytest.mark.parametrize("boxes", [dict(ua=-0.05, ub=0.05), dict(yb=0.3), dict(ya=-0.1, yb=0.25, ua=-0.2, ub=0.1)])
def test_admm_converges_to_kkt_point(boxes):
    inst = _tiny_instance(nx=5, ny=4, nt=3, **boxes)
    o = O.AdmmOptions(delta=1.0, rho=1.618, tol=1e-9, max_iter=20000)
    st = O.admm_direct(inst, o)
    assert max(st.residuals) <= 1e-9
    lo_y, hi_y = O.box_bounds(inst.params, inst.ya, inst.yb)
    lo_u, hi_u = O.box_bounds(inst.params, inst.ua, inst.ub)
    assert np.all(st.zy >= lo_y) and np.all(st.zy <= hi_y)
    assert np.all(st.zu >= lo_u) and np.all(st.zu <= hi_u)
    sol = O.polish(inst, st)
    v = O.kkt_violation(inst, sol)
    assert v["equality"] < 1e-10 and v["box"] < 1e-12 and v["sign_complementarity"] < 1e-8, v
    assert np.allclose(st.y, sol.y, atol=1e-7) and np.allclose(st.u, sol.u, atol=1e-7)
    assert np.allclose(st.wy, sol.mu_y, atol=1e-6) and np.allclose(st.wu, sol.mu_u, atol=1e-6)
    # optimality against random feasible points (the QP is strictly convex)
    B = O.assemble_B(inst.params)
    psi = O.psi_scale(inst.params)
    rng = np.random.default_rng(1)
    for _ in range(5):
        dy = 1e-3 * rng.standard_normal(sol.y.size)
        yy = np.clip(sol.y.ravel() + dy, lo_y.ravel(), hi_y.ravel())
        uu = inst.g.ravel() - (B @ yy) / psi
        if np.all(uu >= lo_u.ravel()) and np.all(uu <= hi_u.ravel()):
            assert O.objective(inst.params, inst.ybar, yy.reshape(sol.y.shape),
                               uu.reshape(sol.y.shape)) >= sol.J - 1e-12


def test_pcg_admm_matches_direct_admm():
    inst = _tiny_instance(nx=6, ny=5, nt=4, ua=-0.2, ub=0.2)
    o = O.AdmmOptions(delta=0.8, rho=1.618)
    a = O.admm_direct(inst, o, iters=15)
    b = O.admm_pcg(inst, o, iters=15, inner_tol=1e-14)
    assert np.allclose(a.y, b.y, atol=1e-11) and np.allclose(a.p, b.p, atol=1e-11)
    assert np.allclose(a.u, b.u, atol=1e-11)


def test_pcg_iterations_flat_in_grid_size():
    """Table 5 trend: preconditioned iteration counts roughly independent of n."""
    counts = []
    for n in (8, 16, 24):
        p = fi.FdeParams(nx=n, ny=n, nt=n, T=1.0, beta_x=1.5, beta_y=1.7, alpha_t=1.0,
                         dp=1.0, dm=0.5, ep=0.8, em=0.3, gamma=1e-4)
        o = O.AdmmOptions(delta=1.0, rho=1.618)
        b = fi.random_field(n, (n, n, n))
        _, k = O.pcg(lambda v: O.apply_S(p, o, v), lambda r: O.apply_preconditioner(p, o, r),
                     b, np.zeros_like(b), 1e-8, 500)
        _, k0 = O.pcg(lambda v: O.apply_S(p, o, v), lambda r: r, b, np.zeros_like(b), 1e-8, 2000)
        counts.append(k)
        assert k < k0
    assert max(counts) <= 2 * min(counts) + 5, counts


# --------------------------------------------------------------------------
# P11: gradient of the optimal value
# --------------------------------------------------------------------------


def test_gradient_matches_central_differences_and_dense_adjoint():
    inst = _tiny_instance(nx=5, ny=4, nt=3, ua=-0.05, ub=0.05)
    p = inst.params
    o = O.AdmmOptions(delta=1.0, rho=1.618, tol=1e-10, max_iter=20000)
    st = O.admm_direct(inst, o)
    sol = O.polish(inst, st)
    act = (st.zy == -np.inf, st.zy == np.inf, st.zu == -0.05, st.zu == 0.05)
    grad = O.objective_gradient(inst, sol)
    h = 1e-6
    for name in ("dp", "dm", "ep", "em"):
        vals = []
        for s in (+1, -1):
            q = fi.FdeParams(**{**p.__dict__})
            setattr(q, name, getattr(p, name) + s * h)
            vals.append(O.kkt_solve(fi.FdeInstance(q, inst.ybar, inst.g, inst.ya, inst.yb, inst.ua, inst.ub, 0),
                                    *act).J)
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - grad[name]) <= 1e-6 * max(1.0, abs(fd)), (name, fd, grad[name])
    rng = np.random.default_rng(3)
    for flat in rng.choice(p.N, 6, replace=False):
        vals = []
        for s in (+1, -1):
            yb = inst.ybar.copy()
            yb.flat[flat] += s * h
            vals.append(O.kkt_solve(fi.FdeInstance(p, yb, inst.g, inst.ya, inst.yb, inst.ua, inst.ub, 0), *act).J)
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - grad["ybar"].flat[flat]) <= 1e-7 * max(1.0, abs(fd))
    padj = O.dense_adjoint(inst, sol)
    assert np.allclose(padj, sol.p, rtol=1e-9, atol=1e-11)


def test_input_generator_is_reproducible_and_standard_normal():
    a = fi.normal(1907, 200000)
    assert np.array_equal(a, fi.normal(1907, 200000))
    assert abs(a.mean()) < 0.01 and abs(a.std() - 1.0) < 0.01
    # splitmix64 reference values for seed 0 (published test vector)
    assert int(fi.splitmix64(0, 1)[0]) == 0xE220A8397B1DCDAF


@pytest.mark.parametrize("boxes", [dict(ua=-0.05, ub=0.05), dict(ua=-0.2, ub=0.02), dict(ua=-1e3, ub=1e3),
                                   dict(ua=0.0, ub=0.1)])
def test_active_set_solve_is_the_admm_limit(boxes):
    inst = _tiny_instance(nx=5, ny=4, nt=3, **boxes)
    sol = O.active_set_solve(inst)
    v = O.kkt_violation(inst, sol)
    assert v["equality"] < 1e-10 and v["box"] < 1e-12 and v["sign_complementarity"] < 1e-8, v
    st = O.admm_direct(inst, O.AdmmOptions(delta=1.0, rho=1.618, tol=1e-11, max_iter=50000))
    assert np.allclose(st.y, sol.y, atol=1e-8) and np.allclose(st.u, sol.u, atol=1e-8)
    assert np.allclose(st.p, sol.p, atol=1e-7)
