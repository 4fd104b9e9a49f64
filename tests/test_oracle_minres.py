"""Pins of the oracle's saddle-point path (Section 3.3.1): MINRES, the coefficient
matrix K and the block-diagonal preconditioner K-tilde.

MINRES is pinned by its defining property, checked by brute force: after k
steps its residual has the smallest M^-1-norm over x0 + K_k(M^-1 A, M^-1 r0)
(a weighted least-squares problem over an explicit Krylov basis). K is pinned by
the dense block assembly, K-tilde by dense T. Chan circulants and a library
eigen-solver, and the whole ADMM by the exact-sub-solve iteration."""
import math

import numpy as np
import pytest

import fde_inputs as fi
import oracle as O


def _instance(nx=4, ny=3, nt=3, seed=5, **boxes):
    p = fi.FdeParams(nx=nx, ny=ny, nt=nt, T=1.0, beta_x=1.4, beta_y=1.7, alpha_t=1.0, dp=1.0, dm=0.5, ep=0.8,
                     em=0.3, gamma=1e-2)
    ybar = fi.desired_state_sine(p, seed)
    g = 0.1 * fi.random_field(seed + 1, (nt, nx, ny))
    return fi.FdeInstance(p, ybar, g, boxes.get("ya"), boxes.get("yb"), boxes.get("ua"), boxes.get("ub"), seed)


def _krylov_min_residual(A, Minv, b, x0, k):
    """min over x in x0 + span{(M^-1 A)^j M^-1 r0, j < k} of ||b - A x||_{M^-1}, by
    weighted least squares over an orthonormalised Krylov basis."""
    r0 = b - A @ x0
    V = []
    v = Minv @ r0
    for _ in range(k):
        for u in V:
            v = v - (u @ v) * u
        v = v / np.linalg.norm(v)
        V.append(v)
        v = Minv @ (A @ v)
    V = np.array(V).T
    L = np.linalg.cholesky(Minv)               # ||r||_{M^-1}^2 = |L^T r|^2
    c, *_ = np.linalg.lstsq(L.T @ (A @ V), L.T @ r0, rcond=None)
    r = r0 - A @ (V @ c)
    return math.sqrt(r @ Minv @ r)


@pytest.mark.parametrize("precond", [False, True])
def test_minres_minimises_the_residual_over_the_krylov_space(precond):
    rng = np.random.default_rng(3)
    n = 24
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(np.concatenate([rng.uniform(0.5, 3, n // 2), -rng.uniform(0.2, 2, n - n // 2)])) @ Q.T
    if precond:
        G = rng.standard_normal((n, n))
        Mm = G @ G.T + n * np.eye(n)
    else:
        Mm = np.eye(n)
    Minv = np.linalg.inv(Mm)
    b = rng.standard_normal(n)
    x0 = rng.standard_normal(n)
    bn = math.sqrt(b @ Minv @ b)
    for k in (1, 2, 5, 9):
        x, it, rel = O.minres(lambda v: A @ v, lambda r: Minv @ r, b, x0, 0.0, k)
        assert it == k
        r = b - A @ x
        true = math.sqrt(r @ Minv @ r)
        assert abs(true - rel * bn) <= 1e-10 * bn           # |eta| is the M^-1-norm of the residual
        assert abs(true - _krylov_min_residual(A, Minv, b, x0, k)) <= 1e-9 * bn
    x, it, rel = O.minres(lambda v: A @ v, lambda r: Minv @ r, b, x0, 1e-12, 200)
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-10)


def test_K_matches_dense_assembly_and_is_symmetric():
    inst = _instance()
    p = inst.params
    for o in (O.AdmmOptions(delta=0.6, rho=1.4), O.AdmmOptions(delta=0.9, rho=0.8, algorithm=2, c_y=1.3, c_u=0.05)):
        K = O.assemble_K(p, o)
        assert np.allclose(K, K.T, atol=1e-14)
        x = fi.random_field(8, (3, p.nt, p.nx, p.ny))
        assert np.allclose(O.apply_K(p, o, x).ravel(), K @ x.ravel(), rtol=1e-12, atol=1e-12)
        # indefinite: N positive and N negative eigenvalues (the p block is a Schur complement)
        ev = np.linalg.eigvalsh(K)
        assert np.sum(ev > 0) == 2 * p.N and np.sum(ev < 0) == p.N


def test_block_preconditioner_matches_dense_circulants():
    inst = _instance(nx=5, ny=4, nt=3)
    p = inst.params
    o = O.AdmmOptions(delta=0.7, rho=1.3)
    Kt = O.dense_block_preconditioner(p, o)
    assert np.allclose(Kt, Kt.T, atol=1e-12)
    assert np.linalg.eigvalsh(Kt)[0] > 0
    r = fi.random_field(4, (3, p.nt, p.nx, p.ny))
    got = O.apply_block_preconditioner(p, o, r).ravel()
    assert np.allclose(got, np.linalg.solve(Kt, r.ravel()), rtol=1e-10, atol=1e-12)
    # Sigma-tilde's spectrum is the symbol m2 + |Lambda|^2 / m1
    N = p.N
    Sig = Kt[2 * N:, 2 * N:]
    assert np.allclose(np.sort(np.linalg.eigvalsh(Sig)), np.sort(O.schur_p_symbol(p, o).ravel()), rtol=1e-10)
    # and it approximates the true p-block Schur complement M2 + B M1^-1 B^T
    M1, _, M2 = O.admm_diagonals(p, o)
    B = O.assemble_B(p)
    Sch = np.diag(M2.ravel()) + B @ np.diag(1 / M1.ravel()) @ B.T
    ev = np.linalg.eigvals(np.linalg.solve(Sig, Sch)).real
    assert 0.1 < ev.min() and ev.max() < 10


def test_saddle_minres_solves_the_merged_system():
    inst = _instance(ua=-0.3, ub=0.3)
    p = inst.params
    o = O.AdmmOptions(delta=0.8, rho=1.5)
    st = O.zero_state(p)
    for k, name in enumerate(("y", "u", "zy", "zu", "p", "wy", "wu")):
        setattr(st, name, fi.random_field(50 + k, (p.nt, p.nx, p.ny)))
    f = np.stack(O.admm_block_rhs(p, o, inst.ybar, inst.g, st))
    x, it, rel = O.minres(lambda v: O.apply_K(p, o, v), lambda r: O.apply_block_preconditioner(p, o, r), f,
                          np.zeros_like(f), 1e-13, 1000)
    assert rel <= 1e-13
    ref = np.linalg.solve(O.assemble_K(p, o), f.ravel())
    assert np.allclose(x.ravel(), ref, rtol=1e-9, atol=1e-11)
    # the y block is the normal-equation solution
    rhs, _, _ = O.admm_rhs(p, o, inst.ybar, inst.g, st)
    assert np.allclose(x[0].ravel(), np.linalg.solve(O.assemble_S(p, o), rhs.ravel()), rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("alg", [1, 2])
def test_admm_minres_matches_direct_admm(alg):
    inst = _instance(nx=5, ny=4, nt=3, ua=-0.05, ub=0.05, yb=0.3)
    o = (O.AdmmOptions(delta=0.8, rho=1.618) if alg == 1 else
         O.AdmmOptions(delta=0.8, rho=1.0, algorithm=2, c_y=1.2, c_u=0.02))
    ref = O.admm_direct(inst, o, iters=8)
    st = O.admm_minres(inst, o, iters=8, inner_tol=1e-13)
    for k in ("y", "u", "p", "zy", "zu", "wy", "wu"):
        assert np.allclose(getattr(st, k), getattr(ref, k), rtol=1e-9, atol=1e-11), k
    assert np.allclose(st.residuals, ref.residuals, rtol=1e-6, atol=1e-12)


def test_minres_iterations_flat_in_grid_size():
    """With K-tilde the MINRES count per solve stays bounded as the grid is refined
    (the preconditioned spectrum lies in intervals independent of n)."""
    counts = []
    for n in (4, 8, 16):
        inst = _instance(nx=n, ny=n, nt=4)
        p = inst.params
        o = O.AdmmOptions(delta=1.0, rho=1.618)
        st = O.zero_state(p)
        f = np.stack(O.admm_block_rhs(p, o, inst.ybar, inst.g, st))
        _, it, _ = O.minres(lambda v: O.apply_K(p, o, v), lambda r: O.apply_block_preconditioner(p, o, r), f,
                            np.zeros_like(f), 1e-8, 2000)
        counts.append(it)
    assert max(counts) <= 2 * min(counts) + 10, counts
