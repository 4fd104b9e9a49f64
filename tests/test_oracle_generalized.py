"""Pins of the oracle's generalized ADMM (Section 3.3.2, Algorithm 2) against
facts fixed elsewhere: its (y, u) step is the minimiser of the augmented
Lagrangian plus the two proximal terms, found here by a dense solve of that
quadratic's own gradient equation (not the merged normal equations); with
R_y = R_u = 0 it is Algorithm 1 step for step; and it converges to the KKT point
of the QP that the active-set polish finds."""
import numpy as np
import pytest

import fde_inputs as fi
import oracle as O


def _instance(nx=4, ny=3, nt=3, seed=5, weights=0, **boxes):
    p = fi.FdeParams(nx=nx, ny=ny, nt=nt, T=1.0, beta_x=1.4, beta_y=1.7, alpha_t=1.0, dp=1.0, dm=0.5, ep=0.8,
                     em=0.3, gamma=1e-2, weights=weights)
    ybar = fi.desired_state_sine(p, seed)
    g = 0.1 * fi.random_field(seed + 1, (nt, nx, ny))
    return fi.FdeInstance(p, ybar, g, boxes.get("ya"), boxes.get("yb"), boxes.get("ua"), boxes.get("ub"), seed)


def _random_state(p, seed):
    st = O.zero_state(p)
    for k, name in enumerate(("y", "u", "zy", "zu", "p", "wy", "wu")):
        setattr(st, name, fi.random_field(seed + 31 * k, (p.nt, p.nx, p.ny)))
    return st


@pytest.mark.parametrize("weights", [0, 1])
def test_generalized_step_minimises_lagrangian_plus_proximal_terms(weights):
    """One Algorithm 2 step from a random state against the definition: minimise
    L_delta(y, u; z^j, p^j, w^j) + 1/2 |y - y^j|^2_{R_y} + 1/2 |u - u^j|^2_{R_u}
    (psi-scaled constraints B y + psi u = psi g, y = z_y, psi u = psi z_u), then
    p^{j+1} = p^j + (rho/delta)(B y + psi u - psi g)."""
    inst = _instance(weights=weights, ua=-0.3, ub=0.3, yb=0.5)
    p = inst.params
    o = O.AdmmOptions(delta=0.7, rho=0.9, algorithm=2, c_y=1.3, c_u=0.05)
    st = _random_state(p, 11)
    st1 = O.admm_direct(inst, o, iters=1, state=st)
    N, psi = p.N, O.psi_scale(p)
    B = O.assemble_B(p)
    w = O.objective_weights(p).ravel()
    Ry = np.diag(o.c_y - w)
    Ru = np.diag(o.c_u - p.gamma * w)
    I = np.eye(N)
    # Hessian and linear term of the quadratic in (y, u)
    H = np.block([[np.diag(w) + Ry + (B.T @ B + I) / o.delta, psi * B.T / o.delta],
                  [psi * B / o.delta, np.diag(p.gamma * w) + Ru + 2 * psi ** 2 * I / o.delta]])
    g = inst.g.ravel()
    yj, uj = st.y.ravel(), st.u.ravel()
    f = np.concatenate([
        w * inst.ybar.ravel() - B.T @ st.p.ravel() - st.wy.ravel() + B.T @ (psi * g) / o.delta
        + st.zy.ravel() / o.delta + Ry @ yj,
        -psi * st.p.ravel() - psi * st.wu.ravel() + psi * psi * g / o.delta + psi ** 2 * st.zu.ravel() / o.delta
        + Ru @ uj])
    sol = np.linalg.solve(H, f)
    y, u = sol[:N], sol[N:]
    assert np.allclose(st1.y.ravel(), y, rtol=1e-9, atol=1e-11)
    assert np.allclose(st1.u.ravel(), u, rtol=1e-9, atol=1e-11)
    pn = st.p.ravel() + (o.rho / o.delta) * (B @ y + psi * u - psi * g)
    assert np.allclose(st1.p.ravel(), pn, rtol=1e-9, atol=1e-11)
    # multiplier steps of Algorithm 2 on the projected copies
    assert np.allclose(st1.wy.ravel(), st.wy.ravel() + (o.rho / o.delta) * (y - st1.zy.ravel()), atol=1e-11)


def test_zero_proximal_terms_give_algorithm_1():
    """Uniform weights, c_y = 1 and c_u = gamma make R_y = R_u = 0: every iterate
    of Algorithm 2 equals Algorithm 1's (same rho in (0, 1])."""
    inst = _instance(weights=1, ua=-0.1, ub=0.1)
    p = inst.params
    a1 = O.admm_direct(inst, O.AdmmOptions(delta=0.8, rho=1.0), iters=7)
    a2 = O.admm_direct(inst, O.AdmmOptions(delta=0.8, rho=1.0, algorithm=2, c_y=1.0, c_u=p.gamma), iters=7)
    for k in ("y", "u", "p", "zy", "zu", "wy", "wu"):
        assert np.allclose(getattr(a1, k), getattr(a2, k), rtol=1e-12, atol=1e-13), k
    # and a positive R changes the iterates (the proximal term is not dropped)
    a3 = O.admm_direct(inst, O.AdmmOptions(delta=0.8, rho=1.0, algorithm=2, c_y=2.0, c_u=p.gamma), iters=7)
    assert np.max(np.abs(a3.y - a1.y)) > 1e-6


@pytest.mark.parametrize("boxes", [dict(ua=-0.05, ub=0.05), dict(ya=-0.1, yb=0.25, ua=-0.2, ub=0.1)])
def test_generalized_admm_converges_to_kkt_point(boxes):
    inst = _instance(nx=5, ny=4, nt=3, **boxes)
    p = inst.params
    o = O.AdmmOptions(delta=1.0, rho=1.0, tol=1e-9, max_iter=40000, algorithm=2, c_y=1.2, c_u=1.2 * p.gamma)
    st = O.admm_direct(inst, o)
    assert max(st.residuals) <= 1e-9
    sol = O.polish(inst, st)
    v = O.kkt_violation(inst, sol)
    assert v["equality"] < 1e-10 and v["box"] < 1e-12 and v["sign_complementarity"] < 1e-8, v
    assert np.allclose(st.y, sol.y, atol=1e-7) and np.allclose(st.u, sol.u, atol=1e-7)
    ref = O.admm_direct(inst, O.AdmmOptions(delta=1.0, rho=1.618, tol=1e-9, max_iter=40000))
    assert np.allclose(st.y, ref.y, atol=1e-7)


def test_generalized_S_is_scalar_diagonal_plus_BtB_and_preconditioner_exact_scalars():
    """Algorithm 2's normal-equation matrix is m1 I + B^T B / m2 with the scalars
    the preconditioner uses, so S-tilde differs from S only by the circulant
    approximation of B."""
    inst = _instance()
    p = inst.params
    o = O.AdmmOptions(delta=0.6, rho=0.8, algorithm=2, c_y=1.5, c_u=0.02)
    S = O.assemble_S(p, o)
    m1, m2 = O.preconditioner_scalars(p, o)
    B = O.assemble_B(p)
    assert np.allclose(S, m1 * np.eye(p.N) + B.T @ B / m2, rtol=1e-12, atol=1e-12)
    psi = O.psi_scale(p)
    assert np.isclose(m1, o.rho * (o.c_y + 1 / o.delta))
    assert np.isclose(m2, psi ** 2 / (o.rho * (o.c_u + psi ** 2 / o.delta)) + o.delta / o.rho)


def test_generalized_options_are_checked():
    inst = _instance()
    p = inst.params
    with pytest.raises(ValueError):
        O.admm_diagonals(p, O.AdmmOptions(rho=1.2, algorithm=2, c_y=2.0, c_u=1.0))
    with pytest.raises(ValueError):
        O.admm_diagonals(p, O.AdmmOptions(rho=1.0, algorithm=2, c_y=0.9, c_u=1.0))
    with pytest.raises(ValueError):
        O.admm_diagonals(p, O.AdmmOptions(rho=1.0, algorithm=2, c_y=1.0, c_u=0.5 * p.gamma))
