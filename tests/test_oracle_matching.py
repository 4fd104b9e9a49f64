"""Pins of the matching Schur complement approximation (Section 3.2.2, Eq. (second
schur complement preconditioner)) in the oracle, with the circulant D-tilde =
C_3(B): its FFT-diagonal form against the dense product D-hat M2^-1 D-hat^T of
dense T. Chan circulants; the theorem's bound: with scalar M1, M2 (Algorithm 2)
and the exact B in D-hat, B + B^T is positive semi-definite and the eigenvalues
of S-bar^-1 S lie in [1/2, 1]; and PCG with S-hat converges to the exact
sub-problem solution in a number of iterations flat in n."""
import math

import numpy as np
import pytest

import fde_inputs as fi
import oracle as O


def _params(nx=5, ny=4, nt=3, **kw):
    base = dict(T=1.0, beta_x=1.4, beta_y=1.7, alpha_t=1.0, dp=1.0, dm=0.5, ep=0.8, em=0.3, gamma=1e-2)
    base.update(kw)
    return fi.FdeParams(nx=nx, ny=ny, nt=nt, **base)


@pytest.mark.parametrize("alg", [1, 2])
def test_matching_symbol_is_spectrum_of_dense_product(alg):
    p = _params()
    o = (O.AdmmOptions(delta=0.7, rho=1.3, precond=1) if alg == 1 else
         O.AdmmOptions(delta=0.7, rho=0.9, algorithm=2, c_y=1.2, c_u=0.02, precond=1))
    Sh = O.dense_matching_preconditioner(p, o)
    assert np.allclose(Sh, Sh.T, atol=1e-10)
    sig = O.preconditioner_symbol(p, o)
    assert np.allclose(np.sort(np.linalg.eigvalsh(Sh)), np.sort(sig.ravel()), rtol=1e-10, atol=1e-12)
    r = fi.random_field(3, (p.nt, p.nx, p.ny))
    assert np.allclose(O.apply_preconditioner(p, o, r).ravel(), np.linalg.solve(Sh, r.ravel()), rtol=1e-9,
                       atol=1e-12)
    # S-hat - S-tilde is the symmetric part of C_3 times 2 sqrt(m1/m2): positive semi-definite
    o0 = O.AdmmOptions(**{**o.__dict__, "precond": 0})
    St = O.dense_preconditioner(p, o0)
    assert np.linalg.eigvalsh(Sh - St)[0] >= -1e-10


@pytest.mark.parametrize("dims", [(5, 4, 3), (6, 6, 4)])
def test_matching_bound_with_scalar_blocks(dims):
    """Second part of the matching theorem: J1, J2 scaled identities (Algorithm 2
    makes the blocks scalar) and B + B^T >= 0 give eigenvalues of S-bar^-1 S in
    [1/2, 1], S-bar = (B^T + sqrt(m1 m2) I)(B + sqrt(m1 m2) I) / m2."""
    p = _params(*dims)
    o = O.AdmmOptions(delta=0.8, rho=1.0, algorithm=2, c_y=1.1, c_u=0.011)
    B = O.assemble_B(p)
    assert np.linalg.eigvalsh(B + B.T)[0] >= -1e-10
    S = O.assemble_S(p, o)
    m1, m2 = O.preconditioner_scalars(p, o)
    c = math.sqrt(m1 * m2)
    Sb = (B.T + c * np.eye(p.N)) @ (B + c * np.eye(p.N)) / m2
    mu = np.linalg.eigvals(np.linalg.solve(Sb, S)).real
    assert mu.min() >= 0.5 - 1e-10 and mu.max() <= 1.0 + 1e-10


def test_pcg_with_matching_preconditioner():
    counts = []
    for n in (4, 8, 16):
        p = _params(n, n, 4)
        inst = fi.FdeInstance(p, fi.desired_state_sine(p, 5), 0.1 * fi.random_field(6, (4, n, n)), None, None,
                              -0.2, 0.2, 5)
        o = O.AdmmOptions(delta=1.0, rho=1.618, precond=1)
        rhs, _, _ = O.admm_rhs(p, o, inst.ybar, inst.g, O.zero_state(p))
        y, it = O.pcg(lambda v: O.apply_S(p, o, v), lambda r: O.apply_preconditioner(p, o, r), rhs,
                      np.zeros_like(rhs), 1e-10, 500)
        if n == 4:
            assert np.allclose(y.ravel(), np.linalg.solve(O.assemble_S(p, o), rhs.ravel()), rtol=1e-8, atol=1e-10)
        counts.append(it)
    assert max(counts) <= 2 * min(counts) + 8, counts
