"""Pins of the oracle's data map, adjoint state, gradient and Jacobian
products (Eq. 4, 7, 15-17): source-receiver reciprocity, adjoint identities
<Au, v> = <u, A^H v> and <Ja, b> = <a, J^H b>, the Jacobian and the gradient
against central finite differences of the forward map and the misfit, the
receiver fields by their definition, and the agreement of the two gradient
routes (adjoint solves vs direct contraction with the receiver fields)."""
import numpy as np
import pytest

import oracle
from oracle import inverse, model, operator
from paper_2604_15796_gb300 import phantoms


def make(shape=(14, 12), n_elem=5, freqs=(1.5e6, 3e6), h=0.1e-3, seed=11,
         amp=0.06):
    dim = len(shape)
    prob = oracle.Problem(shape, h, 1540.0,
                          model.linear_array(n_elem, 0.2e-3, h, dim),
                          np.array(freqs))
    rng = np.random.default_rng(seed)
    m = amp * (rng.standard_normal(shape) + 0.1j * rng.standard_normal(shape))
    return prob, m.astype(np.complex128)


def cn(shape, seed):
    return phantoms.complex_normal(shape, seed)


@pytest.mark.parametrize("shape", [(14, 12), (5, 4, 6)])
def test_reciprocity(shape):
    prob, m = make(shape, n_elem=4)
    _, data = inverse.forward_model(m, prob, "lu")
    for l in range(prob.n_freq):
        assert np.allclose(data[l], data[l].T, rtol=1e-10, atol=1e-14 * np.abs(data[l]).max())


def test_adjoint_identities_of_operators():
    prob, m = make()
    u = cn(prob.shape, 1)
    v = cn(prob.shape, 2)
    for l in range(prob.n_freq):
        Au = operator.apply_A(u, m, prob, l)
        AHv = inverse.apply_AH(v, m, prob, l)
        assert np.isclose(np.vdot(Au, v), np.vdot(u, AHv), rtol=1e-12)
        Bu = u - m * operator.apply_K(u, prob, l)
        BHv = inverse.apply_adjoint_state_op(v, m, prob, l)
        assert np.isclose(np.vdot(Bu, v), np.vdot(u, BHv), rtol=1e-12)
        Ku = operator.apply_K(u, prob, l)
        KHv = np.conj(operator.apply_K(np.conj(v), prob, l))
        assert np.isclose(np.vdot(Ku, v), np.vdot(u, KHv), rtol=1e-12)
    # the dense matrix of K is symmetric (not Hermitian)
    K = operator.dense_K(prob, 0)
    assert np.allclose(K, K.T, rtol=0, atol=1e-15 * np.abs(K).max())


def test_receiver_fields_are_scaled_transmit_fields():
    prob, m = make()
    fields = operator.solve_forward(m, prob, "lu")
    rf = inverse.receiver_fields(m, prob, "lu")
    k = model.wavenumbers(prob)
    for l in range(prob.n_freq):
        assert np.allclose(rf[l], k[l] ** 2 * prob.cell_volume * fields[l],
                           rtol=1e-10, atol=0)


def test_jacobian_adjoint_identity_and_dense_form():
    prob, m = make()
    fields = operator.solve_forward(m, prob, "lu")
    rf = inverse.receiver_fields(m, prob, "lu")
    a = cn(prob.shape, 3)
    b = cn((prob.n_freq, prob.n_elem, prob.n_elem), 4)
    Ja = inverse.jac_forward(a, fields, rf, prob)
    JHb = inverse.jac_adjoint(b, fields, rf, prob)
    assert np.isclose(np.vdot(Ja, b), np.vdot(a.ravel(), JHb), rtol=1e-12)
    J = inverse.jac_dense(fields, rf, prob)
    assert np.allclose(J @ a.ravel(), Ja.ravel(), rtol=1e-12)
    assert np.allclose(np.conj(J.T) @ b.ravel(), JHb, rtol=1e-12)


def test_jacobian_matches_finite_differences_of_forward_map():
    prob, m = make()
    fields = operator.solve_forward(m, prob, "lu")
    rf = inverse.receiver_fields(m, prob, "lu")
    a = cn(prob.shape, 5) * 1e-2
    eps = 1e-4
    _, dp = inverse.forward_model(m + eps * a, prob, "lu")
    _, dm = inverse.forward_model(m - eps * a, prob, "lu")
    fd = (dp - dm) / (2 * eps)
    Ja = inverse.jac_forward(a, fields, rf, prob)
    assert np.linalg.norm(fd - Ja) <= 1e-7 * np.linalg.norm(Ja)


def _problem_with_data(shape=(14, 12)):
    prob, m = make(shape)
    rng = np.random.default_rng(21)
    m_true = m + 0.03 * rng.standard_normal(prob.shape)
    _, d_obs = inverse.forward_model(m_true, prob, "lu")
    return prob, m, d_obs


@pytest.mark.parametrize("direction", ["real", "imag"])
def test_gradient_matches_finite_differences_of_misfit(direction):
    prob, m, d_obs = _problem_with_data()
    out = inverse.gradient(m, d_obs, prob, "lu")
    a = cn(prob.shape, 7).real * 1e-2
    if direction == "imag":
        a = 1j * a
    eps = 1e-4

    def phi(mm):
        _, d = inverse.forward_model(mm, prob, "lu")
        return inverse.misfit(d, d_obs)
    fd = (phi(m + eps * a) - phi(m - eps * a)) / (2 * eps)
    an = np.real(np.vdot(out["grad"], a.ravel()))
    assert abs(fd - an) <= 1e-6 * abs(an)


def test_gradient_routes_agree():
    """Adjoint solves (one per transmit per frequency) and the direct
    contraction J^H r with the receiver fields give the same gradient."""
    prob, m, d_obs = _problem_with_data()
    out = inverse.gradient(m, d_obs, prob, "lu")
    rf = inverse.receiver_fields(m, prob, "lu")
    g2 = inverse.jac_adjoint(out["resid"], out["fields"], rf, prob)
    assert np.linalg.norm(out["grad"] - g2) <= 1e-10 * np.linalg.norm(g2)
    # and Krylov solves reach the same gradient as dense LU
    out_it = inverse.gradient(m, d_obs, prob, "bicgstab", tol=1e-12)
    assert np.linalg.norm(out_it["grad"] - out["grad"]) <= 1e-9 * np.linalg.norm(out["grad"])


def test_adjoint_solve_is_conjugate_forward_solve():
    prob, m, d_obs = _problem_with_data()
    out = inverse.gradient(m, d_obs, prob, "lu")
    for l in range(prob.n_freq):
        y, _ = operator.solve(m, np.conj(out["src"][l]), prob, l, "lu")
        assert np.allclose(np.conj(y), out["lam"][l], rtol=1e-10,
                           atol=1e-14 * np.abs(y).max())


def test_misfit_is_half_squared_norm():
    d = np.array([[1 + 2j, 3.0]])
    assert inverse.misfit(d, np.zeros_like(d)) == 0.5 * (1 + 4 + 9)
