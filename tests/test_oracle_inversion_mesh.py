"""Pins of the oracle's inversion mesh (Sec. IV: the contrast is inverted on
a mesh coarser than the forward mesh; reading: each inversion cell covers
r^d forward pixels with a constant contrast):

* restrict is the adjoint of prolong, <P a, b> = <a, P^T b>;
* the inversion-mesh gradient against central finite differences of the
  misfit of the prolonged model;
* the inversion-mesh normal operator of the m-step (Eq. 12 with J P) is
  Hermitian positive definite, and CG run to convergence solves the
  explicit normal equations built from the dense J and P;
* r = 1 reproduces the forward-mesh step exactly."""
import numpy as np
import pytest

import oracle
from oracle import admm, inverse, model
from paper_2604_15796_gb300 import phantoms


def make(shape=(8, 12), r=2, n_elem=4, freqs=(1.5e6, 3e6), h=0.1e-3, seed=11):
    dim = len(shape)
    prob = oracle.Problem(shape, h, 1540.0, model.linear_array(n_elem, 0.2e-3, h, dim),
                          np.array(freqs))
    prob.extra["inv_factor"] = r
    rng = np.random.default_rng(seed)
    sh = model.inversion_shape(prob)
    m = 0.06 * (rng.standard_normal(sh) + 0.1j * rng.standard_normal(sh))
    return prob, m


def dense_prolong(prob):
    n_inv = int(np.prod(model.inversion_shape(prob)))
    P = np.zeros((prob.n, n_inv))
    for j in range(n_inv):
        e = np.zeros(n_inv)
        e[j] = 1.0
        P[:, j] = model.prolong(e, prob).ravel()
    return P


@pytest.mark.parametrize("shape,r", [((8, 12), 2), ((6, 9), 3), ((4, 6, 8), 2)])
def test_restrict_is_the_adjoint_of_prolong(shape, r):
    prob, _ = make(shape, r)
    sh = model.inversion_shape(prob)
    a = phantoms.complex_normal(sh, 1)
    b = phantoms.complex_normal(prob.shape, 2)
    assert np.isclose(np.vdot(model.prolong(a, prob), b), np.vdot(a, model.restrict(b, prob)),
                      rtol=1e-13)
    assert np.allclose(model.prolong(np.full(sh, 2.5), prob), 2.5)
    assert np.allclose(model.restrict(np.ones(prob.shape), prob), r ** len(shape))


def test_inversion_mesh_gradient_against_finite_differences():
    prob, m = make()
    _, d = inverse.forward_model(model.prolong(1.3 * m + 0.01, prob), prob, "lu")
    ref = inverse.gradient_inversion_mesh(m, d, prob, "lu")
    a = phantoms.complex_normal(m.shape, 3)
    eps = 1e-6

    def phi(mm):
        return inverse.misfit(inverse.forward_model(model.prolong(mm, prob), prob, "lu")[1], d)

    fd = (phi(m + eps * a) - phi(m - eps * a)) / (2 * eps)
    assert ref["grad_inv"].shape == m.shape
    assert np.isclose(fd, np.vdot(ref["grad_inv"], a).real, rtol=1e-6)


def test_inversion_mesh_normal_equations():
    prob, m = make()
    mf = model.prolong(m, prob)
    fields = inverse.forward_model(mf, prob, "lu")[0]
    rf = inverse.receiver_fields(mf, prob, "lu")
    p = admm.AdmmParams(lam=1e-3, rho=0.3, gamma=0.05, n_cg=10)
    sh = model.inversion_shape(prob)
    n_inv = int(np.prod(sh))

    def N(v):
        return admm.normal_matrix_apply(v, fields, rf, prob, p).ravel()

    a = phantoms.complex_normal(sh, 4).ravel()
    b = phantoms.complex_normal(sh, 5).ravel()
    assert np.isclose(np.vdot(N(a), b), np.vdot(a, N(b)), rtol=1e-12)
    assert np.vdot(N(a), a).real > 0
    # explicit normal matrix: (J P)^H (J P) + rho D^T D + gamma I
    JP = inverse.jac_dense(fields, rf, prob) @ dense_prolong(prob)
    cols = np.stack([admm.grad_op_T(admm.grad_op(e.reshape(sh), sh), sh).ravel()
                     for e in np.eye(n_inv)], axis=1)
    Nd = JP.conj().T @ JP + p.rho * cols + p.gamma * np.eye(n_inv)
    assert np.allclose(Nd @ a, N(a), rtol=1e-10, atol=1e-12 * np.abs(Nd @ a).max())
    x = admm.cg(lambda v: N(v), b, 4 * n_inv)
    assert np.allclose(x, np.linalg.solve(Nd, b), rtol=1e-6, atol=1e-9 * np.abs(x).max())


def test_unit_factor_reproduces_the_forward_mesh_step():
    prob, _ = make(r=1)
    m = 0.05 * phantoms.complex_normal(prob.shape, 6)
    _, d = inverse.forward_model(1.5 * m, prob, "lu")
    ref = inverse.gradient_inversion_mesh(m, d, prob, "lu")
    ref0 = inverse.gradient(m, d, prob, "lu")
    assert np.array_equal(ref["grad_inv"].ravel(), ref0["grad"].ravel())
    rf = inverse.receiver_fields(m, prob, "lu")
    p = admm.AdmmParams(lam=1e-3, rho=0.3, gamma=0.05, n_cg=5)
    g = admm.grad_op(m, prob.shape)
    u = np.zeros_like(g)
    out = admm.admm_tv_step(m, g, u, ref["grad_inv"], ref["fields"], rf, prob, p)
    del prob.extra["inv_factor"]
    out0 = admm.admm_tv_step(m, g, u, ref0["grad"], ref0["fields"], rf, prob, p)
    for x, y in zip(out, out0):
        assert np.array_equal(x, y)
