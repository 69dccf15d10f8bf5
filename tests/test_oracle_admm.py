"""Pins of the oracle's TV/ADMM iteration (Eq. 9-14, Algorithm 1): the
discrete gradient on functions whose gradient is known, its adjoint, the
isotropic shrink against numerical minimisation of its defining problem and
its special cases, conjugate gradients against a dense solve of the normal
equation built from the explicit Jacobian, and the whole step's bookkeeping
(g0 = grad m0, u0 = 0, dual factor)."""
import numpy as np
import pytest
from scipy import optimize

import oracle
from oracle import admm, inverse, model, operator
from paper_2604_15796_gb300 import phantoms


@pytest.mark.parametrize("shape", [(6, 7), (4, 5, 3)])
def test_grad_of_affine_function(shape):
    """m = a.x_index + c: interior differences equal a, last slice 0."""
    idx = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
    coef = [2.0 - 1j, 0.5, -3.0][:len(shape)]  # per array axis
    m = sum(c * i for c, i in zip(coef, idx)) + 7.0
    g = admm.grad_op(m, shape)
    d = len(shape)
    for q in range(d):
        ax = d - 1 - q  # component q differentiates along array axis d-1-q
        comp = np.moveaxis(g[q], ax, 0)
        assert np.allclose(comp[:-1], coef[ax])
        assert np.all(comp[-1] == 0)


@pytest.mark.parametrize("shape", [(6, 7), (4, 5, 3)])
def test_grad_adjoint_identity(shape):
    m = phantoms.complex_normal(shape, 1)
    a = phantoms.complex_normal((len(shape),) + shape, 2)
    lhs = np.vdot(admm.grad_op(m, shape), a)
    rhs = np.vdot(m, admm.grad_op_T(a, shape))
    assert np.isclose(lhs, rhs, rtol=1e-13)


def test_grad_T_grad_is_neumann_laplacian():
    """nabla^T nabla is the negative graph Laplacian of the grid: rows sum to
    zero and the diagonal counts the neighbours."""
    shape = (3, 4)
    n = 12
    M = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        M[:, j] = admm.grad_op_T(admm.grad_op(e.reshape(shape), shape),
                                 shape).real.ravel()
    assert np.allclose(M.sum(1), 0)
    deg = np.zeros(shape)
    for iz in range(3):
        for ix in range(4):
            deg[iz, ix] = (ix > 0) + (ix < 3) + (iz > 0) + (iz < 2)
    assert np.allclose(np.diag(M), deg.ravel())


@pytest.mark.parametrize("tau", [0.0, 0.3, 1.0, 10.0])
def test_shrink_is_the_prox_of_the_l12_norm(tau):
    """shrink_tau(a) = argmin_g tau ||g||_2 + 1/2 ||g - a||^2 per pixel
    (Eq. 13-14 with tau = lambda/rho), by numerical minimisation."""
    rng = np.random.default_rng(4)
    a = rng.standard_normal((2, 5)) + 1j * rng.standard_normal((2, 5))
    got = admm.shrink(a, tau)
    for n in range(a.shape[1]):
        an = a[:, n]

        def obj(x):
            g = x[:2] + 1j * x[2:]
            return tau * np.linalg.norm(g) + 0.5 * np.linalg.norm(g - an) ** 2
        x0 = np.concatenate([an.real, an.imag]) * 0.5
        res = optimize.minimize(obj, x0, method="Nelder-Mead",
                                options=dict(xatol=1e-10, fatol=1e-14,
                                             maxiter=20000))
        ref = res.x[:2] + 1j * res.x[2:]
        assert np.allclose(got[:, n], ref, atol=1e-6)


def test_shrink_special_cases():
    a = phantoms.complex_normal((3, 4, 5), 8)
    assert np.array_equal(admm.shrink(a, 0.0), a)
    big = np.sqrt((np.abs(a) ** 2).sum(0)).max()
    assert np.all(admm.shrink(a, big) == 0)
    z = np.zeros((2, 3), dtype=np.complex128)
    assert np.all(admm.shrink(z, 0.5) == 0)
    # optimality: g != 0 => (g - a) + tau g/||g|| = 0
    tau = 0.4
    g = admm.shrink(a, tau)
    ng = np.sqrt((np.abs(g) ** 2).sum(0))
    nz = ng > 0
    resid = (g - a)[:, nz] + tau * g[:, nz] / ng[nz]
    assert np.abs(resid).max() < 1e-12
    assert np.all(np.sqrt((np.abs(a) ** 2).sum(0))[~nz] <= tau + 1e-15)


def _step_setup(shape=(8, 7), n_elem=4):
    prob = oracle.Problem(shape, 0.1e-3, 1540.0,
                          model.linear_array(n_elem, 0.2e-3, 0.1e-3, 2),
                          np.array([2e6, 3.5e6]))
    rng = np.random.default_rng(2)
    m = 0.05 * rng.standard_normal(shape).astype(np.complex128)
    m_true = m + 0.02 * rng.standard_normal(shape)
    _, d_obs = inverse.forward_model(m_true, prob, "lu")
    out = inverse.gradient(m, d_obs, prob, "lu")
    rf = inverse.receiver_fields(m, prob, "lu")
    return prob, m, d_obs, out, rf


def test_cg_to_convergence_equals_dense_normal_equation():
    prob, m, d_obs, out, rf = _step_setup()
    params = admm.AdmmParams(lam=1e-4, rho=2e-3, gamma=1e-5, n_cg=400)
    g = admm.grad_op(m, prob.shape)
    u = 0.01 * phantoms.complex_normal(g.shape, 3)
    b = admm.normal_rhs(m, g, u, out["grad"], prob, params)
    J = inverse.jac_dense(out["fields"], rf, prob)
    n = prob.n
    L = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        L[:, j] = admm.grad_op_T(admm.grad_op(e.reshape(prob.shape), prob.shape),
                                 prob.shape).real.ravel()
    A = np.conj(J.T) @ J + params.rho * L + params.gamma * np.eye(n)
    assert np.allclose(A, np.conj(A.T), atol=1e-12 * np.abs(A).max())
    assert np.linalg.eigvalsh(A).min() > 0
    ref = np.linalg.solve(A, b.ravel())
    got = admm.cg(lambda v: admm.normal_matrix_apply(
        v, out["fields"], rf, prob, params).ravel(), b.ravel(), params.n_cg)
    assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref)
    # b_k's data term is J^H (d - F)
    rhs0 = admm.normal_rhs(m, admm.grad_op(m, prob.shape),
                           np.zeros_like(g), out["grad"], prob,
                           admm.AdmmParams(rho=1.0, gamma=0.0))
    assert np.allclose(rhs0.ravel(), np.conj(J.T) @ (d_obs - out["data"]).ravel())


def test_admm_step_bookkeeping():
    prob, m, d_obs, out, rf = _step_setup()
    params = admm.AdmmParams(lam=5e-4, rho=1e-3, gamma=1e-5, n_cg=5)
    g0 = admm.grad_op(m, prob.shape)
    u0 = np.zeros_like(g0)
    m1, g1, u1, sos, dm = admm.admm_tv_step(m, g0, u0, out["grad"],
                                            out["fields"], rf, prob, params)
    assert np.allclose(m1, m + dm)
    gm = admm.grad_op(m1, prob.shape)
    assert np.allclose(g1, admm.shrink(gm - u0, params.lam / params.rho))
    assert np.allclose(u1, u0 + params.rho * (g1 - gm))
    assert np.allclose(sos, 1540.0 / np.sqrt(1 + m1.real))
    p2 = admm.AdmmParams(lam=5e-4, rho=1e-3, gamma=1e-5, n_cg=5, dual_step=1.0)
    _, g2, u2, _, _ = admm.admm_tv_step(m, g0, u0, out["grad"], out["fields"],
                                        rf, prob, p2)
    assert np.allclose(u2, u0 + (g2 - gm))
    # with lambda = 0 the g-step returns grad m - u
    p3 = admm.AdmmParams(lam=0.0, rho=1e-3, gamma=1e-5, n_cg=5)
    m3, g3, u3, _, _ = admm.admm_tv_step(m, g0, u0, out["grad"], out["fields"],
                                         rf, prob, p3)
    assert np.allclose(g3, admm.grad_op(m3, prob.shape) - u0)
    assert np.allclose(u3, u0)


def test_m_step_decreases_the_linearised_objective():
    """Delta m from CG decreases the quadratic model of Eq. 9 (the
    Gauss-Newton linearisation) relative to Delta m = 0."""
    prob, m, d_obs, out, rf = _step_setup()
    params = admm.AdmmParams(lam=1e-4, rho=1e-3, gamma=1e-5, n_cg=10)
    g = admm.grad_op(m, prob.shape)
    u = np.zeros_like(g)
    _, _, _, _, dm = admm.admm_tv_step(m, g, u, out["grad"], out["fields"],
                                       rf, prob, params)

    def model_obj(delta):
        r = out["data"] + inverse.jac_forward(delta, out["fields"], rf, prob) - d_obs
        mm = m + delta
        return (0.5 * np.vdot(r, r).real
                + 0.5 * params.gamma * np.vdot(mm, mm).real
                + 0.5 * params.rho * np.linalg.norm(g - admm.grad_op(mm, prob.shape) + u) ** 2)
    assert model_obj(dm) < model_obj(np.zeros_like(m))


def test_sos_contrast_round_trip():
    c = np.array([1480.0, 1540.0, 1600.0])
    m = model.contrast_from_sos(c, 1540.0)
    assert np.allclose(model.sos_from_contrast(m, 1540.0), c, rtol=1e-15)
    assert m[1] == 0


def test_algorithm_1_reconstructs_an_inclusion():
    """Five iterations of Algorithm 1 (strict distorted-Born Jacobian, the
    paper's dual step u += rho (g - grad m)) on a 24 x 24 grid with one
    inclusion seen from one side: the misfit falls at every iteration and by
    more than 100x, the SoS moves toward the true map with the right sign,
    and TV keeps the background flat.  (With a single-sided array a smooth,
    lower-contrast inclusion already fits the data, so the SoS error falls
    by about a sixth, not severalfold.)"""
    import oracle
    from oracle import admm, inverse, model
    h = 0.1e-3
    shape = (24, 24)
    prob = oracle.Problem(shape, h, 1540.0, model.linear_array(12, 0.2e-3, h, 2),
                          np.array([1.0e6, 2.0e6, 3.0e6]))
    z, x = np.meshgrid(np.arange(24.0), np.arange(24.0), indexing="ij")
    sos_true = np.full(shape, 1540.0)
    sos_true[(x - 11.5) ** 2 + (z - 8.0) ** 2 <= 9.0] = 1580.0
    m_true = model.contrast_from_sos(sos_true, 1540.0)
    _, d = inverse.forward_model(m_true, prob, "lu")
    m0 = np.zeros(shape, dtype=np.complex128)
    scale = float(np.abs(inverse.gradient(m0, d, prob, "lu")["grad"]).max())
    p = admm.AdmmParams(lam=1e-4 * scale, rho=1e-2 * scale, gamma=1e-6 * scale, n_cg=10)
    m, g, u, sos, hist = admm.reconstruct(m0, d, prob, p, 5, "lu")
    mis = [h_[0] for h_ in hist]
    assert all(b < a for a, b in zip(mis, mis[1:]))
    assert mis[-1] < 1e-2 * mis[0]
    err0 = np.linalg.norm(1540.0 - sos_true)
    err = np.linalg.norm(sos - sos_true)
    assert err < 0.9 * err0
    inside = sos_true > 1540.0
    assert sos[inside].mean() > 1545.0                 # the inclusion appears, faster than c0
    assert np.abs(sos[~inside] - 1540.0).mean() < 2.0  # the background stays near c0


def _tv_prox_objective(m, d, lam, gamma, shape):
    """1/2 ||m - d||^2 + lam sum_n ||(nabla m)_n||_2 + gamma/2 ||m||^2: the
    objective of Eq. 7 when the data map is the identity and m_ref = 0."""
    gm = admm.grad_op(m.reshape(shape), shape)
    tv = np.sqrt((np.abs(gm) ** 2).sum(axis=0)).sum()
    r = m.ravel() - d.ravel()
    return 0.5 * np.vdot(r, r).real + lam * tv + 0.5 * gamma * np.vdot(m, m).real


@pytest.mark.parametrize("dual_step", [None, 1.0])
def test_admm_with_identity_jacobian_converges_to_the_tv_prox(dual_step):
    """With J = I (point fields p_e = delta_e and one receiver field equal
    to 1, so J a = a and grad = m - d), rho = 1 and the dual factor rho
    (the paper's) or 1 (they coincide at rho = 1), Algorithm 1 is scaled
    ADMM for the TV-denoising problem min 1/2||m - d||^2 + lam TV(m) +
    gamma/2 ||m||^2, whose minimiser is unique (the objective is
    1-strongly convex).  The iterates must reach the minimiser that a
    generic optimiser finds on the smoothed objective: a wrong sign or
    factor in the u-update, the shrink threshold or the m-step right-hand
    side converges elsewhere or not at all.  Strong convexity bounds the
    distance: F(m) - F* >= 1/2 ||m - m*||^2."""
    shape = (4, 4)
    n = 16
    rng = np.random.default_rng(5)
    d = 0.1 * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    d[:2, :] += 0.3  # a step edge for TV to keep
    lam, gamma = 0.02, 1e-3
    prob = oracle.Problem(shape, 1e-4, 1540.0, model.linear_array(n, 1e-4, 1e-4, 2),
                          np.array([1.0e6]))
    fields = np.eye(n, dtype=np.complex128).reshape((1, n) + shape)
    rfields = np.ones((1, 1) + shape, dtype=np.complex128)
    a = phantoms.complex_normal(shape, 9)
    assert np.allclose(inverse.jac_forward(a, fields, rfields, prob).ravel(), a.ravel())
    p = admm.AdmmParams(lam=lam, rho=1.0, gamma=gamma, n_cg=n, dual_step=dual_step)
    m = np.zeros(shape, dtype=np.complex128)
    g = admm.grad_op(m, shape)
    u = np.zeros_like(g)
    for _ in range(400):
        grad = m - d  # J^H (J m - d)
        m, g, u, _, _ = admm.admm_tv_step(m, g, u, grad, fields, rfields, prob, p)
    # generic optimiser on the smoothed objective (real and imaginary parts)
    eps = 1e-10

    def f(x):
        mm = (x[:n] + 1j * x[n:]).reshape(shape)
        gm = admm.grad_op(mm, shape)
        tv = np.sqrt((np.abs(gm) ** 2).sum(axis=0) + eps ** 2).sum()
        r = (mm - d).ravel()
        return 0.5 * np.vdot(r, r).real + lam * tv + 0.5 * gamma * np.vdot(mm, mm).real

    best = None
    for x0 in (np.concatenate([d.real.ravel(), d.imag.ravel()]), np.zeros(2 * n)):
        res = optimize.minimize(f, x0, method="BFGS", options={"gtol": 1e-12, "maxiter": 20000})
        if best is None or res.fun < best.fun:
            best = res
    m_opt = (best.x[:n] + 1j * best.x[n:]).reshape(shape)
    F_admm = _tv_prox_objective(m, d, lam, gamma, shape)
    F_opt = _tv_prox_objective(m_opt, d, lam, gamma, shape)
    assert F_admm <= F_opt + 1e-9
    assert np.linalg.norm(m - m_opt) <= 1e-3 * np.linalg.norm(d)
    # the constraint g = nabla m holds at the fixed point
    assert np.linalg.norm(g - admm.grad_op(m, shape)) <= 1e-6 * np.linalg.norm(g)
    # TV keeps the edge: the solution is not the plain shrunk data
    assert np.linalg.norm(m - d / (1 + gamma)) > 1e-2 * np.linalg.norm(d)


def test_admm_identity_jacobian_detects_a_flipped_dual_update():
    """The same iteration with the u-update's sign flipped (planted in a copy
    of the step, on the CPU) does not reach the TV-prox minimiser."""
    shape = (4, 4)
    n = 16
    rng = np.random.default_rng(5)
    d = 0.1 * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    d[:2, :] += 0.3
    lam, gamma = 0.02, 1e-3
    prob = oracle.Problem(shape, 1e-4, 1540.0, model.linear_array(n, 1e-4, 1e-4, 2),
                          np.array([1.0e6]))
    fields = np.eye(n, dtype=np.complex128).reshape((1, n) + shape)
    rfields = np.ones((1, 1) + shape, dtype=np.complex128)
    p = admm.AdmmParams(lam=lam, rho=1.0, gamma=gamma, n_cg=n)
    res = {}
    for flip in (False, True):
        m = np.zeros(shape, dtype=np.complex128)
        g = admm.grad_op(m, shape)
        u = np.zeros_like(g)
        for _ in range(400):
            u_prev = u
            m, g, u, _, _ = admm.admm_tv_step(m, g, u, m - d, fields, rfields, prob, p)
            if flip:
                u = u_prev - (u - u_prev)
        res[flip] = _tv_prox_objective(m, d, lam, gamma, shape)
    assert res[True] > res[False] + 1e-6
