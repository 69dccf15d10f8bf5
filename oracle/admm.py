"""TV-regularised ADMM iteration (Sec. III, Eq. 7-14, Algorithm 1).
FP64 oracle; test infrastructure only.

Readings of points the paper leaves open:

* Discrete gradient: forward difference in index units (no 1/h),
  (d_q m)_n = m_{n + e_q} - m_n, zero on the last slice of axis q
  (Neumann).  Components are ordered (x, [y], z), stored [d, *shape].
  nabla^T is the exact adjoint (a negative backward divergence).
* m-step: the Gauss-Newton normal equation (Eq. 11-12) is solved with
  conjugate gradients for exactly ``n_cg`` iterations from dm = 0, no
  preconditioner (the paper allows "GMRES or conjugate gradient").
* Dual update uses the factor the paper prints, u += rho (g - grad m);
  ``dual_step`` exposes the factor (1 gives the usual scaled form).
* Initialisation (Algorithm 1): g0 = nabla m0, u0 = 0.
"""
from dataclasses import dataclass

import numpy as np

from . import inverse, model


@dataclass
class AdmmParams:
    lam: float = 1e-4      # lambda, TV weight (Eq. 7)
    rho: float = 1e-3      # ADMM penalty (Eq. 8)
    gamma: float = 1e-5    # reference-model weight (Eq. 7)
    n_cg: int = 10         # CG iterations of the m-step
    dual_step: float = None  # factor of the u-update; None -> rho


def _axes(shape):
    """Array axis of each gradient component, components ordered (x,[y],z)."""
    d = len(shape)
    return [d - 1 - q for q in range(d)]


def grad_op(m, shape):
    """nabla m, [d, *shape] (forward differences, Neumann)."""
    m = np.asarray(m, dtype=np.complex128).reshape(shape)
    out = np.zeros((len(shape),) + tuple(shape), dtype=np.complex128)
    for q, ax in enumerate(_axes(shape)):
        sl_hi = [slice(None)] * len(shape)
        sl_lo = [slice(None)] * len(shape)
        sl_hi[ax] = slice(1, None)
        sl_lo[ax] = slice(0, -1)
        out[q][tuple(sl_lo)] = m[tuple(sl_hi)] - m[tuple(sl_lo)]
    return out


def grad_op_T(a, shape):
    """nabla^T a = sum_q d_q^T a_q (the adjoint of grad_op)."""
    a = np.asarray(a, dtype=np.complex128).reshape((len(shape),) + tuple(shape))
    out = np.zeros(tuple(shape), dtype=np.complex128)
    for q, ax in enumerate(_axes(shape)):
        sl_hi = [slice(None)] * len(shape)
        sl_lo = [slice(None)] * len(shape)
        sl_hi[ax] = slice(1, None)
        sl_lo[ax] = slice(0, -1)
        # d_q maps m -> a with a_lo = m_hi - m_lo; its transpose sends a_lo
        # to +a at hi and -a at lo.
        out[tuple(sl_hi)] += a[q][tuple(sl_lo)]
        out[tuple(sl_lo)] -= a[q][tuple(sl_lo)]
    return out


def cg(apply, b, n_iter):
    """Conjugate gradients (Hestenes-Stiefel) for a Hermitian positive
    (semi-)definite operator, exactly ``n_iter`` iterations from x = 0
    (stopping early only on an exactly zero residual)."""
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b)
    r = b.copy()
    d = r.copy()
    rr = np.vdot(r, r).real
    for _ in range(n_iter):
        if rr == 0.0:
            break
        q = apply(d)
        alpha = rr / np.vdot(d, q).real
        x = x + alpha * d
        r = r - alpha * q
        rr_new = np.vdot(r, r).real
        d = r + (rr_new / rr) * d
        rr = rr_new
    return x


def normal_matrix_apply(a, fields, rfields, prob, params):
    """A_k a = J^H J a + rho nabla^T nabla a + gamma a   (Eq. 12), on the
    inversion mesh: J acts on the prolonged vector and J^H is restricted
    (J_inv = J P, model.prolong / model.restrict; identity when the meshes
    coincide)."""
    shape = model.inversion_shape(prob)
    a = np.asarray(a, dtype=np.complex128).reshape(shape)
    af = model.prolong(a, prob)
    out = model.restrict(inverse.jac_adjoint(inverse.jac_forward(af, fields, rfields, prob),
                                             fields, rfields, prob).reshape(prob.shape), prob)
    out += params.rho * grad_op_T(grad_op(a, shape), shape)
    out += params.gamma * a
    return out


def normal_rhs(m, g, u, grad, prob, params, m_ref=None):
    """b_k = J^H(d - F(m)) + rho nabla^T(g + u - nabla m) + gamma(m_ref - m)
    (Eq. 12), with J^H(d - F(m)) = -grad; m, g, u, grad on the inversion
    mesh."""
    shape = model.inversion_shape(prob)
    m = np.asarray(m, dtype=np.complex128).reshape(shape)
    b = -np.asarray(grad, dtype=np.complex128).reshape(shape)
    b = b + params.rho * grad_op_T(np.asarray(g) + np.asarray(u)
                                   - grad_op(m, shape), shape)
    mr = np.zeros(shape, dtype=np.complex128) if m_ref is None \
        else np.asarray(m_ref, dtype=np.complex128).reshape(shape)
    return b + params.gamma * (mr - m)


def shrink(a, tau):
    """Isotropic shrinkage (Eq. 14), per pixel over the d components of
    ``a`` [d, *shape]: max(1 - tau/||a_n||, 0) a_n, and 0 where a_n = 0."""
    a = np.asarray(a, dtype=np.complex128)
    nrm = np.sqrt((np.abs(a) ** 2).sum(axis=0))
    scale = np.zeros_like(nrm)
    nz = nrm > 0
    scale[nz] = np.maximum(1.0 - tau / nrm[nz], 0.0)
    return a * scale[None]


def admm_tv_step(m, g, u, grad, fields, rfields, prob, params, m_ref=None):
    """One iteration of Algorithm 1 after the forward simulation and the
    gradient: Gauss-Newton m-step (Eq. 10-12), g-step (Eq. 13), u-step.
    m, g, u, grad (and the results) live on the inversion mesh, the fields
    on the forward mesh.  Returns (m_new, g_new, u_new, sos_new, dm)."""
    shape = model.inversion_shape(prob)
    b = normal_rhs(m, g, u, grad, prob, params, m_ref)
    dm = cg(lambda v: normal_matrix_apply(v, fields, rfields, prob, params),
            b, params.n_cg)
    m_new = np.asarray(m, dtype=np.complex128).reshape(shape) + dm
    gm = grad_op(m_new, shape)
    g_new = shrink(gm - np.asarray(u), params.lam / params.rho)
    step = params.rho if params.dual_step is None else params.dual_step
    u_new = np.asarray(u) + step * (g_new - gm)
    sos = model.sos_from_contrast(m_new, prob.c0, model.background_alpha(prob))
    return m_new, g_new, u_new, sos, dm


def reconstruct(m0, d_obs, prob, params, n_iter, method="bicgstab", tol=1e-10, weights=None,
                refresh_every=1, m_ref=None):
    """Algorithm 1 for ``n_iter`` iterations with the hybrid Born /
    distorted-Born Jacobian of Sec. IV-B: every iteration solves the
    transmit fields and the adjoint states at the current model (gradient),
    while the receiver fields ptilde_j = A^{-1} R_j (solved separately, one
    solve per receiver and frequency) are refreshed only on iterations
    k = 0, refresh_every, 2 refresh_every, ... and kept fixed in between
    (a Born approximation for the adjoint problem).  refresh_every = 1 is
    the strict distorted-Born Jacobian.  ``weights``: synthesised transmits
    (plane waves, Sec. V-A).  The model lives on the inversion mesh
    (model.prolong).  Returns (m, g, u, sos, history) with
    history[k] = (misfit, refreshed)."""
    shape = model.inversion_shape(prob)
    m = np.asarray(m0, dtype=np.complex128).reshape(shape).copy()
    g = grad_op(m, shape)
    u = np.zeros_like(g)
    rfields = None
    sos = model.sos_from_contrast(m, prob.c0, model.background_alpha(prob))
    history = []
    for k in range(n_iter):
        ref = inverse.gradient_inversion_mesh(m, d_obs, prob, method, tol, weights)
        refreshed = rfields is None or k % refresh_every == 0
        if refreshed:
            rfields = inverse.receiver_fields(model.prolong(m, prob), prob, method, tol)
        m, g, u, sos, _ = admm_tv_step(m, g, u, ref["grad_inv"], ref["fields"], rfields, prob,
                                       params, m_ref)
        history.append((ref["misfit"], refreshed))
    return m, g, u, sos, history

