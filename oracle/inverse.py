"""Data equation, misfit, adjoint state and Jacobian products (Eq. 4, 7,
15-17; Sec. IV-B, IV-C).  FP64 oracle; test infrastructure only.

Discretisation (readings):

* Receiver j is a point at the element position (Eq. 4 integrates over the
  element's sensing region Omega_j; a point element is taken), and the
  volume integral of Eq. 4 is a pixel sum:
      P^s_{l,e,j} = sum_n R_{l,j}(n) m_n p_{l,e}(n),
      R_{l,j}(n)  = k_l^2 dV G_l(x_j, x_n).
  Data are stored [l][e][j] (frequency, transmit, receive).
* The exact derivative of the discrete data map is
      dP_{l,e,j}/dm_n = ptilde_{l,j}(n) p_{l,e}(n),
      ptilde_{l,j} = A_l^{-1} R_{l,j}   (K is complex-symmetric),
  i.e. Eq. 15 with k^2 and the cell volume carried inside ptilde, and with
  "approximately equal" exact because ptilde is computed at the current
  iterate.  Because each receiver sits at an element position,
  R_{l,j} = k_l^2 dV p0_{l,j} and ptilde_{l,j} = k_l^2 dV p_{l,j} for the
  element's point-source field.  With point transmits at every element no
  extra solves are needed; with synthesised transmits (plane waves,
  Sec. V-A) the transmit fields differ from the receiver fields, which
  receiver_fields solves separately (refreshed on the schedule of
  Sec. IV-B, admm.reconstruct).
* Gradient of phi = 1/2 ||F(m) - d||^2 in the complex (Wirtinger) sense:
  grad = J^H r with r = F(m) - d, so that
  d phi(m + eps a)/d eps = Re <grad, a>.
"""
import numpy as np

from . import model, operator


def receiver_rows(prob):
    """R_{l,j}(n) = k_l^2 dV G_l(x_j, x_n), the receiver's sensing of pixel n
    (for 3-D line elements the mean of G over the element, see
    operator.element_green).  [N_F, N_R, *shape]."""
    k = model.wavenumbers(prob)
    g = operator.element_green(prob)
    return g * (k * k * prob.cell_volume).reshape((-1,) + (1,) * (prob.dim + 1))


def _flat(a, prob):
    return a.reshape(a.shape[:a.ndim - prob.dim] + (prob.n,))


def forward_data(m, fields, prob, rows=None):
    """P^s_{l,e,j} = sum_n R_{l,j}(n) m_n p_{l,e}(n)   (Eq. 4)."""
    if rows is None:
        rows = receiver_rows(prob)
    mf = np.asarray(m, dtype=np.complex128).ravel()
    p = _flat(fields, prob)
    R = _flat(rows, prob)
    return np.einsum("len,ljn->lej", p * mf[None, None, :], R)


def misfit(d, d_obs):
    """phi = 1/2 ||F(m) - d_obs||_2^2 (first term of Eq. 7)."""
    r = np.asarray(d) - np.asarray(d_obs)
    return 0.5 * float(np.vdot(r, r).real)


def forward_model(m, prob, method="lu", tol=1e-10, weights=None):
    """F(m): fields and data (Eq. 4-6).  Returns (fields, data).

    With ``weights`` [N_F, N_T, N_E] the transmits are synthesised ones
    (plane waves, Sec. V-A): each transmit field is solved directly from
    its own incident field, A_l p_{l,i} = sum_e w_{l,i,e} p0_{l,e}, and the
    data are [l][i][j] with every element receiving."""
    p0 = None if weights is None else operator.transmit_incident_fields(prob, weights)
    fields = operator.solve_forward(m, prob, method, tol, p0=p0)
    return fields, forward_data(m, fields, prob)


def receiver_fields(m, prob, method="lu", tol=1e-10):
    """ptilde_{l,j} = A_l^{-1} R_{l,j} by its definition (one solve each)."""
    rows = receiver_rows(prob)
    out = np.empty_like(rows)
    for l in range(prob.n_freq):
        out[l], _ = operator.solve(m, rows[l], prob, l, method, tol)
    return out


def adjoint_sources(resid, prob, rows=None):
    """s_{l,e} = sum_j conj(R_{l,j}) r_{l,e,j}: the right-hand sides of the
    adjoint-state equations (Sec. IV-B)."""
    if rows is None:
        rows = receiver_rows(prob)
    R = _flat(rows, prob)
    s = np.einsum("lej,ljn->len", np.asarray(resid), np.conj(R))
    return s.reshape(s.shape[:2] + tuple(prob.shape))  # [N_F, N_T, *shape]


def apply_AH(v, m, prob, l, spec=None):
    """A^H v for A = I - K M:  A^H = I - conj(M) K^H, and K^H w = conj(K conj(w))
    because K is complex-symmetric."""
    m = np.asarray(m, dtype=np.complex128).reshape(prob.shape)
    return v - np.conj(m) * np.conj(operator.apply_K(np.conj(v), prob, l, spec))


def apply_adjoint_state_op(v, m, prob, l, spec=None):
    """(I - M K)^H v = v - K^H(conj(m) v): the operator of the adjoint-state
    equations.  (I - M K)^H = conj(I - K M) = conj(A) since K^T = K."""
    m = np.asarray(m, dtype=np.complex128).reshape(prob.shape)
    return v - np.conj(operator.apply_K(m * np.conj(v), prob, l, spec))


def solve_adjoint(m, src, prob, method="lu", tol=1e-10):
    """Adjoint fields lambda_{l,e} solving (I - M K)^H lambda = s_{l,e}.

    Note (I - M K)^H = (I - K M)^T conjugated = conj(A), since K^T = K.
    'lu' factorises the conjugate transpose of dense (I - M K) directly;
    'bicgstab' iterates with apply_adjoint_state_op.
    """
    src = np.asarray(src, dtype=np.complex128)
    out = np.empty_like(src)
    mm = np.asarray(m, dtype=np.complex128).ravel()
    for l in range(prob.n_freq):
        nb = src.shape[1]
        rhs = src[l].reshape(nb, prob.n)
        if method == "lu":
            K = operator.dense_K(prob, l)
            IMK = np.eye(prob.n, dtype=np.complex128) - mm[:, None] * K
            sol = np.linalg.solve(np.conj(IMK.T), rhs.T).T
        else:
            spec = operator.kernel_spectrum(prob, l)

            def apply(v, l=l, spec=spec):
                return apply_adjoint_state_op(v.reshape(prob.shape), mm, prob,
                                              l, spec).ravel()

            sol = np.empty_like(rhs)
            for i in range(nb):
                sol[i], _, _ = operator.bicgstab(apply, rhs[i], tol)
        out[l] = sol.reshape(src[l].shape)
    return out


def gradient_adjoint_state(fields, lam, prob):
    """grad_n = sum_{l,e} conj(p_{l,e}(n)) lambda_{l,e}(n)  (= J^H r)."""
    return np.einsum("len,len->n", np.conj(_flat(fields, prob)),
                     _flat(lam, prob))


def jac_forward(a, fields, rfields, prob):
    """(J a)_{l,e,j} = sum_n p_{l,e}(n) ptilde_{l,j}(n) a_n   (Eq. 16)."""
    af = np.asarray(a, dtype=np.complex128).ravel()
    return np.einsum("len,ljn->lej", _flat(fields, prob) * af,
                     _flat(rfields, prob))


def jac_adjoint(b, fields, rfields, prob):
    """(J^H b)_n = sum_{l,e,j} conj(p_{l,e}(n)) conj(ptilde_{l,j}(n)) b_{l,e,j}
    (Eq. 17, with the k^2 factor moved inside the sum over l)."""
    inner = np.einsum("lej,ljn->len", np.asarray(b),
                      np.conj(_flat(rfields, prob)))
    return np.einsum("len,len->n", np.conj(_flat(fields, prob)), inner)


def jac_dense(fields, rfields, prob):
    """Explicit J: rows (l, e, j), columns n (small grids only)."""
    p = _flat(fields, prob)
    q = _flat(rfields, prob)
    J = p[:, :, None, :] * q[:, None, :, :]
    return J.reshape(-1, prob.n)


def gradient(m, d_obs, prob, method="lu", tol=1e-10, weights=None):
    """One gradient evaluation: forward solves, data, misfit, adjoint
    sources, adjoint solves, assembly.  Returns a dict with every
    intermediate (fields, data, resid, misfit, lam, grad).  ``weights``:
    synthesised transmits (see forward_model); one forward and one adjoint
    solve per transmit and frequency."""
    fields, data = forward_model(m, prob, method, tol, weights)
    resid = data - np.asarray(d_obs)
    src = adjoint_sources(resid, prob)
    lam = solve_adjoint(m, src, prob, method, tol)
    return dict(fields=fields, data=data, resid=resid,
                misfit=misfit(data, d_obs), src=src, lam=lam,
                grad=gradient_adjoint_state(fields, lam, prob))


def gradient_inversion_mesh(m_inv, d_obs, prob, method="lu", tol=1e-10, weights=None):
    """Gradient with respect to the contrast on the inversion mesh: the
    forward model runs on the prolonged contrast, F(P m), and the gradient
    is P^T J^H r (chain rule).  The dict of gradient() plus "grad_inv"."""
    ref = gradient(model.prolong(m_inv, prob), d_obs, prob, method, tol, weights)
    ref["grad_inv"] = model.restrict(ref["grad"], prob)
    return ref

