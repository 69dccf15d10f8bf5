"""Pins of the oracle's synthesised (plane-wave) transmits (Sec. V-A) and of
the hybrid Born / distorted-Born refresh schedule (Sec. IV-B):

* superposition: plane-wave data solved directly from the plane-wave
  incident fields equal the weighted sums of the point-source data;
* mirror symmetry: in a medium symmetric in x, the data of angle theta at
  receiver j equal those of -theta at the mirrored receiver;
* steering: the synthesised incident field advances its phase along x at
  the rate k sin(theta) under the array (sign and size of the delay law);
* the plane-wave gradient and Jacobian against central finite differences
  of the misfit and of the data map, and <Ja, b> = <a, J^H b> with
  N_T != N_R;
* the refresh schedule: receiver fields are re-solved exactly on the
  iterations it names and reused otherwise."""
import numpy as np
import pytest

import oracle
from oracle import admm, inverse, model, operator
from paper_2604_15796_gb300 import phantoms


def make(shape=(14, 12), n_elem=5, freqs=(1.5e6, 3e6), h=0.1e-3, seed=11, amp=0.06):
    dim = len(shape)
    prob = oracle.Problem(shape, h, 1540.0, model.linear_array(n_elem, 0.2e-3, h, dim),
                          np.array(freqs))
    rng = np.random.default_rng(seed)
    m = amp * (rng.standard_normal(shape) + 0.1j * rng.standard_normal(shape))
    return prob, m.astype(np.complex128)


ANGLES = np.deg2rad([-40.0, -7.5, 0.0, 25.0])


def test_plane_wave_data_are_weighted_sums_of_point_source_data():
    prob, m = make()
    w = model.plane_wave_weights(prob, ANGLES)
    _, d_pw = inverse.forward_model(m, prob, "lu", weights=w)
    _, d_ps = inverse.forward_model(m, prob, "lu")
    synth = np.einsum("lie,lej->lij", w, d_ps)
    assert d_pw.shape == (prob.n_freq, len(ANGLES), prob.n_elem)
    assert np.allclose(d_pw, synth, rtol=1e-10, atol=1e-12 * np.abs(synth).max())


def test_mirror_symmetry_of_plane_wave_data():
    prob, m = make(shape=(10, 12), n_elem=6)
    m = 0.5 * (m + m[:, ::-1])  # symmetric in x; the array is centred
    ang = np.deg2rad([-30.0, -10.0, 10.0, 30.0])
    w = model.plane_wave_weights(prob, ang)
    _, d = inverse.forward_model(m, prob, "lu", weights=w)
    # theta_i and -theta_i are entries i and 3 - i; receiver j mirrors to N_E - 1 - j
    mirrored = d[:, ::-1, ::-1]
    assert np.allclose(d, mirrored, rtol=1e-10, atol=1e-12 * np.abs(d).max())
    # and the steering is not trivial: +theta and -theta differ at one receiver
    assert not np.allclose(d[:, 0, 0], d[:, 3, 0], rtol=1e-3)


@pytest.mark.parametrize("deg", [-20.0, 20.0])
def test_synthesised_wave_travels_in_the_steering_direction(deg):
    """Wide aperture (12.8 mm, 42 wavelengths at 5 MHz): at 2 mm depth under
    the array centre the phase advances along x at k sin(theta)."""
    h = 0.1e-3
    prob = oracle.Problem((24, 64), h, 1540.0, model.linear_array(128, 0.1e-3, h, 2),
                          np.array([5e6]))
    theta = np.deg2rad(deg)
    p0 = operator.transmit_incident_fields(prob, model.plane_wave_weights(prob, [theta]))
    row = p0[0, 0, 20]                       # depth 20 h = 2 mm
    dphi = np.angle(row[33] / row[31]) / (2 * h)
    k = model.wavenumbers(prob)[0]
    assert abs(dphi / k - np.sin(theta)) < 0.05


def test_plane_wave_gradient_and_jacobian_against_finite_differences():
    prob, m = make(n_elem=4)
    w = model.plane_wave_weights(prob, ANGLES)      # N_T = 4 = N_R here ...
    w = w[:, :3]                                    # ... and 3 != 4 here
    _, d_true = inverse.forward_model(m + 0.02, prob, "lu", weights=w)
    ref = inverse.gradient(m, d_true, prob, "lu", weights=w)
    a = phantoms.complex_normal(prob.shape, 3)
    eps = 1e-6

    def phi(mm):
        return inverse.misfit(inverse.forward_model(mm, prob, "lu", weights=w)[1], d_true)

    fd = (phi(m + eps * a) - phi(m - eps * a)) / (2 * eps)
    assert np.isclose(fd, np.vdot(ref["grad"], a).real, rtol=1e-6)
    # J a by the receiver fields (separate solves) against the data map
    rf = inverse.receiver_fields(m, prob, "lu")
    ja = inverse.jac_forward(a, ref["fields"], rf, prob)
    dfd = (inverse.forward_model(m + eps * a, prob, "lu", weights=w)[1]
           - inverse.forward_model(m - eps * a, prob, "lu", weights=w)[1]) / (2 * eps)
    assert np.allclose(ja, dfd, rtol=1e-6, atol=1e-7 * np.abs(dfd).max())
    b = phantoms.complex_normal(ja.shape, 4)
    jhb = inverse.jac_adjoint(b, ref["fields"], rf, prob)
    assert np.isclose(np.vdot(ja, b), np.vdot(a, jhb), rtol=1e-12)
    # the gradient is J^H r with the strict (current) receiver fields
    assert np.allclose(inverse.jac_adjoint(ref["resid"], ref["fields"], rf, prob),
                       ref["grad"], rtol=1e-9, atol=1e-12 * np.abs(ref["grad"]).max())


def test_hybrid_born_refresh_schedule():
    prob, m_true = make(n_elem=4, freqs=(2e6,))
    w = model.plane_wave_weights(prob, ANGLES[:3])
    _, d = inverse.forward_model(m_true, prob, "lu", weights=w)
    m0 = np.zeros(prob.shape, dtype=np.complex128)
    scale = float(np.abs(inverse.gradient(m0, d, prob, "lu", weights=w)["grad"]).max())
    p = admm.AdmmParams(lam=1e-3 * scale, rho=0.5 * scale, gamma=1e-3 * scale, n_cg=6)
    strict = admm.reconstruct(m0, d, prob, p, 2, "lu", weights=w, refresh_every=1)
    hybrid = admm.reconstruct(m0, d, prob, p, 2, "lu", weights=w, refresh_every=2)
    assert [r for _, r in strict[4]] == [True, True]
    assert [r for _, r in hybrid[4]] == [True, False]
    # iteration 0 is the same; iteration 1 reuses the receiver fields of m0
    m1, g1, u1, _, _ = admm.reconstruct(m0, d, prob, p, 1, "lu", weights=w)
    ref1 = inverse.gradient(m1, d, prob, "lu", weights=w)
    rf0 = inverse.receiver_fields(m0, prob, "lu")
    rf1 = inverse.receiver_fields(m1, prob, "lu")
    exp_h = admm.admm_tv_step(m1, g1, u1, ref1["grad"], ref1["fields"], rf0, prob, p)
    exp_s = admm.admm_tv_step(m1, g1, u1, ref1["grad"], ref1["fields"], rf1, prob, p)
    assert np.allclose(hybrid[0], exp_h[0], rtol=1e-12, atol=1e-15)
    assert np.allclose(strict[0], exp_s[0], rtol=1e-12, atol=1e-15)
    assert not np.allclose(hybrid[0], strict[0], rtol=1e-9, atol=0)
    # the misfit decreases over the two strict iterations
    assert strict[4][1][0] < strict[4][0][0]
