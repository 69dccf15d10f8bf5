"""Several iterations of Algorithm 1 on the GPU against the oracle's, with
the strict distorted-Born Jacobian and with the hybrid Born schedule of
Sec. IV-B (receiver fields refreshed every K iterations, frozen in
between), through the C ABI:

* fwi_freeze_receiver_fields: after a snapshot at m1 and a forward solve
  at m2, J a and J^H y take p_e from the fields at m2 and ptilde_j from the
  fields at m1, as the oracle's jac_forward / jac_adjoint with those two
  field sets (FP32 on the tensor cores and on CUDA cores, and FP64);
* whole reconstructions through the server (n_iter = 3 with the strict
  Jacobian; n_iter = 4 with refresh_every = 3, so that iteration 3 uses the
  receiver fields of iteration 0) against oracle.admm.reconstruct, in FP32
  (SoS change at 1e-3) and FP64 (1e-8);
* the argument checks of the snapshot call."""
import numpy as np
import pytest

from gpu_common import contrast, oracle_problem, rel_l2, small_workload, to_gpu, to_np
from oracle import admm, inverse, model, operator
from paper_2604_15796_gb300 import phantoms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2604_15796_gb300 import build, libfwi
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return libfwi


@pytest.mark.parametrize("mode", ["tensor", "cuda_core", "fp64"])
def test_frozen_receiver_fields_in_the_jacobian(lib, mode):
    import torch
    w = small_workload((32, 32), n_elem=6, freqs=(1.5e6, 3.0e6), seed=12)
    prob = oracle_problem(w)
    m2 = contrast(w)
    m1 = 0.5 * m2
    fp64 = mode == "fp64"
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs, hybrid_born=True,
                      precision=lib.FWI_FP64 if fp64 else lib.FWI_MIXED,
                      tol=1e-12 if fp64 else 1e-6)
    if mode == "cuda_core":
        ctx.set_jac_tensor_cores(False)
    ctx.forward(to_gpu(m1, torch.complex128))
    ctx.freeze_receiver_fields(True)
    ctx.forward(to_gpu(m2, torch.complex128))
    a = phantoms.complex_normal(w.shape, 3)
    y = phantoms.complex_normal((w.n_freq, w.n_elem, w.n_elem), 4)
    ja = to_np(ctx.jac_forward(to_gpu(a, torch.complex128)))
    jhy = to_np(ctx.jac_adjoint(to_gpu(y, torch.complex128)))
    ctx.freeze_receiver_fields(False)
    ja_strict = to_np(ctx.jac_forward(to_gpu(a, torch.complex128)))
    ctx.close()
    p2 = operator.solve_forward(m2, prob, "lu")
    rf1 = inverse.receiver_fields(m1, prob, "lu")
    rf2 = inverse.receiver_fields(m2, prob, "lu")
    tol = 1e-9 if fp64 else 1e-4
    assert rel_l2(ja, inverse.jac_forward(a, p2, rf1, prob)) < tol
    assert rel_l2(jhy, inverse.jac_adjoint(y, p2, rf1, prob)) < tol
    assert rel_l2(ja_strict, inverse.jac_forward(a, p2, rf2, prob)) < tol
    # the snapshot changes the product: the test is not vacuous
    assert rel_l2(ja, ja_strict) > 1e-2


def test_receiver_snapshot_argument_checks(lib):
    import torch
    w = small_workload((16, 16), n_elem=2, freqs=(2e6,))
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs)
    with pytest.raises(lib.FwiError) as e:
        ctx.freeze_receiver_fields(True)  # no snapshot buffer
    assert e.value.status == lib.FWI_ERR_INVALID_ARG
    ctx.close()
    ctx = lib.Context(w.shape, w.h, w.c0, w.elem, w.freqs, hybrid_born=True)
    with pytest.raises(lib.FwiError) as e:
        ctx.freeze_receiver_fields(True)  # no forward fields yet
    assert e.value.status == lib.FWI_ERR_INVALID_ARG
    ctx.forward(to_gpu(contrast(w), torch.complex128))
    ctx.freeze_receiver_fields(True)
    ctx.freeze_receiver_fields(False)
    ctx.close()


def _reconstruction_case():
    w = small_workload((32, 32), n_elem=6, freqs=(1.5e6, 2.5e6), seed=21)
    prob = oracle_problem(w)
    sos0 = np.full(w.shape, w.c0) + 0.5 * (w.sos - w.c0)
    m0 = model.contrast_from_sos(sos0, w.c0)
    _, d_true = inverse.forward_model(model.contrast_from_sos(w.sos, w.c0), prob, "lu")
    d = d_true.astype(np.complex64)
    scale = float(np.abs(inverse.gradient(m0, d.astype(np.complex128), prob, "lu")["grad"]).max())
    p = admm.AdmmParams(lam=1e-3 * scale, rho=0.5 * scale, gamma=1e-3 * scale, n_cg=6)
    return w, prob, sos0, m0, d, p


@pytest.mark.parametrize("n_iter,refresh", [(3, 1), (4, 3)])
@pytest.mark.parametrize("fp64", [False, True])
def test_reconstruction_matches_oracle_algorithm_1(lib, n_iter, refresh, fp64):
    w, prob, sos0, m0, d, p = _reconstruction_case()
    _, _, _, sos_ref, hist = admm.reconstruct(m0, d.astype(np.complex128), prob, p, n_iter,
                                              "lu", refresh_every=refresh)
    assert [h[1] for h in hist] == [k % refresh == 0 for k in range(n_iter)]
    srv = lib.Server(max_active=1)
    extra = dict(precision=lib.FWI_FP64, tol=1e-12) if fp64 else {}
    rid = srv.submit(w.shape, w.h, w.c0, w.elem, w.freqs, sos0, d, n_iter=n_iter, lam=p.lam,
                     rho=p.rho, gamma=p.gamma, n_cg=p.n_cg, refresh_every=refresh, **extra)
    sos, res = srv.wait(rid)
    srv.close()
    assert res["status"] == 0
    tol = 1e-8 if fp64 else 1e-3
    assert rel_l2(sos - sos0, sos_ref - sos0) < tol, rel_l2(sos - sos0, sos_ref - sos0)
    assert abs(res["misfit_first"] - hist[0][0]) <= tol * hist[0][0]
    assert abs(res["misfit_last"] - hist[-1][0]) <= 10 * tol * hist[0][0]


def test_refresh_schedule_changes_the_reconstruction(lib):
    """The frozen receiver fields make a difference the tests above can see:
    four iterations with refresh_every = 3 differ from the strict Jacobian
    on the GPU as they do in the oracle."""
    w, prob, sos0, m0, d, p = _reconstruction_case()
    out = {}
    for refresh in (1, 3):
        srv = lib.Server(max_active=1)
        rid = srv.submit(w.shape, w.h, w.c0, w.elem, w.freqs, sos0, d, n_iter=4, lam=p.lam,
                         rho=p.rho, gamma=p.gamma, n_cg=p.n_cg, refresh_every=refresh,
                         precision=lib.FWI_FP64, tol=1e-12)
        out[refresh] = srv.wait(rid)[0]
        srv.close()
    assert rel_l2(out[3] - sos0, out[1] - sos0) > 1e-6
