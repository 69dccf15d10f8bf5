"""Serving runtime (continuous batching of whole reconstructions) through the
C ABI: every request's result is the same alone and in a concurrent mix,
a one-iteration request matches the oracle's Algorithm-1 iteration, and
admission respects the HBM budget."""
import numpy as np
import pytest

from gpu_common import oracle_problem, rel_l2, small_workload
from oracle import admm, inverse, model
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


_CACHE = {}


def _requests():
    """Small reconstructions: observed data = oracle forward data of the
    phantom; start = half the phantom's SoS perturbation; ADMM weights
    scaled to the oracle gradient at the start."""
    if "reqs" in _CACHE:
        return _CACHE["reqs"]
    specs = [((32, 32), 6, (1.5e6, 3.0e6), 1), ((64, 64), 8, (1.0e6, 2.0e6, 3.0e6), 2),
             ((16, 64), 5, (2.0e6,), 3), ((8, 8, 16), 4, (1.0e6, 2.0e6), 4),
             ((32, 32), 4, (2.5e6,), 5)]
    reqs = []
    for shape, ne, freqs, seed in specs:
        w = small_workload(shape, n_elem=ne, freqs=freqs, seed=seed)
        prob = oracle_problem(w)
        sos0 = np.full(w.shape, w.c0) + 0.5 * (w.sos - w.c0)
        _, d = inverse.forward_model(model.contrast_from_sos(w.sos, w.c0), prob, "bicgstab",
                                     tol=1e-12)
        g = inverse.gradient(model.contrast_from_sos(sos0, w.c0), d, prob, "bicgstab",
                             tol=1e-10)["grad"]
        sc = float(np.abs(g).max())
        params = dict(n_iter=2, lam=1e-3 * sc, rho=0.5 * sc, gamma=1e-3 * sc, n_cg=4)
        reqs.append((w, sos0, d.astype(np.complex64), params))
    _CACHE["reqs"] = reqs
    return reqs


def test_results_are_the_same_alone_and_in_the_mix(lib):
    reqs = _requests()
    alone = []
    srv = lib.Server(max_active=1)
    for w, sos0, d, prm in reqs:
        rid = srv.submit(w.shape, w.h, w.c0, w.elem, w.freqs, sos0, d, **prm)
        alone.append(srv.wait(rid)[0])
    srv.close()
    srv = lib.Server(max_active=4)
    ids = [srv.submit(w.shape, w.h, w.c0, w.elem, w.freqs, sos0, d, **prm)
           for w, sos0, d, prm in reqs]
    mix = [srv.wait(i) for i in ids]
    srv.close()
    for a, (b, res) in zip(alone, mix):
        assert res["status"] == 0
        assert np.all(np.isfinite(b))
        assert rel_l2(b, a) < 1e-12  # bitwise in practice: independent contexts
        assert res["rhs_solves"] > 0 and res["latency_ms"] >= res["run_ms"]


@pytest.mark.parametrize("fp64", [False, True])
def test_one_iteration_matches_the_oracle(lib, fp64):
    """The batched FP32 request path, and the plain unbatched FP64 one
    (complex128 fields, one right-hand side per Krylov launch) that the
    serving benchmark compares against."""
    w = small_workload((32, 32), n_elem=6, freqs=(1.5e6, 3.0e6), seed=8)
    prob = oracle_problem(w)
    sos0 = np.full(w.shape, w.c0) + 0.5 * (w.sos - w.c0)
    m0 = model.contrast_from_sos(sos0, w.c0)
    m_true = model.contrast_from_sos(w.sos, w.c0)
    fields_t, d_true = inverse.forward_model(m_true, prob, "lu")
    d = d_true.astype(np.complex64)
    ref = inverse.gradient(m0, d.astype(np.complex128), prob, "bicgstab", tol=1e-12)
    scale = float(np.abs(ref["grad"]).max())
    p = admm.AdmmParams(lam=1e-3 * scale, rho=0.5 * scale, gamma=1e-3 * scale, n_cg=6)
    kk = (2 * np.pi * np.asarray(w.freqs) / w.c0) ** 2 * w.h ** 2
    rf = ref["fields"] * kk[:, None, None, None]
    g0 = admm.grad_op(m0, w.shape)
    _, _, _, sos1, _ = admm.admm_tv_step(m0, g0, np.zeros_like(g0), ref["grad"], ref["fields"],
                                         rf, prob, p)
    srv = lib.Server(max_active=2)
    extra = dict(precision=lib.FWI_FP64, max_batch=1, tol=1e-12) if fp64 else {}
    rid = srv.submit(w.shape, w.h, w.c0, w.elem, w.freqs, sos0, d, n_iter=1, lam=p.lam,
                     rho=p.rho, gamma=p.gamma, n_cg=p.n_cg, **extra)
    sos, res = srv.wait(rid)
    srv.close()
    tol = 1e-8 if fp64 else 1e-3
    assert res["status"] == 0
    assert rel_l2(sos - sos0, sos1 - sos0) < tol
    assert abs(res["misfit_first"] - ref["misfit"]) <= tol * ref["misfit"]


def test_admission_respects_the_budget(lib):
    reqs = _requests()[:3]
    import ctypes
    from paper_2604_15796_gb300.libfwi import FwiError
    sizes = []
    for w, _, _, _ in reqs:
        desc, keep = lib.make_desc(w.shape, w.h, w.c0, w.elem, w.freqs)
        sizes.append(int(lib.fwi_workspace_bytes(ctypes.byref(desc))))
        del keep
    big = max(sizes)
    budget = int(1.6 * big) + (8 << 20)
    srv = lib.Server(hbm_budget=budget, max_active=3)
    ids = [srv.submit(w.shape, w.h, w.c0, w.elem, w.freqs, sos0, d, **prm)
           for w, sos0, d, prm in reqs]
    for i in ids:
        _, res = srv.wait(i)
        assert res["status"] == 0 and res["bytes"] <= budget
    w, sos0, d, prm = _requests()[1]
    small = lib.Server(hbm_budget=1 << 20, max_active=1)
    with pytest.raises(FwiError) as e:
        small.submit(w.shape, w.h, w.c0, w.elem, w.freqs, sos0, d, **prm)
    assert e.value.status == lib.FWI_ERR_NOMEM
    small.close()
    srv.close()


def test_cancelled_requests(lib):
    """A queued request cancelled leaves at once; a running one stops at its
    next check; the request behind them runs as if alone."""
    import time
    reqs = _requests()
    w1, s1, d1, p1 = reqs[1]
    w0, s0, d0, p0 = reqs[0]
    w2, s2, d2, p2 = reqs[2]
    alone = lib.Server(max_active=1)
    ref, _ = alone.wait(alone.submit(w2.shape, w2.h, w2.c0, w2.elem, w2.freqs, s2, d2, **p2))
    alone.close()
    srv = lib.Server(max_active=1)
    # a: far more iterations than the test waits for (a few ms each)
    a = srv.submit(w1.shape, w1.h, w1.c0, w1.elem, w1.freqs, s1, d1, **dict(p1, n_iter=20000))
    b = srv.submit(w0.shape, w0.h, w0.c0, w0.elem, w0.freqs, s0, d0, **p0)
    c = srv.submit(w2.shape, w2.h, w2.c0, w2.elem, w2.freqs, s2, d2, **p2)
    srv.cancel(b)                       # queued behind a
    t0 = time.perf_counter()
    while srv.stats()[0] == 0 and time.perf_counter() - t0 < 30.0:
        time.sleep(0.01)                # until a is admitted
    time.sleep(0.3)
    srv.cancel(a)                       # running
    sa, ra = srv.wait(a)
    sb, rb = srv.wait(b)
    sc, rc = srv.wait(c)
    srv.close()
    assert rb["status"] == lib.FWI_ERR_CANCELLED and sb is None and rb["run_ms"] == 0.0
    assert ra["status"] == lib.FWI_ERR_CANCELLED and sa is None
    assert ra["run_ms"] < 60e3
    assert rc["status"] == 0 and rel_l2(sc, ref) < 1e-12
