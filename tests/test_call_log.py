"""The binding's JSON-lines call log: one record per call with its status,
times and per-solve Krylov summary (a stand-in context, no GPU)."""
import io
import json

from paper_2604_15796_gb300 import libfwi


class _Ctx:
    shape = (32, 48)
    n_rhs = 12


def test_call_log_records():
    buf = io.StringIO()
    libfwi.set_call_log(buf)
    try:
        rep = libfwi.SolveReport(12)
        rep.info.max_iters, rep.info.n_not_converged, rep.info.device_ms = 5, 1, 2.5
        libfwi._log_call("gradient", _Ctx(), libfwi.FWI_OK, 0.004, forward=rep, adjoint=rep)
        libfwi._log_call("forward", _Ctx(), libfwi.FWI_ERR_CANCELLED, 0.001, forward=rep)
    finally:
        libfwi.set_call_log(None)
    libfwi._log_call("forward", _Ctx(), libfwi.FWI_OK, 0.001)  # logging off: nothing
    recs = [json.loads(line) for line in buf.getvalue().splitlines()]
    assert len(recs) == 2
    assert recs[0]["call"] == "gradient" and recs[0]["status"] == "OK"
    assert recs[0]["grid"] == [32, 48] and recs[0]["n_rhs"] == 12
    assert abs(recs[0]["wall_ms"] - 4.0) < 1e-9
    assert recs[0]["adjoint"]["max_iters"] == 5 and recs[0]["forward"]["not_converged"] == 1
    assert abs(recs[0]["forward"]["device_ms"] - 2.5) < 1e-6
    assert recs[1]["status"] == "CANCELLED"
