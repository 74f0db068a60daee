"""The Phase II per-iteration log (lorads_params.iter_log): one row per ADMM iteration with the
iteration number, rho, the primal infeasibility of U V^T and of U_hat U_hat^T, the CG
iterations so far and the device time.  It agrees with the solve's own totals, follows the
penalty schedule of Section 5.1, stops at its cap, and, from the oracle's own Phase I output,
repeats the oracle's per-iteration trace (the residuals the paper's Table 3 statistics come
from)."""
import numpy as np
import pytest

from oracle import SDP, Params
import oracle.lorads as OL
from paper_2403_09133_gb300 import instances as I
from paper_2403_09133_gb300 import lorads as L

pytestmark = pytest.mark.gpu


def _solve_logged(torch, inst, cap, **kw):
    log = torch.full((cap, 6), float("nan"), dtype=torch.float64, device="cuda")
    p = L.Problem(inst)
    res = p.solve(iter_log=log.data_ptr(), iter_log_cap=cap, **kw)
    p.close()
    torch.cuda.synchronize()
    return res, log.cpu().numpy()


@pytest.mark.parametrize("case", ["er200", "mc60"])
@pytest.mark.parametrize("prec", [L.LORADS_PREC_FP64, L.LORADS_PREC_MIXED])
def test_log_matches_totals_and_schedule(cuda, case, prec):
    torch = cuda
    inst = (I.maxcut_er(200, 6.0, seed=5) if case == "er200"
            else I.matrix_completion(30, 30, 3, 500, seed=2))
    res, log = _solve_logged(torch, inst, 8000, precision=prec)
    k = res["admm_iters"]
    assert res["status"] == 0 and k > 5
    rows = log[:k]
    assert np.isfinite(rows).all() and np.isnan(log[k:]).all()
    np.testing.assert_array_equal(rows[:, 0], np.arange(1, k + 1))
    assert rows[-1, 4] == res["cg_iters"]
    assert np.all(np.diff(rows[:, 4]) >= 0) and np.all(np.diff(rows[:, 5]) >= 0)
    # rho grows by 1.2 after every 5th iteration up to 5000 (Section 5.1)
    want = np.minimum(rows[0, 1] * 1.2 ** (np.arange(k) // 5), 5000.0)
    np.testing.assert_allclose(rows[:, 1], want, rtol=1e-10)
    # the solve ends where the output's primal test passes
    assert rows[-1, 3] <= 1e-6


def test_log_stops_at_its_cap(cuda):
    torch = cuda
    res, log = _solve_logged(torch, I.maxcut_er(200, 6.0, seed=5), 10)
    assert res["admm_iters"] > 10
    assert np.isfinite(log).all()
    np.testing.assert_array_equal(log[:, 0], np.arange(1, 11))


def test_log_follows_the_oracle_trace(cuda):
    """FP64, both from the oracle's Phase I output: per-iteration rho equal, r_P of U V^T and of
    U_hat U_hat^T within 1e-6 relative over the first 40 iterations (rounding only)."""
    torch = cuda
    inst = I.maxcut_er(200, 6.0, seed=5)
    sdp = SDP.from_instance(inst)
    prm = OL.resolve_auto(sdp, Params())
    ph1 = OL.lralm(sdp, OL.initial_factor(sdp, OL.initial_rank(sdp.m, sdp.n, prm), prm.seed), prm)
    rho0 = min(prm.h * ph1["sigma"], prm.rho_max)
    trace = []
    OL.lradmm(sdp, ph1["U"], ph1["U"], ph1["lam"], rho0, prm, trace)
    cap = 40
    log = torch.full((cap, 6), float("nan"), dtype=torch.float64, device="cuda")
    p = L.Problem(inst)
    assert L.lorads_set_start(p.handle, ph1["U"], ph1["lam"], rho0) == 0
    res = p.solve(phase1=0, precision=L.LORADS_PREC_FP64, iter_log=log.data_ptr(),
                  iter_log_cap=cap)
    p.close()
    torch.cuda.synchronize()
    got = log.cpu().numpy()
    n = min(cap, len(trace), res["admm_iters"])
    assert n >= 20
    want_rho = np.array([t["rho"] for t in trace[:n]])
    want_rp = np.array([t["rp"] for t in trace[:n]])
    want_rph = np.array([t["rp_hat"] for t in trace[:n]])
    np.testing.assert_allclose(got[:n, 1], want_rho, rtol=1e-12)
    np.testing.assert_allclose(got[:n, 2], want_rp, rtol=1e-6)
    np.testing.assert_allclose(got[:n, 3], want_rph, rtol=1e-6)
