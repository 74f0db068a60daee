"""Phase II rank growth on the GPU against the oracle.

The instance is the 770-vertex graph of the 512-graph batch (seeded Erdos-Renyi, unit
weights).  At the initial rank ceil(log2 m) = 10 both sides reach a point whose primal
infeasibility and gap pass at 1e-6 while lambda_min(C - A^T y) stays negative: the rank-10
problem is stationary there but the SDP is not solved.  Pins: that point's lambda_min from a
dense eigensolver is clearly negative (no growth allowed); with growth both sides raise the
rank once (10 -> 15) and converge; the objectives agree and the dense certificate passes."""
import numpy as np
import pytest

from oracle import SDP, Params, solve
from oracle.certify import min_eig_dual_slack
from paper_2403_09133_gb300 import instances as I
from paper_2403_09133_gb300 import lorads as L

pytestmark = pytest.mark.gpu


def _instance():
    return [x for x in I.workload_batch() if x.n == 770][0]


def test_stall_without_growth(cuda):
    inst = _instance()
    sdp = SDP.from_instance(inst)
    p = L.Problem(inst)
    res = p.solve(escape_scale=0.0, max_admm_iter=2000)
    sol = p.solution()
    p.close()
    assert res["status"] == L.LORADS_ERR_MAXITER and res["rank"] == 10
    assert res["r_P"] <= 1e-6 and abs(res["gap"]) <= 1e-6
    lmin = min_eig_dual_slack(sdp, sol["y"])
    assert max(0.0, -lmin) / (1.0 + sdp.C_rowsum_max) > 1e-6
    assert abs(res["lambda_min"] - lmin) <= 1e-7 + 1e-2 * abs(lmin)


@pytest.mark.parametrize("prec", [L.LORADS_PREC_FP64, L.LORADS_PREC_MIXED])
def test_growth_matches_oracle(cuda, prec):
    inst = _instance()
    sdp = SDP.from_instance(inst)
    ref = solve(sdp, Params())
    p = L.Problem(inst)
    res = p.solve(precision=prec)
    sol = p.solution()
    p.close()
    assert ref["converged"] and ref["rank"] == 15 and ref["growths"] == 1
    assert res["status"] == 0 and res["rank"] == 15 and res["rank_growths"] == 1
    assert abs(res["objective"] - ref["objective"]) <= 1e-6 * abs(ref["objective"])
    lmin = min_eig_dual_slack(sdp, sol["y"])
    assert max(0.0, -lmin) / (1.0 + sdp.C_rowsum_max) <= 1e-6


@pytest.mark.parametrize("which", ["er770", "torus141"])
def test_kept_lanczos_blocks_match_second_pass(cuda, which):
    """The escape's eigenvector from the first pass's kept blocks (the default when the state
    has room) against the second pass of the recurrence (lanczos_store_mb = 0): the same vector
    up to the rounding order, so the same growths and rank, the same objective to rounding, and
    no second-pass steps where the blocks are kept."""
    inst = _instance() if which == "er770" else I.workload_torus141()
    p = L.Problem(inst)
    kept = p.solve(precision=L.LORADS_PREC_MIXED)
    again = p.solve(precision=L.LORADS_PREC_MIXED, lanczos_store_mb=0)
    p.close()
    assert kept["status"] == 0 and again["status"] == 0
    assert kept["rank"] == again["rank"] and kept["rank_growths"] == again["rank_growths"] >= 1
    assert abs(kept["objective"] - again["objective"]) <= 1e-9 * abs(again["objective"])
    assert kept["r_D"] <= 1e-6 and kept["dual_psd"] <= 1e-6
    assert kept["lanczos_steps"] < again["lanczos_steps"]
