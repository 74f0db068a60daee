"""GPU solves (Algorithm 2 in one persistent launch) against the oracle, closed forms and
certificates.

Pins: the MaxCut SDP value of K_n (n^2/4) and of unit tori (n lambda_max(L)/4); the
oracle's own solve of the same seeded instance with the same seed; lambda_min(C - A^T y)
and the duality gap computed by the oracle from the GPU's y; matrix completion's 2||M||_*.
The iterates of two runs need not agree (the method is nonconvex and reductions differ in
order), so objectives are compared to the accuracy the stopping rule implies."""
import math

import numpy as np
import pytest

from oracle import SDP, Params, solve
from oracle.certify import min_eig_dual_slack
from paper_2403_09133_gb300 import instances as I
from paper_2403_09133_gb300 import lorads as L

pytestmark = pytest.mark.gpu


def lam_max_cycle(k):
    return 4.0 if k % 2 == 0 else 2.0 + 2.0 * math.cos(math.pi / k)


def gpu_solve(inst, **kw):
    p = L.Problem(inst)
    res = p.solve(**kw)
    sol = p.solution() if res["status"] in (0, L.LORADS_ERR_MAXITER) else None
    p.close()
    return res, sol


@pytest.mark.parametrize("prec", [L.LORADS_PREC_FP64, L.LORADS_PREC_MIXED])
def test_complete_graph(cuda, prec):
    n = 12
    res, sol = gpu_solve(I.maxcut_complete(n), precision=prec, tol=1e-9, max_admm_iter=3000)
    assert res["status"] in (0, L.LORADS_ERR_MAXITER)
    assert abs(res["objective"] + n * n / 4) <= 1e-7 * n * n / 4
    np.testing.assert_allclose(sol["y"], -n / 4, atol=1e-5 * n)


@pytest.mark.parametrize("prec", [L.LORADS_PREC_FP64, L.LORADS_PREC_MIXED])
def test_unit_torus(cuda, prec):
    a, b = 6, 8
    res, sol = gpu_solve(I.maxcut_torus(a, b, seed=None), precision=prec, tol=1e-9,
                         max_admm_iter=3000)
    want = a * b * (lam_max_cycle(a) + lam_max_cycle(b)) / 4
    assert abs(-res["objective"] - want) <= 1e-7 * want


@pytest.mark.parametrize("prec", [L.LORADS_PREC_FP64, L.LORADS_PREC_MIXED])
def test_er500_against_oracle(cuda, prec):
    inst = I.workload_er500()
    sdp = SDP.from_instance(inst)
    ref = solve(sdp, Params())
    res, sol = gpu_solve(inst, precision=prec)
    assert res["status"] == 0, L.lorads_status_string(res["status"])
    # the final test: r_P, the Appendix B gap, the stationarity r_D and the dual measure
    assert res["r_P"] <= 1e-6 and abs(res["gap"]) <= 1e-6 and res["r_D"] <= 1e-6
    assert res["dual_psd"] <= 1e-6
    assert ref["converged"] and ref["r_P"] <= 1e-6 and abs(ref["gap"]) <= 1e-6
    assert ref["r_D"] <= 1e-6 and ref["dual_psd"] <= 1e-6
    # both hand the same Phase II iterate to the Newton refinement (Phase III)
    assert res["polished"] == 1 and ref["polished"]
    assert abs(res["admm_iters"] - ref["admm_iters"]) <= 2
    assert abs(res["newton_steps"] - ref["newton_steps"]) <= 2
    assert abs(res["objective"] - ref["objective"]) <= 1e-6 * abs(ref["objective"])
    # the library's own residual report agrees with the oracle's evaluation of its output
    rep = OLkkt(sdp, sol)
    assert abs(rep["objective"] - res["objective"]) <= 1e-10 * abs(res["objective"])
    assert abs(rep["r_P"] - res["r_P"]) <= 1e-9
    assert abs(rep["r_D"] - res["r_D"]) <= 1e-6 * max(rep["r_D"], 1e-12) + 1e-12
    assert abs(rep["gap"] - res["gap"]) <= 1e-10
    # the Lanczos estimate of lambda_min(C - A^T y) against a dense eigensolver
    lmin = min_eig_dual_slack(sdp, sol["y"])
    assert abs(res["lambda_min"] - lmin) <= 1e-7 + 1e-2 * abs(lmin), (res["lambda_min"], lmin)
    assert abs(res["p_infeas"] - np.linalg.norm(sdp.A_of(sol["U_hat"], sol["U_hat"]) - sdp.b)
               / (1.0 + sdp.b_one)) <= 1e-12


def OLkkt(sdp, sol):
    from oracle.lorads import kkt_report
    return kkt_report(sdp, sol["U_hat"], sol["y"])


def test_grid_scope_matches_block_scope(cuda):
    inst = I.workload_er500()
    rb, _ = gpu_solve(inst, grid=1)
    rg, _ = gpu_solve(inst, grid=16)
    assert rb["status"] == 0 and rg["status"] == 0
    assert abs(rb["objective"] - rg["objective"]) <= 1e-6 * abs(rb["objective"])


def test_deterministic(cuda):
    inst = I.maxcut_er(300, 6.0, seed=3)
    r1, s1 = gpu_solve(inst, grid=8)
    r2, s2 = gpu_solve(inst, grid=8)
    assert r1["objective"] == r2["objective"]
    assert np.array_equal(s1["U_hat"], s2["U_hat"])


def test_matrix_completion_small(cuda):
    inst = I.matrix_completion(30, 30, 2, 500, seed=3)
    res, sol = gpu_solve(inst, switch_tol=1e-3, h=5.0, tol=1e-9, max_admm_iter=3000)
    want = 2.0 * np.linalg.svd(inst.mc_P @ inst.mc_Q.T, compute_uv=False).sum()
    assert abs(res["objective"] - want) <= 1e-7 * want
    # the one-CTA solve of a general (non-diagonal) problem is deterministic
    again, _ = gpu_solve(inst, switch_tol=1e-3, h=5.0, tol=1e-9, max_admm_iter=3000)
    assert again["objective"] == res["objective"] and again["admm_iters"] == res["admm_iters"]


def test_status_codes(cuda):
    inst = I.maxcut_er(100, 5.0, seed=1)
    res, _ = gpu_solve(inst, max_admm_iter=2)
    assert res["status"] == L.LORADS_ERR_MAXITER


def test_phase2_start_from_caller(cuda):
    """phase1 = 0 starts Algorithm 1 from a caller-supplied (U_0, lambda_0, rho_0); here the
    oracle's own Phase I output, so both sides then run the same Phase II."""
    import oracle.lorads as OL
    inst = I.maxcut_er(60, 6.0, seed=11)
    sdp = SDP.from_instance(inst)
    prm = OL.resolve_auto(sdp, Params())
    U_init = OL.initial_factor(sdp, OL.initial_rank(sdp.m, sdp.n, prm), prm.seed)
    ph1 = OL.lralm(sdp, U_init, prm)
    rho0 = min(prm.h * ph1["sigma"], prm.rho_max)
    p = L.Problem(inst)
    assert L.lorads_set_start(p.handle, ph1["U"], ph1["lam"], rho0) == 0
    res = p.solve(phase1=0)
    p.close()
    ref = solve(sdp, Params(phase1=False), U0=ph1["U"], lam0=ph1["lam"], rho0=rho0)
    assert res["status"] == 0 and ref["converged"]
    assert abs(res["admm_iters"] - ref["admm_iters"]) <= 2
    assert abs(res["objective"] - ref["objective"]) <= 1e-7 * abs(ref["objective"])


@pytest.mark.parametrize("prec", [L.LORADS_PREC_FP64, L.LORADS_PREC_MIXED])
def test_rank_growth_matches_oracle(cuda, prec):
    """Section 4.3's dynamic rank: with an inner cap of 3 L-BFGS iterations every ALM
    subproblem stalls, so the rank grows by 1.5x (rounded up) until the cap floor(sqrt(2m)):
    n = m = 100, r0 = ceil(log2 100) = 7 -> 11 -> 14 (cap), two growths on both sides."""
    inst = I.maxcut_er(100, 6.0, seed=3)
    sdp = SDP.from_instance(inst)
    ref = solve(sdp, Params(inner_max_iter=3))
    res, sol = gpu_solve(inst, precision=prec, inner_max_iter=3)
    assert ref["rank"] == 14 and ref["growths"] == 2
    assert res["rank"] == ref["rank"] and res["rank_growths"] == ref["growths"]
    assert sol["U_hat"].shape == (100, 14)
    assert res["status"] == 0 and ref["converged"]
    assert abs(res["objective"] - ref["objective"]) <= 1e-6 * abs(ref["objective"])


def test_matrix_completion_grid_scope_both_forms(cuda):
    """n = 1,000 (the whole-GPU scope) on the general path: both forms pass the final test,
    agree on the objective, and the FP64 form is deterministic."""
    inst = I.matrix_completion(500, 500, 3, 60000, seed=4)
    r64, _ = gpu_solve(inst, precision=L.LORADS_PREC_FP64)
    r32, _ = gpu_solve(inst, precision=L.LORADS_PREC_MIXED)
    again, _ = gpu_solve(inst, precision=L.LORADS_PREC_FP64)
    assert r64["status"] == 0 and r32["status"] == 0
    assert abs(r64["objective"] - r32["objective"]) <= 1e-5 * abs(r64["objective"])
    assert again["objective"] == r64["objective"] and again["admm_iters"] == r64["admm_iters"]


@pytest.mark.parametrize("prec", [L.LORADS_PREC_FP64, L.LORADS_PREC_MIXED])
def test_row_direct_against_oracle(cuda, prec):
    """The exact row-block subproblem solve (subsolver 1) on ER n = 500 against the oracle's
    own row_direct solve: both pass the final test; the FP64 form follows the oracle's
    trajectory (same iteration count within 2, objective to 1e-9)."""
    inst = I.workload_er500()
    sdp = SDP.from_instance(inst)
    ref = solve(sdp, Params(subsolver="row_direct"))
    res, sol = gpu_solve(inst, precision=prec, subsolver=L.LORADS_SUB_ROW_DIRECT)
    assert ref["converged"] and ref["cg_iters"] == 0
    assert res["status"] == 0, L.lorads_status_string(res["status"])
    assert res["cg_iters"] == 0
    assert res["r_P"] <= 1e-6 and abs(res["gap"]) <= 1e-6 and res["r_D"] <= 1e-6
    assert res["dual_psd"] <= 1e-6
    if prec == L.LORADS_PREC_FP64:
        assert abs(res["admm_iters"] - ref["admm_iters"]) <= 2
        assert abs(res["objective"] - ref["objective"]) <= 1e-9 * abs(ref["objective"])
    else:
        assert abs(res["objective"] - ref["objective"]) <= 1e-6 * abs(ref["objective"])
    lmin = min_eig_dual_slack(sdp, sol["y"])
    assert max(0.0, -lmin) / (1.0 + sdp.C_rowsum_max) <= 1e-6


@pytest.mark.parametrize("prec", [L.LORADS_PREC_FP64, L.LORADS_PREC_MIXED])
def test_row_direct_closed_forms(cuda, prec):
    n = 12
    res, _ = gpu_solve(I.maxcut_complete(n), precision=prec, tol=1e-9, max_admm_iter=3000,
                       subsolver=L.LORADS_SUB_ROW_DIRECT)
    assert abs(res["objective"] + n * n / 4) <= 1e-7 * n * n / 4
    a, b = 6, 8
    res, _ = gpu_solve(I.maxcut_torus(a, b, seed=None), precision=prec, tol=1e-9,
                       max_admm_iter=3000, subsolver=L.LORADS_SUB_ROW_DIRECT)
    want = a * b * (lam_max_cycle(a) + lam_max_cycle(b)) / 4
    assert abs(-res["objective"] - want) <= 1e-7 * want


def test_row_direct_grid_scope_against_oracle(cuda):
    """40 x 40 signed torus (grid scope, 152 CTAs): FP64 direct solve against the oracle's."""
    inst = I.maxcut_torus(40, 40, seed=2)
    sdp = SDP.from_instance(inst)
    ref = solve(sdp, Params(subsolver="row_direct"))
    res, _ = gpu_solve(inst, precision=L.LORADS_PREC_FP64, subsolver=L.LORADS_SUB_ROW_DIRECT)
    assert ref["converged"] and res["status"] == 0
    assert abs(res["admm_iters"] - ref["admm_iters"]) <= 2
    assert abs(res["objective"] - ref["objective"]) <= 1e-9 * abs(ref["objective"])


def test_row_direct_statuses(cuda):
    # not row-separable: matrix completion's off-diagonal constraints
    res, _ = gpu_solve(I.matrix_completion(10, 10, 2, 40, seed=1),
                       subsolver=L.LORADS_SUB_ROW_DIRECT)
    assert res["status"] == L.LORADS_ERR_UNSUPPORTED
    res, _ = gpu_solve(I.maxcut_er(50, 4.0, seed=1), subsolver=2)
    assert res["status"] == L.LORADS_ERR_ARG
    # batches take it too: every problem row-separable
    insts = [I.maxcut_er(n, 6.0, seed=90 + n) for n in (80, 200, 330)]
    hs = [L.Problem(x) for x in insts]
    prm = hs[0].params(subsolver=L.LORADS_SUB_ROW_DIRECT, threads=256, team_mult=1)
    out, _, _ = L.lorads_solve_batch([h.handle for h in hs], prm)
    for h, x, r in zip(hs, insts, out):
        one = h.solve(subsolver=L.LORADS_SUB_ROW_DIRECT, grid=1, threads=256)
        assert r["status"] == 0 and r["cg_iters"] == 0
        assert r["objective"] == one["objective"] and r["admm_iters"] == one["admm_iters"]
        h.close()


@pytest.mark.parametrize("prec", [L.LORADS_PREC_FP64, L.LORADS_PREC_MIXED])
def test_general_path_scopes_agree(cuda, prec):
    """Off-diagonal constraints (matrix completion) on one CTA and on two CTAs of the grid scope:
    the first three ADMM iterations take the same CG iterations (within 3) and reach the same
    objective to what the reduction order changes, and the one-CTA solve repeats itself."""
    inst = I.matrix_completion(60, 60, 3, 1200, seed=4)
    p = L.Problem(inst)
    one = p.solve(precision=prec, max_admm_iter=3)
    again = p.solve(precision=prec, max_admm_iter=3)
    two = p.solve(precision=prec, max_admm_iter=3, grid=2)
    p.close()
    assert one["objective"] == again["objective"] and one["cg_iters"] == again["cg_iters"]
    assert abs(one["cg_iters"] - two["cg_iters"]) <= 3
    tol = 1e-9 if prec == L.LORADS_PREC_FP64 else 1e-6
    assert abs(one["objective"] - two["objective"]) <= tol * abs(two["objective"])


@pytest.fixture(scope="module")
def mc500_oracle():
    inst = I.matrix_completion(500, 500, 3, 20000, seed=7)
    sdp = SDP.from_instance(inst)
    return inst, sdp, solve(sdp, Params())


@pytest.mark.parametrize("prec", [L.LORADS_PREC_FP64, L.LORADS_PREC_MIXED])
def test_matrix_completion_against_oracle(cuda, mc500_oracle, prec):
    """Matrix completion (Section 5.4's SDP, n1 = n2 = 500, rank-3 M, 20,000 samples; off-diagonal
    constraints, so Phase III continues Phase I's augmented Lagrangian method) against the
    oracle's solve of the same instance: both pass the final test, both reach 2 ||M||_* (exact
    recovery), and the objectives agree to 1e-6."""
    inst, sdp, ref = mc500_oracle
    res, sol = gpu_solve(inst, precision=prec)
    want = 2.0 * np.linalg.svd(inst.mc_P @ inst.mc_Q.T, compute_uv=False).sum()
    assert ref["converged"] and res["status"] == 0, L.lorads_status_string(res["status"])
    assert res["polished"] == 2 and ref["polished"]
    assert res["r_P"] <= 1e-6 and res["r_D"] <= 1e-6 and abs(res["gap"]) <= 1e-6
    assert res["dual_psd"] <= 1e-6
    assert abs(res["objective"] - ref["objective"]) <= 1e-6 * abs(ref["objective"])
    assert abs(res["objective"] - want) <= 1e-6 * want
    assert abs(ref["objective"] - want) <= 1e-6 * want
    # the oracle's evaluation of the library's output agrees with the library's report
    from oracle.lorads import kkt_report
    rep = kkt_report(sdp, sol["U_hat"], sol["y"])
    assert rep["r_D"] <= 1e-6 and rep["r_P"] <= 1e-6
