"""Whole-solve pins for the oracle (Algorithm 2) against what the MaxCut and
matrix-completion SDPs fix in closed form, and against certificates.

MaxCut SDP (Section 5.3) in min form: min <-L/4, X>, X_jj = 1.
  * K_n, unit weights: value n^2/4; dual y = -(n/4) 1 (S = J/4 is PSD).
  * vertex-transitive graphs (cycles, tori), unit weights: value n lambda_max(L)/4 with a
    uniform dual; lambda_max(C_n) = 4 for even n, 2 + 2 cos(pi/n) for odd n; a torus adds
    the two cycles' values.
  * Goemans-Williamson: 0.878 SDP <= max cut <= SDP for nonnegative weights.
Matrix completion (Section 5.4): under exact recovery the optimum is 2 ||M||_*.
"""
import dataclasses
import math
import os

import numpy as np
import pytest

from oracle import SDP, Params, solve
import oracle.lorads as L
from oracle.certify import exhaustive_maxcut, min_eig_dual_slack
from paper_2403_09133_gb300 import instances as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TIGHT = dict(tol=1e-9, max_admm_iter=3000)


def lam_max_cycle(k):
    return 4.0 if k % 2 == 0 else 2.0 + 2.0 * math.cos(math.pi / k)


def _solve(inst, **kw):
    sdp = SDP.from_instance(inst)
    return sdp, solve(sdp, Params(**{**TIGHT, **kw}))


def _check_certificates(sdp, res, obj_tol=1e-7, dual_tol=1e-5):
    lmin = min_eig_dual_slack(sdp, res["y"])
    scale = 1.0 + sdp.C_rowsum_max
    assert lmin >= -dual_tol * scale, lmin
    assert abs(res["gap"]) <= dual_tol
    assert res["r_P"] <= 1e-8


@pytest.mark.parametrize("n", [8, 12])
def test_complete_graph_value_and_dual(n):
    sdp, res = _solve(I.maxcut_complete(n))
    assert abs(res["objective"] + n * n / 4) <= 1e-7 * n * n / 4
    np.testing.assert_allclose(res["y"], -n / 4 * np.ones(n), atol=1e-5 * n)
    _check_certificates(sdp, res)


@pytest.mark.parametrize("a,b", [(6, 8), (5, 7)])
def test_unit_torus_value(a, b):
    sdp, res = _solve(I.maxcut_torus(a, b, seed=None))
    want = a * b * (lam_max_cycle(a) + lam_max_cycle(b)) / 4
    assert abs(-res["objective"] - want) <= 1e-7 * want
    np.testing.assert_allclose(res["y"], -(lam_max_cycle(a) + lam_max_cycle(b)) / 4, atol=1e-4)
    _check_certificates(sdp, res)


def test_odd_cycle_value():
    n = 11
    sdp, res = _solve(I.maxcut_cycle(n))
    want = n * lam_max_cycle(n) / 4          # (n/2)(1 + cos(pi/n))
    assert abs(-res["objective"] - want) <= 1e-7 * want


def test_goemans_williamson_sandwich():
    rng = np.random.default_rng(7)
    e = I.erdos_renyi_edges(16, 40, rng)
    w = rng.uniform(0.5, 2.0, len(e))
    sdp, res = _solve(I.maxcut_sdp(16, e, w, "er16w"))
    sdp_value = -res["objective"]
    cut = exhaustive_maxcut(16, e, w)
    assert 0.878 * sdp_value <= cut <= sdp_value + 1e-9
    _check_certificates(sdp, res)


def test_matrix_completion_nuclear_norm():
    inst = I.matrix_completion(30, 30, 2, 500, seed=3)
    sdp, res = _solve(inst, switch_tol=1e-3, h=5.0)
    want = 2.0 * np.linalg.svd(inst.mc_P @ inst.mc_Q.T, compute_uv=False).sum()
    assert abs(res["objective"] - want) <= 1e-7 * want
    # the Z block of X = U_hat U_hat^T reproduces M away from the samples too
    Uh = res["U_hat"]
    Z = Uh[:30] @ Uh[30:].T
    M = inst.mc_P @ inst.mc_Q.T
    assert np.linalg.norm(Z - M) <= 1e-4 * np.linalg.norm(M)


def test_default_tolerance_reaches_kkt_on_er():
    """At the default tolerance (1e-6) the output is primal feasible and the objective agrees
    with a tight solve to the accuracy the stopping rule implies."""
    inst = I.maxcut_er(60, 6.0, seed=11)
    sdp = SDP.from_instance(inst)
    res = solve(sdp, Params())
    assert res["converged"] and res["r_P"] <= 1e-6
    tight = solve(sdp, Params(tol=1e-9, max_admm_iter=6000))
    assert abs(res["objective"] - tight["objective"]) <= 1e-5 * abs(tight["objective"])


def test_table2_rank_rule():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table2_ranks.txt"))
            if l.strip() and not l.startswith("#")]
    for name, n, m, r0, rsq, rfinal in rows:
        m, r0, rsq, rfinal = int(m), int(r0), int(rsq), int(rfinal)
        p = Params(rank_rule="paper", rank_max=10 ** 9)
        assert L.initial_rank(m, 10 ** 9, p) == r0, name
        assert int(round(math.sqrt(2 * m))) == rsq, name
        assert rfinal in L.paper_rank_sequence(m, 6), name


def test_splitmix64_known_answers():
    for line in open(os.path.join(GOLDEN, "splitmix64_kat.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        seed, idx, out = (int(x) for x in line.split())
        assert int(L.splitmix64_at(np.uint64(seed), np.uint64(idx))) == out


def test_box_muller_moments():
    z = L.normal_matrix(L.stream_key(3, 0), 20000, 5)
    assert abs(z.mean()) < 0.02 and abs(z.std() - 1.0) < 0.02
    assert abs(np.mean(z ** 4) - 3.0) < 0.1            # Gaussian kurtosis


def test_initial_factor_feasible_for_diagonal_constraints():
    sdp = SDP.from_instance(I.maxcut_er(50, 4.0, seed=2))
    U = L.initial_factor(sdp, 6, seed=9)
    np.testing.assert_allclose(np.sum(U * U, axis=1), 1.0, rtol=1e-14)


def test_rank_growth_on_a_stalled_instance():
    """At rank ceil(log2 m) = 10 the 770-vertex batch graph stalls with lambda_min(S) < 0;
    Phase III grows the rank along the eigenvector and the dense certificate then passes, at an
    objective below the stalled one (a larger feasible set can only lower the minimum).  The
    same growth inside Phase II (no Phase III) is covered by the resume test below."""
    inst = [x for x in I.workload_batch() if x.n == 770][0]
    sdp = SDP.from_instance(inst)
    stalled = solve(sdp, Params(escape_scale=0.0, max_admm_iter=600))
    grown = solve(sdp, Params())
    assert not stalled["converged"] and stalled["rank"] == 10
    assert stalled["dual_psd"] > 1e-6
    assert grown["converged"] and grown["rank"] > 10 and grown["growths"] >= 1
    lmin = min_eig_dual_slack(sdp, grown["y"])
    assert max(0.0, -lmin) / (1.0 + sdp.C_rowsum_max) <= 1e-6
    assert grown["r_D"] <= 1e-6 and grown["r_P"] <= 1e-6 and abs(grown["gap"]) <= 1e-6
    assert grown["objective"] < stalled["objective"] - 1e-3


def test_lradmm_resume_repeats_the_uninterrupted_run():
    """A checkpoint (U^k, V^k, lambda^k, rho, k and the final-test schedule) holds all that
    Algorithm 1 carries between iterations: continuing from one taken before the first failed
    dual-infeasibility test, between failed tests and after a Phase II rank growth repeats
    the uninterrupted run bit for bit.  Rank 2 on a 60-vertex graph stalls (a failed test at
    k = 409, a second at 987 that grows the rank to 3), so every part of the schedule is used;
    dropping the remembered dual infeasibility changes the run (the growth comes later)."""
    sdp = SDP.from_instance(I.maxcut_er(60, 6.0, seed=11))
    p = L.resolve_auto(sdp, Params(r0=2, rank_max=6, max_admm_iter=1500, polish="off"))
    ph1 = L.lralm(sdp, L.initial_factor(sdp, 2, p.seed), p)
    rho = min(p.h * ph1["sigma"], p.rho_max)
    full, conv = L.lradmm(sdp, ph1["U"], ph1["U"], ph1["lam"], rho, p)
    assert full.U.shape[1] == 3 and full.growths == 1 and not conv
    for k1 in (300, 700, 1200):
        part, _ = L.lradmm(sdp, ph1["U"], ph1["U"], ph1["lam"], rho,
                           dataclasses.replace(p, max_admm_iter=k1))
        assert part.k == k1
        res, conv_r = L.lradmm_resume(sdp, part, p)
        assert conv_r == conv and res.k == full.k and res.cg_iters == full.cg_iters
        assert res.rho == full.rho and res.growths == full.growths
        assert np.array_equal(res.U, full.U) and np.array_equal(res.V, full.V)
        assert np.array_equal(res.lam, full.lam)
        if k1 == 700:
            assert part.next_dual_test == 409 + 40 and part.prev_dinf is not None
            forgetful = dataclasses.replace(part, prev_dinf=None)
            trace: list = []
            L.lradmm_resume(sdp, forgetful, p, trace)
            grown_at = [i["k"] for i in trace if "grow_to" in i]
            assert grown_at and grown_at[0] > 987


def test_auto_parameters_by_problem_class():
    """The "auto" readings: Section 5.1's switch tolerance 1e-2 and h = 10 for MaxCut, 1e-3 for
    other problems (h = 1 and the gamma scale 1 / 2 are readings); explicit values are kept."""
    from oracle.lorads import resolve_auto, penalty_gamma
    mc = SDP.from_instance(I.maxcut_er(30, 4.0, seed=1))
    q = resolve_auto(mc, Params())
    assert (q.switch_tol, q.h, q.gamma_scale) == (1e-2, 10.0, 1.0)
    assert penalty_gamma(mc, Params()) == mc.C_rowsum_max
    comp = SDP.from_instance(I.matrix_completion(6, 5, 2, 12, seed=3))
    q = resolve_auto(comp, Params())
    assert (q.switch_tol, q.h, q.gamma_scale) == (1e-3, 1.0, 2.0)
    assert penalty_gamma(comp, Params()) == 2.0 * comp.C_rowsum_max
    q = resolve_auto(comp, Params(switch_tol=1e-4, h=2.5, gamma_scale=3.0))
    assert (q.switch_tol, q.h, q.gamma_scale) == (1e-4, 2.5, 3.0)
