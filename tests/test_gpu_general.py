"""General constraint structures on the device, through the C ABI, against the oracle:
multi-entry constraints (the Lovasz theta SDP's tr X = 1), rank-one constraints with long
vectors (the bisection relaxation's <e e^T, X> = 0; normalised Gaussian vectors added to a
MaxCut SDP) and rank-one constraints with short vectors (sensor network localisation,
Section 2.3).  Section 5.5's general benchmarks (SDPLIB theta and gpp) are these structures;
the instances are seeded stand-ins of that shape.

  * operators element by element against the oracle's definitions (FP64 1e-12, FP32 1e-5 of a
    bound that Cauchy-Schwarz gives for each output: the same products on absolute values);
  * whole solves against closed forms (theta(C_5) = sqrt 5, theta(Petersen) = 4, the bisection
    of C_12 and K_8) and against the oracle's solve of the same seeded instance (objective to
    1e-6 relative, the final test passing on both sides, the oracle's evaluation of the
    library's output passing it too);
  * one CTA against two CTAs of the whole-GPU scope, and a batch against single solves.
"""
import math

import numpy as np
import pytest

from oracle import SDP, Params, solve
import oracle.lorads as OL
from paper_2403_09133_gb300 import instances as I
from paper_2403_09133_gb300 import lorads as L

pytestmark = pytest.mark.gpu


def _er_edges(n, deg, seed):
    rng = np.random.default_rng(seed)
    return I.erdos_renyi_edges(n, int(n * deg / 2), rng)


def petersen_edges():
    outer = [(i, (i + 1) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    return np.array([tuple(sorted(e)) for e in outer + spokes + inner])


OPS = {
    "theta": lambda: I.lovasz_theta(60, _er_edges(60, 5.0, 3)),          # tr X: 2 chunks
    "bisection": lambda: I.graph_bisection(70, _er_edges(70, 4.0, 5), np.ones(140)),  # 2,485 entries
    "maxcut_r1": lambda: I.maxcut_rank_one(90, 5.0, 3, 60, seed=4),
    "snl": lambda: I.sensor_network(40, 5, 2, 0.45, seed=3),
}
RANKS = [1, 5, 12, 33]


def _abs_instance(inst):
    """The same instance with every value replaced by its absolute value."""
    out = I.SDPInstance(
        n=inst.n, m=inst.m, C_row=inst.C_row, C_col=inst.C_col, C_val=np.abs(inst.C_val),
        A_con=inst.A_con, A_row=inst.A_row, A_col=inst.A_col, A_val=np.abs(inst.A_val),
        b=inst.b, rank1=[(c, i, np.abs(a), abs(s)) for c, i, a, s in inst.rank1])
    return SDP.from_instance(out)


def _pad(X, ld):
    out = np.zeros((X.shape[0], ld))
    out[:, : X.shape[1]] = X
    return out


@pytest.fixture(scope="module")
def op_problems(cuda):
    out = {}
    for k, f in OPS.items():
        inst = f()
        out[k] = (inst, SDP.from_instance(inst), _abs_instance(inst), L.Problem(inst))
    yield out
    for *_, p in out.values():
        p.close()


def _dev(torch, X, ld, prec):
    dt = torch.float64 if prec == L.LORADS_PREC_FP64 else torch.float32
    return torch.tensor(_pad(X, ld), dtype=dt, device="cuda")


def _inputs(n, r, seed, prec):
    rng = np.random.default_rng(seed)
    U, V = rng.standard_normal((n, r)), rng.standard_normal((n, r))
    if prec == L.LORADS_PREC_MIXED:
        U, V = U.astype(np.float32).astype(np.float64), V.astype(np.float32).astype(np.float64)
    return U, V


def _tol(prec):
    return 1e-12 if prec == L.LORADS_PREC_FP64 else 1e-5


@pytest.mark.parametrize("name", list(OPS))
@pytest.mark.parametrize("r", RANKS)
@pytest.mark.parametrize("prec", [L.LORADS_PREC_FP64, L.LORADS_PREC_MIXED])
def test_sddmm_general(op_problems, cuda, name, r, prec):
    torch = cuda
    inst, sdp, sabs, prob = op_problems[name]
    ld = (r + 3) // 4 * 4
    U, V = _inputs(sdp.n, r, 10 + r, prec)
    q = torch.full((sdp.m,), np.nan, dtype=torch.float64, device="cuda")
    assert L.lorads_op_sddmm(prob.handle, prec, r, ld, _dev(torch, U, ld, prec),
                             _dev(torch, V, ld, prec), q) == 0
    torch.cuda.synchronize()
    want = sdp.A_of(U, V)
    bound = sabs.A_of(np.linalg.norm(U, axis=1)[:, None], np.linalg.norm(V, axis=1)[:, None])
    assert np.all(np.abs(q.cpu().numpy() - want) <= _tol(prec) * bound + 1e-300)


@pytest.mark.parametrize("name", list(OPS))
@pytest.mark.parametrize("r", RANKS)
@pytest.mark.parametrize("prec", [L.LORADS_PREC_FP64, L.LORADS_PREC_MIXED])
def test_spmm_general(op_problems, cuda, name, r, prec):
    torch = cuda
    inst, sdp, sabs, prob = op_problems[name]
    ld = (r + 3) // 4 * 4
    _, V = _inputs(sdp.n, r, 20 + r, prec)
    w = np.random.default_rng(r).standard_normal(sdp.m)
    gamma = 0.75
    out = _dev(torch, np.full((sdp.n, r), np.nan), ld, prec)
    assert L.lorads_op_spmm(prob.handle, prec, r, ld, torch.tensor(w, device="cuda"), gamma,
                            _dev(torch, V, ld, prec), out) == 0
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)[:, :r]
    want = sdp.At_times(w, V) - sdp.C_times(V) + gamma * V
    v = np.linalg.norm(V, axis=1)[:, None]
    bound = (sabs.At_times(np.abs(w), v) + sabs.C_times(v) + gamma * v).ravel()
    err = np.linalg.norm(got - want, axis=1)
    assert np.all(err <= _tol(prec) * bound + 1e-300)


@pytest.mark.parametrize("name", list(OPS))
@pytest.mark.parametrize("r", RANKS)
@pytest.mark.parametrize("prec", [L.LORADS_PREC_FP64, L.LORADS_PREC_MIXED])
def test_hessian_general(op_problems, cuda, name, r, prec):
    torch = cuda
    inst, sdp, sabs, prob = op_problems[name]
    ld = (r + 3) // 4 * 4
    P, V = _inputs(sdp.n, r, 30 + r, prec)
    rho, gamma = 3.5, 0.75
    out = _dev(torch, np.full((sdp.n, r), np.nan), ld, prec)
    assert L.lorads_op_hessian(prob.handle, prec, r, ld, rho, gamma, _dev(torch, V, ld, prec),
                               _dev(torch, P, ld, prec), out) == 0
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)[:, :r]
    want = OL.hessian_apply(sdp, V, P, rho, gamma)
    p, v = np.linalg.norm(P, axis=1)[:, None], np.linalg.norm(V, axis=1)[:, None]
    bound = (rho * sabs.At_times(sabs.A_of(p, v), v) + gamma * p).ravel()
    err = np.linalg.norm(got - want, axis=1)
    assert np.all(err <= 4 * _tol(prec) * bound + 1e-300)


CLOSED = {
    "theta_C5": (lambda: I.lovasz_theta(5, I.cycle_edges(5)), -math.sqrt(5.0)),
    "theta_Petersen": (lambda: I.lovasz_theta(10, petersen_edges()), -4.0),
    "bisection_C12": (lambda: I.graph_bisection(12, I.cycle_edges(12), np.ones(12)),
                      12 * (1 - math.cos(2 * math.pi / 12)) / 2),
    "bisection_K8": (lambda: I.graph_bisection(8, I.complete_edges(8), np.ones(28)), 16.0),
}


@pytest.mark.parametrize("case", sorted(CLOSED))
@pytest.mark.parametrize("prec", [L.LORADS_PREC_FP64, L.LORADS_PREC_MIXED])
def test_closed_forms_general(cuda, case, prec):
    make, want = CLOSED[case]
    p = L.Problem(make())
    res = p.solve(precision=prec)
    p.close()
    assert res["status"] == 0, L.lorads_status_string(res["status"])
    assert abs(res["objective"] - want) <= 1e-6 * abs(want)
    assert res["r_P"] <= 1e-6 and res["r_D"] <= 1e-6 and res["dual_psd"] <= 1e-6


AGAINST = {
    "theta_er120": lambda: I.lovasz_theta(120, _er_edges(120, 6.0, 11)),
    "maxcut_r1_400": lambda: I.maxcut_rank_one(400, 6.0, 8, 100, seed=7),
    "snl_60": lambda: I.sensor_network(60, 6, 2, 0.4, seed=13),
}


@pytest.fixture(scope="module")
def oracle_solves():
    out = {}
    for k, f in AGAINST.items():
        inst = f()
        sdp = SDP.from_instance(inst)
        out[k] = (inst, sdp, solve(sdp, Params()))
    return out


@pytest.mark.parametrize("case", sorted(AGAINST))
@pytest.mark.parametrize("prec", [L.LORADS_PREC_FP64, L.LORADS_PREC_MIXED])
def test_general_against_oracle(cuda, oracle_solves, case, prec):
    inst, sdp, ref = oracle_solves[case]
    p = L.Problem(inst)
    res = p.solve(precision=prec)
    sol = p.solution()
    p.close()
    assert ref["converged"] and res["status"] == 0, L.lorads_status_string(res["status"])
    assert res["r_P"] <= 1e-6 and res["r_D"] <= 1e-6 and abs(res["gap"]) <= 1e-6
    assert res["dual_psd"] <= 1e-6
    scale = max(abs(ref["objective"]), 1.0)
    assert abs(res["objective"] - ref["objective"]) <= 1e-6 * scale
    rep = OL.kkt_report(sdp, sol["U_hat"], sol["y"])
    assert rep["r_P"] <= 1e-6 and rep["r_D"] <= 1e-6 and abs(rep["gap"]) <= 1e-6
    if inst.name.startswith("snl"):
        Z = sol["U_hat"] @ sol["U_hat"].T
        d = inst.mc_P.shape[0]
        assert np.abs(Z[:d, d:] - inst.mc_P).max() <= 1e-3


@pytest.mark.parametrize("prec", [L.LORADS_PREC_FP64, L.LORADS_PREC_MIXED])
def test_general_scopes_agree(cuda, prec):
    """The theta SDP's Phase II on one CTA and on two CTAs of the whole-GPU scope (chunk sums
    combined across CTAs), both from the oracle's Phase I output (Phase I's 23 outer steps
    amplify reduction-order rounding, so the comparison starts after it): five ADMM iterations
    take the same CG iterations (within 3) and reach the same objective to what the reduction
    order changes; the one-CTA solve repeats itself bit for bit."""
    inst = I.lovasz_theta(120, _er_edges(120, 6.0, 11))
    sdp = SDP.from_instance(inst)
    prm = OL.resolve_auto(sdp, Params())
    ph1 = OL.lralm(sdp, OL.initial_factor(sdp, OL.initial_rank(sdp.m, sdp.n, prm), prm.seed), prm)
    rho0 = min(prm.h * ph1["sigma"], prm.rho_max)
    p = L.Problem(inst)
    runs = []
    for grid in (0, 0, 2):
        assert L.lorads_set_start(p.handle, ph1["U"], ph1["lam"], rho0) == 0
        runs.append(p.solve(precision=prec, phase1=0, max_admm_iter=5, polish=0, grid=grid))
    p.close()
    one, again, two = runs
    assert one["objective"] == again["objective"] and one["cg_iters"] == again["cg_iters"]
    assert abs(one["cg_iters"] - two["cg_iters"]) <= 3
    tol = 1e-9 if prec == L.LORADS_PREC_FP64 else 1e-5
    assert abs(one["objective"] - two["objective"]) <= tol * abs(two["objective"])


def test_general_batch_matches_single_solves(cuda):
    insts = [f() for f in AGAINST.values()]
    probs = [L.Problem(x) for x in insts]
    prm = probs[0].params(precision=L.LORADS_PREC_FP64)
    res, _, _ = L.lorads_solve_batch([p.handle for p in probs], prm)
    singles = [p.solve(precision=L.LORADS_PREC_FP64) for p in probs]
    for p in probs:
        p.close()
    for b, s in zip(res, singles):
        assert b["status"] == 0 and s["status"] == 0
        assert abs(b["objective"] - s["objective"]) <= 1e-6 * max(abs(s["objective"]), 1.0)


def test_empty_constraint_is_an_argument_error(cuda):
    inst = I.lovasz_theta(6, I.cycle_edges(6))
    inst.A_val[-1] = 0.0                      # the last edge constraint has no entry left
    p = L.Problem(inst)
    assert p.solve()["status"] == L.LORADS_ERR_ARG
    p.close()
