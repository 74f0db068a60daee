"""FP64 CPU oracle -- LoRADS (Algorithm 2) with LRALM (Phase I) and LRADMM + CG (Phase II).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this module; the CUDA library never calls it.

The method is an iteration, so this file restates its steps in the paper's order and
notation, one function per step, with no fusion or reordering:

  * Phase I (Section 4.1): the augmented Lagrangian method on the Burer-Monteiro problem
    (eq. prob:BM), each subproblem by L-BFGS with an exact line search, plus the dynamic
    rank rule of Section 4.3.
  * Switch (Algorithm 2): U = V = U_BM, lambda = the Phase I multiplier, rho <- h * rho
    (Section 5.1, "The heuristic factor").
  * Phase II (Algorithm 1): U-step and V-step are the linear systems eq. linU / eq. linV,
    each solved by unpreconditioned CG warm-started from the other factor (Section 4.4);
    then lambda += rho (A(U V^T) - b); rho *= 1.2 every 5 iterations up to 5000
    (Section 5.1, "The control of penalty factor").
  * Output: U_hat = (U + V)/2, X = U_hat U_hat^T, y = -lambda.
  * Option (Section 1 admits direct solvers for the subproblems): when every constraint is
    one diagonal entry, ``Params(subsolver="row_direct")`` solves eq. linU / eq. linV exactly,
    row block by row block (``row_block_solve``, Sherman-Morrison), instead of by CG.
  * Checkpoint/resume: ``AdmmState`` holds all Algorithm 1 carries between iterations
    (U, V, lambda, rho, k, the final-test schedule); ``lradmm_resume`` continues from it.

Readings of points the paper leaves open are parameters of ``Params`` (their defaults
are the readings the CUDA library uses as well):
  * gamma is never given a value; gamma = s ||C||_inf (largest absolute row sum of C), with
    s = 1 for the MaxCut class (every constraint one diagonal entry on its own row, b/a > 0)
    and s = 2 otherwise; the phase-switch tolerance and the heuristic factor h follow the same
    class (1e-2 and 10 for MaxCut, Section 5.1; 1e-3 and 1 otherwise): ``resolve_auto``;
  * the multiplier enters eq. ALF with a plus sign, so the SDP dual is y = -lambda;
  * with phi's multiplier normalised as in eq. ALF, the switch takes lambda_0 = lambda_hat
    (the paper's 1/2 factor belongs to the normalisation of eq. def:eKKT);
  * CG stops at ||R|| <= max(1e-3 ||R_0||, 1e-13 ||G||), R_0 the residual of the warm
    start, at most cg_max_iter steps;
  * the CG for the V-step starts from U^{k+1};
  * Phase II stops when the output X = U_hat U_hat^T, y = -lambda meets the paper's own
    termination (primal infeasibility ||A(X) - b||_2 / (1 + ||b||_inf) <= tol, Section 5.2),
    then Appendix B's primal-dual gap, the stationarity of eq. def:eKKT
    r_D = ||(C - A^T y) U_hat||_F / (1 + ||C||_F) and the dual measure
    max(0, -lambda_min(C - A^T y)) / (1 + ||C||_inf), each <= tol (Appendix B divides the
    eigenvalue by 1 + ||vec C||_1, which grows with n).  The tests are taken in that order
    (each only when the previous ones hold); after a failed dual test the next one waits
    max(10, k // 10) iterations.  Eq. stop's second term gamma ||dV|| / (1 + ||V||) is
    reported, not tested.  An output that passes r_P and the gap with r_D > tol goes to
    Phase III (not in the paper: ``bm_newton_polish`` on the product of spheres, else
    ``alm_refine``);
  * a dual infeasibility that fell by less than 10% since the previous (failed) test means
    the rank is too small for the instance (lambda_min(C - A^T y) < 0 persists at a primal-dual
    pair that is otherwise converged): Phase II then raises the rank as Section 4.3 does
    (factor 1.5, same cap), the new columns of U and V being tau z, 0, ..., 0 with z the unit
    eigenvector of lambda_min and tau = escape_scale ||U_hat||_F / sqrt(r);
  * Phase I: sigma_0 = 1/(1+||b||_inf), sigma *= 2 when r_P fails to fall 4x in an outer
    step, up to sigma_max = 1e4 (twice rho_max; an uncapped sigma overflowed on the theta SDP,
    whose primal infeasibility falls slowly), L-BFGS memory 4, inner stop at ||grad||_F/(1+||C||_F) <= min(0.1, 10 r_P), rank growth
    when an inner solve needs more than 300 iterations (switch test first).

Random draws (the initial factor and the columns added by rank growth) come from a
counter-based SplitMix64 generator (Steele, Lea and Flood, OOPSLA 2014) followed by the
Box-Muller transform (Box and Muller, 1958); the CUDA library implements the same
generator independently.
"""
from __future__ import annotations

import dataclasses
import math
import time
from dataclasses import dataclass, field, asdict
from typing import Callable, List, Optional

import numpy as np

from .certify import min_eig_dual_slack, min_eig_pair_dual_slack
from .sdp import SDP


# ======================================================================================
# parameters
# ======================================================================================
@dataclass
class Params:
    r0: int = 0                   # 0 -> rule below
    rank_rule: str = "log2"       # "log2": ceil(log2 m); "paper": round(2 ln m) (Table 2)
    rank_max: int = 0             # 0 -> min(floor(sqrt(2 m)), n, 256)
    rank_factor: float = 1.5      # Section 4.3 / 5.1
    tol: float = 1e-6             # final tolerance
    switch_tol: Optional[float] = None   # Section 5.1: None = by problem class (resolve_auto)
    h: Optional[float] = None     # Section 5.1: heuristic factor; None = by problem class
    rho_max: float = 5000.0       # Section 5.1
    rho_growth: float = 1.2       # Section 5.1
    rho_every: int = 5            # Section 5.1
    gamma_scale: Optional[float] = None  # gamma = gamma_scale * ||C||_inf (paper silent);
                                  # None = by problem class (resolve_auto) ...
    gamma_fixed: float = 0.0      # ... unless gamma_fixed > 0
    max_admm_iter: int = 5000     # Section 5.2
    cg_max_iter: int = 1000
    cg_rel_tol: float = 1e-3      # ||R|| <= cg_rel_tol ||R_0|| (R_0: warm-start residual)
    cg_abs_floor: float = 1e-13   # ... or ||R|| <= cg_abs_floor ||G||
    lbfgs_mem: int = 4
    inner_max_iter: int = 300     # K_in: rank-growth trigger
    inner_tol_factor: float = 10.0
    inner_tol_max: float = 0.1
    inner_tol_abs: float = 1e-12
    max_outer: int = 500
    sigma_factor: float = 2.0
    sigma_decrease: float = 0.25
    sigma_max: float = 1e4          # ALM penalty cap (paper silent): twice rho_max
    new_col_std: float = 1e-2
    seed: int = 1
    phase1: bool = True           # False: caller supplies U0 / lambda0 / rho0
    kkt_dinf: bool = True         # the Appendix B dual infeasibility is part of the stop
    dinf_every: int = 10          # after a failed dual test: wait max(dinf_every, k // 10)
    escape_scale: float = 0.3     # Phase II rank growth along the lambda_min eigenvector
    subsolver: str = "cg"         # eq. linU / linV: "cg" (Section 4.4) or "row_direct"
                                  # (exact block solve; every constraint one diagonal entry)
    polish: str = "auto"          # Phase III, a refinement of eq. prob:BM's stationarity once
                                  # Phase II's output passes r_P and the gap: "auto" = Newton
                                  # on the product of spheres where every row carries one
                                  # diagonal constraint, else the Phase I method continued;
                                  # "off" = Phase II alone
    newton_max: int = 200         # Phase III Newton steps, at most
    newton_cg_max: int = 1000     # CG iterations of one Newton step, at most


# ======================================================================================
# counter-based random numbers: SplitMix64 + Box-Muller
# ======================================================================================
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_mix(z):
    """The SplitMix64 output function applied to uint64 state(s) z."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def splitmix64_at(key, i):
    """i-th output (i = 0, 1, ...) of the SplitMix64 stream seeded with ``key``."""
    i = np.asarray(i, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return splitmix64_mix(np.uint64(key) + (i + np.uint64(1)) * _GAMMA)


def stream_key(seed: int, stream: int) -> np.uint64:
    """Key of sub-stream ``stream``: stream 0 draws U_0, stream g draws the g-th rank growth."""
    return np.uint64(splitmix64_at(np.uint64(seed), np.uint64(stream)))


def uniform_open01(key, i):
    """Uniform in (0, 1) from the top 53 bits of output i."""
    x = splitmix64_at(key, i)
    return ((x >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


def normal_matrix(key, rows: int, cols: int) -> np.ndarray:
    """rows x cols standard normals; entry e = j*cols + c uses outputs 2e and 2e+1."""
    e = np.arange(rows * cols, dtype=np.uint64)
    u1 = uniform_open01(key, 2 * e)
    u2 = uniform_open01(key, 2 * e + np.uint64(1))
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return z.reshape(rows, cols)


# ======================================================================================
# rank rules (Sections 4.3 and 5.1)
# ======================================================================================
def initial_rank(m: int, n: int, p: Params) -> int:
    if p.r0 > 0:
        r = p.r0
    elif p.rank_rule == "paper":
        r = int(round(2.0 * math.log(m)))          # Table 2, "2 log(m)" column
    else:
        r = int(math.ceil(math.log2(max(m, 2))))
    return max(1, min(r, n, rank_cap(m, n, p)))


def rank_cap(m: int, n: int, p: Params) -> int:
    if p.rank_max > 0:
        return min(p.rank_max, n)
    return max(1, min(int(math.floor(math.sqrt(2.0 * m))), n, 256))


def next_rank(r: int, cap: int, p: Params) -> int:
    """Dynamic rank rule: multiply by the factor (1.5), round up, cap."""
    return min(int(math.ceil(p.rank_factor * r - 1e-9)), cap)


def paper_rank_sequence(m: int, steps: int, factor: float = 1.5) -> List[int]:
    """Table 2's ranks: round(2 ln m) at start, then floor(2 ln m * factor^k), capped at
    round(sqrt(2 m)) (the table's sqrt(2m) column)."""
    cap = int(round(math.sqrt(2.0 * m)))
    out = [int(round(2.0 * math.log(m)))]
    for k in range(1, steps + 1):
        out.append(min(int(math.floor(2.0 * math.log(m) * factor ** k)), cap))
    return out


# ======================================================================================
# residual measures
# ======================================================================================
def primal_infeasibility(sdp: SDP, U, V) -> float:
    """||A(U V^T) - b||_2 / (1 + ||b||_inf)  (Section 5.2)."""
    return float(np.linalg.norm(sdp.A_of(U, V) - sdp.b) / (1.0 + sdp.b_inf))


def pd_gap(sdp: SDP, Uh, y) -> float:
    """Appendix B primal-dual gap (<C, X> - b^T y) / (1 + |<C, X>| + |b^T y|), X = Uh Uh^T."""
    pobj = sdp.C_inner(Uh, Uh)
    dobj = float(sdp.b @ y)
    return (pobj - dobj) / (1.0 + abs(pobj) + abs(dobj))


def dual_infeasibility(sdp: SDP, y) -> float:
    """Appendix B dual infeasibility max(0, -lambda_min(C - A^T y)) / (1 + ||c||_1)."""
    return max(0.0, -min_eig_dual_slack(sdp, y)) / (1.0 + sdp.c_one)


def dual_psd_measure(sdp: SDP, y) -> float:
    """Size-independent dual infeasibility max(0, -lambda_min(C - A^T y)) / (1 + ||C||_inf).
    Appendix B divides the same eigenvalue by 1 + ||vec C||_1, which grows with n (about
    4 10^4 on the 141 x 141 torus) and so lets lambda_min = -2 10^-4 pass at 10^-6; the row-sum
    norm ||C||_inf bounds ||C||_2 and does not grow with n."""
    return max(0.0, -min_eig_dual_slack(sdp, y)) / (1.0 + sdp.C_rowsum_max)


def dual_stationarity(sdp: SDP, Uh, lam) -> float:
    """||(C + A^T(lambda)) U_hat||_F / (1 + ||C||_F): first line of eq. def:eKKT with
    f = <C, .> and multiplier 2 lambda (Theorem 1), i.e. y = -lambda."""
    S_U = sdp.C_times(Uh) + sdp.At_times(lam, Uh)
    return float(np.linalg.norm(S_U) / (1.0 + sdp.C_fro))


def augmented_lagrangian(sdp: SDP, U, V, lam, rho, gamma) -> float:
    """L_rho(U, V, lambda) of eq. ALF with f(U V^T) = <C, U V^T>."""
    e = sdp.A_of(U, V) - sdp.b
    return (sdp.C_inner(U, V) + 0.5 * gamma * float(np.sum((U - V) ** 2))
            + float(lam @ e) + 0.5 * rho * float(e @ e))


# ======================================================================================
# Phase II pieces: the linear systems eq. linU / eq. linV and CG (Section 4.4)
# ======================================================================================
def hessian_apply(sdp: SDP, W, P, rho, gamma):
    """(rho sum_i vec(A_i W) vec(A_i W)^T + gamma I) vec(P), W the fixed factor.

    <vec(A_i W), vec(P)> = <A_i, P W^T>, so this is rho A^T(A(P W^T)) W + gamma P.
    """
    q = sdp.A_of(P, W)
    return rho * sdp.At_times(q, W) + gamma * P


def subproblem_rhs(sdp: SDP, W, lam, rho, gamma):
    """Right-hand side of eq. linU (W = V^k) / eq. linV (W = U^{k+1}):
    -(C W - gamma W + A^T(lambda) W - rho A^T(b) W) = (A^T(rho b - lambda) - C) W + gamma W."""
    return sdp.At_times(rho * sdp.b - lam, W) - sdp.C_times(W) + gamma * W


def conjugate_gradient(apply_H: Callable, G, X0, rel_tol: float, abs_floor: float,
                       max_iter: int):
    """Textbook unpreconditioned CG on H X = G from the warm start X0.

    Stops at ||R|| <= max(rel_tol ||R_0||, abs_floor ||G||), R_0 = G - H X0."""
    X = X0.copy()
    R = G - apply_H(X)
    P = R.copy()
    rr = float(np.vdot(R, R))
    target = max(rel_tol * math.sqrt(rr), abs_floor * float(np.linalg.norm(G)))
    it = 0
    while math.sqrt(rr) > target and it < max_iter:
        HP = apply_H(P)
        alpha = rr / float(np.vdot(P, HP))
        X = X + alpha * P
        R = R - alpha * HP
        rr_new = float(np.vdot(R, R))
        it += 1
        if math.sqrt(rr_new) <= target:
            rr = rr_new
            break
        P = R + (rr_new / rr) * P
        rr = rr_new
    return X, it


def row_separable(sdp: SDP) -> bool:
    """Every constraint is a single diagonal entry, A_i = a_i e_j e_j^T (MaxCut's diag(X) = 1)."""
    return (sdp.R1 is None and not np.any(sdp.A_off)
            and np.bincount(sdp.A_con, minlength=sdp.m).max(initial=0) <= 1)


def row_block_solve(sdp: SDP, W, G, rho, gamma):
    """Exact solution of eq. linU / eq. linV for row-separable constraints.  With
    A_i = a_i e_j e_j^T, <A_i, X W^T> = a_i X_j.W_j, so the matrix rho A^T(A(. W^T)) W + gamma I
    is block diagonal with the r x r block gamma I + rho s_j W_j W_j^T on row j
    (s_j = sum of a_i^2 over the constraints on row j, 0 without one).  Section 1 notes that
    the subproblems may be solved by direct methods as well as by CG; the Sherman-Morrison
    formula inverts each block:
        X_j = (G_j - c_j (W_j.G_j) W_j) / gamma,   c_j = rho s_j / (gamma + rho s_j ||W_j||^2)."""
    s = np.bincount(sdp.A_row, weights=sdp.A_val ** 2, minlength=sdp.n)
    w2 = np.einsum("ij,ij->i", W, W)
    wg = np.einsum("ij,ij->i", W, G)
    c = rho * s / (gamma + rho * s * w2)
    return (G - (c * wg)[:, None] * W) / gamma


def maxcut_class(sdp: SDP) -> bool:
    """Every constraint is a single diagonal entry on a row of its own with b_i / a_i > 0 (the
    MaxCut SDP of Section 5.3, X_jj = 1): the class for which Section 5.1 states a phase-switch
    tolerance of 1e-2."""
    return diagonal_row_scaling(sdp) is not None


def resolve_auto(sdp: SDP, p: Params) -> Params:
    """Fills the parameters left at None by the problem class (Section 5.1 states 1e-2 as the
    switch tolerance for MaxCut and 1e-3 for other problems, and h = 10 for MaxCut; h and gamma
    otherwise are readings): MaxCut class -> switch_tol 1e-2, h 10, gamma_scale 1; any other
    problem -> switch_tol 1e-3, h 1, gamma_scale 2.  Explicit values are kept."""
    mc = maxcut_class(sdp)
    q = Params(**{**asdict(p)})
    if q.switch_tol is None:
        q.switch_tol = 1e-2 if mc else 1e-3
    if q.h is None:
        q.h = 10.0 if mc else 1.0
    if q.gamma_scale is None:
        q.gamma_scale = 1.0 if mc else 2.0
    return q


def penalty_gamma(sdp: SDP, p: Params) -> float:
    """gamma of eq. prob:penalty.  The paper fixes no value; the U-step moves U along
    -(C + A^T lambda) V / gamma, so gamma is tied to the scale of C through the row-sum
    norm ||C||_inf = max_j sum_k |C_jk| (an upper bound on ||C||_2)."""
    if p.gamma_fixed > 0:
        return p.gamma_fixed
    cinf = sdp.C_rowsum_max
    scale = p.gamma_scale if p.gamma_scale is not None else resolve_auto(sdp, p).gamma_scale
    return scale * (cinf if cinf > 0 else 1.0)


@dataclass
class AdmmState:
    U: np.ndarray
    V: np.ndarray
    lam: np.ndarray
    rho: float
    k: int = 0
    cg_iters: int = 0
    rp: float = math.inf
    growths: int = 0
    # final-test schedule: first k at which the dual infeasibility may be tested again, and
    # the dual infeasibility of the latest failed test since the last rank growth
    next_dual_test: int = 0
    prev_dinf: Optional[float] = None
    # set when Phase II hands over to Phase III (primal test and gap passed, r_D not yet)
    polish: bool = False


def admm_iteration(sdp: SDP, st: AdmmState, p: Params) -> dict:
    """One pass of Algorithm 1 (U-step, V-step, dual step) plus the penalty schedule."""
    rho = st.rho
    gamma = penalty_gamma(sdp, p)
    direct = p.subsolver == "row_direct"
    if direct and not row_separable(sdp):
        raise ValueError("row_direct needs every constraint to be one diagonal entry")
    # U-step: eq. linU, CG warm-started from V^k (or the exact block solve)
    V = st.V
    G = subproblem_rhs(sdp, V, st.lam, rho, gamma)
    if direct:
        U, itU = row_block_solve(sdp, V, G, rho, gamma), 0
    else:
        U, itU = conjugate_gradient(lambda X: hessian_apply(sdp, V, X, rho, gamma), G, V,
                                    p.cg_rel_tol, p.cg_abs_floor, p.cg_max_iter)
    # V-step: eq. linV, CG warm-started from U^{k+1} (or the exact block solve)
    G = subproblem_rhs(sdp, U, st.lam, rho, gamma)
    if direct:
        V, itV = row_block_solve(sdp, U, G, rho, gamma), 0
    else:
        V, itV = conjugate_gradient(lambda X: hessian_apply(sdp, U, X, rho, gamma), G, U,
                                    p.cg_rel_tol, p.cg_abs_floor, p.cg_max_iter)
    # dual step: lambda^{k+1} = lambda^k + rho (A(U^{k+1} V^{k+1 T}) - b)
    e = sdp.A_of(U, V) - sdp.b
    lam = st.lam + rho * e
    rp = float(np.linalg.norm(e) / (1.0 + sdp.b_inf))
    Uh = 0.5 * (U + V)
    rp_hat = primal_infeasibility(sdp, Uh, Uh)
    # second term of eq. stop: gamma ||V^{k+1} - V^k||_F / (1 + ||V^k||_F)
    rs = gamma * float(np.linalg.norm(V - st.V)) / (1.0 + float(np.linalg.norm(st.V)))
    st.U, st.V, st.lam, st.rp = U, V, lam, rp
    st.k += 1
    st.cg_iters += itU + itV
    info = dict(k=st.k, rho=rho, gamma=gamma, rp=rp, rp_hat=rp_hat, rs=rs, cg_u=itU, cg_v=itV)
    # penalty schedule
    if st.k % p.rho_every == 0:
        st.rho = min(st.rho * p.rho_growth, p.rho_max)
    return info


def lradmm(sdp: SDP, U0, V0, lam0, rho0: float, p: Params, trace: Optional[list] = None):
    """Algorithm 1 from (U0, V0, lam0, rho0) until the final test of ``_lradmm_loop`` passes
    or hands the iterate over to Phase III."""
    st = AdmmState(U=U0.copy(), V=V0.copy(), lam=lam0.copy(), rho=rho0,
                   rp=primal_infeasibility(sdp, U0, V0))
    return _lradmm_loop(sdp, st, p, trace)


def lradmm_resume(sdp: SDP, state: AdmmState, p: Params, trace: Optional[list] = None):
    """Continues Algorithm 1 from a checkpointed iterate: (U^k, V^k, lambda^k), the penalty
    of iteration k+1, k, and the final-test schedule are all the iteration carries from one
    step to the next (each CG solve starts from W), so the continuation repeats the
    uninterrupted run.  `state` is not modified."""
    st = AdmmState(U=state.U.copy(), V=state.V.copy(), lam=state.lam.copy(), rho=state.rho,
                   k=state.k, cg_iters=state.cg_iters, rp=state.rp, growths=state.growths,
                   next_dual_test=state.next_dual_test, prev_dinf=state.prev_dinf)
    return _lradmm_loop(sdp, st, p, trace)


def polish_applies(sdp: SDP, p: Params) -> bool:
    """Phase III takes its Newton form when every row carries exactly one diagonal constraint
    a_i U_j.U_j = b_i with b_i / a_i > 0 (MaxCut, Section 5.3, with n = m): the feasible set of
    eq. prob:BM is then a product of spheres of radius sqrt(b_i / a_i), on which the projection
    is a row scaling.  Other problems take the augmented-Lagrangian form (alm_refine)."""
    return p.polish == "auto" and sdp.n == sdp.m and maxcut_class(sdp)


def _lradmm_loop(sdp: SDP, st: AdmmState, p: Params, trace: Optional[list]):
    """Algorithm 1 with the final test on the output X = U_hat U_hat^T, y = -lambda:
    r_P(X) <= tol (Section 5.2), |gap| <= tol (Appendix B), the stationarity of eq. def:eKKT
    r_D = ||(C - A^T y) U_hat||_F / (1 + ||C||_F) <= tol and the dual measure
    max(0, -lambda_min(C - A^T y)) / (1 + ||C||_inf) <= tol (tested at most once per
    max(dinf_every, k // 10) iterations after a test that did not end the solve).  Where Phase III
    applies, the first iterate that passes the primal test and the gap while r_D > tol is handed
    over to it (st.polish)."""
    converged = False
    cap = rank_cap(sdp.m, sdp.n, p)
    polish = p.polish == "auto"
    while st.k < p.max_admm_iter:
        info = admm_iteration(sdp, st, p)
        if info["rp_hat"] <= p.tol:
            Uh = 0.5 * (st.U + st.V)
            y = -st.lam
            info["gap"] = pd_gap(sdp, Uh, y)
            info["r_D"] = dual_stationarity(sdp, Uh, st.lam)
            if abs(info["gap"]) <= p.tol:
                if polish and info["r_D"] > p.tol:
                    st.polish = True
                elif not p.kkt_dinf:
                    converged = info["r_D"] <= p.tol
                elif st.k >= st.next_dual_test:
                    info["d_psd"] = dual_psd_measure(sdp, y)
                    if info["d_psd"] <= p.tol and info["r_D"] <= p.tol:
                        converged = True
                    else:
                        st.next_dual_test = st.k + max(p.dinf_every, st.k // 10)
                        if info["d_psd"] <= p.tol:
                            pass
                        elif (st.prev_dinf is not None and info["d_psd"] > 0.9 * st.prev_dinf
                                and p.escape_scale > 0):
                            Ws, grew = escape(sdp, [st.U, st.V], Uh, y, p, cap)
                            if Ws is not None:
                                st.U, st.V = Ws
                                st.growths += int(grew)
                                info["grow_to"] = st.U.shape[1]
                                st.prev_dinf = None
                        else:
                            st.prev_dinf = info["d_psd"]
        if trace is not None:
            trace.append(info)
        if converged or st.polish:
            break
    return st, converged


def escape_columns(sdp: SDP, W, Uh, y, r_new: int, p: Params):
    """W with r_new - r columns appended: tau z, then zeros, where z is the unit eigenvector of
    lambda_min(C - A^T y) and tau = escape_scale ||U_hat||_F / sqrt(r) (the size of an average
    column): a descent direction of eq. prob:BM's objective when lambda_min < 0."""
    _, z = min_eig_pair_dual_slack(sdp, y)
    r = W.shape[1]
    tau = p.escape_scale * float(np.linalg.norm(Uh)) / math.sqrt(r)
    add = np.zeros((sdp.n, r_new - r))
    add[:, 0] = tau * z
    return np.concatenate([W, add], axis=1)


def first_zero_column(W) -> int:
    """Index of the first all-zero column of W (the zero padding a rank growth leaves, which every
    step of the method keeps at zero), or -1."""
    zero = np.nonzero(~np.any(W != 0.0, axis=0))[0]
    return int(zero[0]) if zero.size else -1


def escape(sdp: SDP, Ws, Uh, y, p: Params, cap: int):
    """The escape from a point where lambda_min(C - A^T y) < 0: U is then rank-deficient in the
    zero columns a growth left, and [U, tau z] descends (second order, tau^2 lambda_min), so the
    first zero column takes tau z, with tau = escape_scale ||U_hat||_F / sqrt(r); with no zero
    column left the rank grows first (Section 4.3's factor 1.5, at most the cap).  Ws: the
    factors to change alike (U and V in Phase II, U in Phase III).  Returns (new factors,
    whether the rank grew), or (None, False) at the cap with no zero column."""
    c = first_zero_column(Ws[0])
    if c >= 0:
        _, z = min_eig_pair_dual_slack(sdp, y)
        r = Ws[0].shape[1]
        tau = p.escape_scale * float(np.linalg.norm(Uh)) / math.sqrt(r)
        out = []
        for W in Ws:
            W = W.copy()
            W[:, c] = tau * z
            out.append(W)
        return out, False
    r = Ws[0].shape[1]
    if r >= cap:
        return None, False
    r_new = max(next_rank(r, cap, p), r + 1)
    return [escape_columns(sdp, W, Uh, y, r_new, p) for W in Ws], True


# ======================================================================================
# Phase III (not in the paper): Newton refinement of eq. prob:BM's stationarity
# ======================================================================================
# Algorithm 1's dual stationarity falls only like 1/k on degenerate instances (the +-1 torus:
# r_D = 4.8e-4 after 10^3 iterations, 1.7e-5 after 3.2 10^4), while r_D <= 1e-6 asks for a
# relative gap of about 1e-13 there.  When every row carries one diagonal constraint the
# feasible set of eq. prob:BM is a product of spheres, and Newton's method on that manifold
# (Absil, Mahony and Sepulchre, "Optimization Algorithms on Matrix Manifolds", 2008, Ch. 6;
# the Burer-Monteiro MaxCut setting of Boumal, Voroninski and Bandeira, 2016) converges
# quadratically from the point Phase II reaches; its trust-region form reaches second-order
# critical points, where the rank test of Section 4.3's staircase is meaningful.  Each step
# solves its model by truncated CG (Steihaug-Toint) with Hessian-vector products built from
# the same C-times-dense product as the ADMM subproblems.
def sphere_structure(sdp: SDP):
    """Per row j: the sphere radius sqrt(b_i / a_i) of its constraint i, i, and a_i."""
    rows, target = diagonal_row_scaling(sdp)
    rad = np.zeros(sdp.n)
    rad[rows] = target
    con = np.full(sdp.n, -1, dtype=np.int64)
    con[sdp.A_row] = sdp.A_con
    a = np.zeros(sdp.n)
    a[sdp.A_row] = sdp.A_val
    return rad, con, a


def retract(U, rad):
    """Projection onto the product of spheres: row j scaled to length rad_j."""
    return U * (rad / np.linalg.norm(U, axis=1))[:, None]


def tangent_project(U, Z):
    """Row j of Z minus its component along U_j (the tangent space of the sphere at U_j)."""
    return Z - (np.einsum("ij,ij->i", Z, U) / np.einsum("ij,ij->i", U, U))[:, None] * U


def manifold_multiplier(sdp: SDP, U, con, a):
    """On the product of spheres, the multiplier minimising ||(C + A^T lambda) U||_F: row j
    gives (C U)_j + a_i lambda_i U_j, so a_i lambda_i = -(C U)_j.U_j / ||U_j||^2 =: -mu_j.
    Returns lambda (indexed by constraint), mu and C U."""
    CU = sdp.C_times(U)
    mu = np.einsum("ij,ij->i", CU, U) / np.einsum("ij,ij->i", U, U)
    lam = np.zeros(sdp.m)
    lam[con] = -mu / a
    return lam, mu, CU


def riemannian_hessian(sdp: SDP, U, mu, Z):
    """Hessian of <C, U U^T> on the product of spheres applied to a tangent Z:
    2 P_U(C Z - mu Z) (the Euclidean Hessian 2 C Z projected, plus the curvature term of the
    spheres -2 mu_j Z_j)."""
    return 2.0 * tangent_project(U, sdp.C_times(Z) - mu[:, None] * Z)


def boundary_step(d, pdir, delta: float) -> float:
    """tau >= 0 with ||d + tau p|| = delta (the positive root of a quadratic in tau)."""
    a = float(np.vdot(pdir, pdir))
    b = 2.0 * float(np.vdot(d, pdir))
    c = float(np.vdot(d, d)) - delta * delta
    return (-b + math.sqrt(max(b * b - 4.0 * a * c, 0.0))) / (2.0 * a)


def truncated_cg(hess: Callable, g, delta: float, max_iter: int):
    """Steihaug-Toint truncated CG for the trust-region model min g.d + d.Hess d / 2 subject to
    ||d|| <= delta (Absil, Mahony and Sepulchre 2008, Algorithm 11; Nocedal and Wright,
    Algorithm 7.2), from d = 0: stops at ||Hess d + g|| <= eta ||g||, eta = min(0.5, sqrt(||g||)),
    and, where a CG direction has non-positive curvature or the next iterate would leave the
    region, at the boundary point along that direction.  Returns (d, Hessian products, whether d
    lies on the boundary)."""
    gn = float(np.linalg.norm(g))
    eta = min(0.5, math.sqrt(gn))
    d = np.zeros_like(g)
    res = -g
    pdir = res.copy()
    rr = float(np.vdot(res, res))
    for j in range(max_iter):
        Hp = hess(pdir)
        pHp = float(np.vdot(pdir, Hp))
        if pHp <= 0.0:
            return d + boundary_step(d, pdir, delta) * pdir, j + 1, True
        alpha = rr / pHp
        d_next = d + alpha * pdir
        if float(np.vdot(d_next, d_next)) >= delta * delta:
            return d + boundary_step(d, pdir, delta) * pdir, j + 1, True
        d = d_next
        res = res - alpha * Hp
        rr_new = float(np.vdot(res, res))
        if math.sqrt(rr_new) <= eta * gn:
            return d, j + 1, False
        pdir = res + (rr_new / rr) * pdir
        rr = rr_new
    return d, max_iter, False


def bm_newton_polish(sdp: SDP, U0, p: Params) -> dict:
    """Phase III from U0 (Phase II's U_hat): the Riemannian trust-region Newton method on the
    product of spheres (Absil, Mahony and Sepulchre 2008, Algorithm 10; Absil, Baker and
    Gallivan 2007), which reaches second-order critical points: each step minimises the
    quadratic model within radius Delta by truncated CG, then compares the model's decrease with
    the true one along the retraction, rho = (f(U) - f(R(U + d))) / (m(0) - m(d)); the step is
    taken when rho > 0.1, Delta shrinks by 4 when rho < 1/4 and doubles (up to Delta_max =
    ||U||_F) when rho > 3/4 on the boundary; Delta starts at Delta_max / 8.  It runs until
    r_D(U, lambda(U)) <= tol, then tests max(0, -lambda_min(C - A^T y)) / (1 + ||C||_inf) <= tol.
    A failed dual test at a second-order critical point means the rank is too small: the rank
    grows as in Phase II (a column tau z along the eigenvector of lambda_min) and the steps go
    on.  On the manifold A(U U^T) = b holds to rounding and the gap with y = -lambda(U) vanishes
    identically (<C, U U^T> = sum_j mu_j ||U_j||^2 = b^T y)."""
    rad, con, a = sphere_structure(sdp)
    cap = rank_cap(sdp.m, sdp.n, p)
    U = retract(U0, rad)
    delta_max = float(np.linalg.norm(U))
    delta = delta_max / 8.0
    steps = cg_total = growths = 0
    converged = False
    lam = np.zeros(sdp.m)
    while True:
        lam, mu, CU = manifold_multiplier(sdp, U, con, a)
        g = 2.0 * (CU - mu[:, None] * U)                 # the Riemannian gradient, 2 S U
        r_D = float(np.linalg.norm(g)) / (2.0 * (1.0 + sdp.C_fro))
        if r_D <= p.tol:
            if not p.kkt_dinf or dual_psd_measure(sdp, -lam) <= p.tol:
                converged = True
                break
            Ws, grew = escape(sdp, [U], U, -lam, p, cap) if p.escape_scale > 0 else (None, False)
            if Ws is None:
                break
            U = retract(Ws[0], rad)
            growths += int(grew)
            continue
        if steps >= p.newton_max:
            break
        hess = lambda Z: riemannian_hessian(sdp, U, mu, Z)
        d, j, on_boundary = truncated_cg(hess, g, delta, p.newton_cg_max)
        cg_total += j + 2                 # the CG's Hessian products and the model's
        pred = -(float(np.vdot(g, d)) + 0.5 * float(np.vdot(d, hess(d))))
        Un = retract(U + d, rad)
        actual = sdp.C_inner(U, U) - sdp.C_inner(Un, Un)
        ratio = actual / pred if pred > 0.0 else -1.0
        if ratio < 0.25:
            delta *= 0.25
        elif ratio > 0.75 and on_boundary:
            delta = min(2.0 * delta, delta_max)
        if ratio > 0.1:
            U = Un
        steps += 1
    return dict(U=U, lam=lam, converged=converged, steps=steps, cg=cg_total, growths=growths)


# ======================================================================================
# Phase I pieces: LRALM on the BM problem (Section 4.1)
# ======================================================================================
def bm_objective_and_gradient(sdp: SDP, U, lam, sigma):
    """phi(U) = <C, U U^T> + <lam, A(U U^T) - b> + sigma/2 ||A(U U^T) - b||^2 and
    grad phi = 2 (C + A^T(lam + sigma e)) U, e = A(U U^T) - b."""
    e = sdp.A_of(U, U) - sdp.b
    phi = sdp.C_inner(U, U) + float(lam @ e) + 0.5 * sigma * float(e @ e)
    grad = 2.0 * (sdp.C_times(U) + sdp.At_times(lam + sigma * e, U))
    return phi, grad, e


def quartic_coefficients(sdp: SDP, U, D, lam, sigma, e0):
    """phi(U + tD) - phi(U) = a1 t + a2 t^2 + a3 t^3 + a4 t^4, using
    A((U+tD)(U+tD)^T) - b = e0 + t e1 + t^2 e2."""
    e1 = sdp.A_of(U, D) + sdp.A_of(D, U)
    e2 = sdp.A_of(D, D)
    c1 = sdp.C_inner(U, D) + sdp.C_inner(D, U)
    c2 = sdp.C_inner(D, D)
    a1 = c1 + lam @ e1 + sigma * (e0 @ e1)
    a2 = c2 + lam @ e2 + 0.5 * sigma * (e1 @ e1 + 2.0 * (e0 @ e2))
    a3 = sigma * (e1 @ e2)
    a4 = 0.5 * sigma * (e2 @ e2)
    return float(a1), float(a2), float(a3), float(a4)


def exact_line_search(a1, a2, a3, a4) -> float:
    """argmin over t > 0 of a1 t + a2 t^2 + a3 t^3 + a4 t^4 (0 if none decreases)."""
    poly = lambda t: ((a4 * t + a3) * t + a2) * t * t + a1 * t
    deriv = [4.0 * a4, 3.0 * a3, 2.0 * a2, a1]
    while len(deriv) > 1 and deriv[0] == 0.0:
        deriv = deriv[1:]
    if len(deriv) == 1:
        return 0.0
    roots = np.roots(deriv)
    cands = [float(z.real) for z in roots if abs(z.imag) <= 1e-10 * (1.0 + abs(z.real))
             and z.real > 0.0]
    if not cands:
        return 0.0
    best = min(cands, key=poly)
    return best if poly(best) < 0.0 else 0.0


def lbfgs_direction(g, S: list, Y: list):
    """-H g by the L-BFGS two-loop recursion (Nocedal and Wright, Algorithm 7.4)."""
    q = g.copy()
    alphas = []
    for s, y in zip(reversed(S), reversed(Y)):
        rho_i = 1.0 / float(np.vdot(y, s))
        a = rho_i * float(np.vdot(s, q))
        q = q - a * y
        alphas.append((rho_i, a))
    if S:
        s, y = S[-1], Y[-1]
        q = (float(np.vdot(s, y)) / float(np.vdot(y, y))) * q
    for (s, y), (rho_i, a) in zip(zip(S, Y), reversed(alphas)):
        beta = rho_i * float(np.vdot(y, q))
        q = q + (a - beta) * s
    return -q


def diagonal_row_scaling(sdp: SDP):
    """If every constraint is a single diagonal entry a e_j e_j^T on distinct rows with
    b / a > 0 (MaxCut: X_jj = 1), return (rows, target norms) so that rows of U can be
    scaled onto the constraint set; otherwise None."""
    if sdp.R1 is not None or len(sdp.A_con) != sdp.m:
        return None
    if np.any(sdp.A_off) or len(np.unique(sdp.A_con)) != sdp.m:
        return None
    if len(np.unique(sdp.A_row)) != sdp.m:
        return None
    ratio = sdp.b[sdp.A_con] / sdp.A_val
    if np.any(ratio <= 0):
        return None
    return sdp.A_row, np.sqrt(ratio)


def initial_factor(sdp: SDP, r: int, seed: int):
    """U_0 = N(0,1)/sqrt(r) (stream 0), rows scaled onto diagonal constraints if any."""
    U = normal_matrix(stream_key(seed, 0), sdp.n, r) / math.sqrt(r)
    sc = diagonal_row_scaling(sdp)
    if sc is not None:
        rows, target = sc
        nrm = np.linalg.norm(U[rows], axis=1)
        U[rows] = U[rows] * (target / nrm)[:, None]
    return U


def grow_rank(U, r_new: int, seed: int, growth_index: int, std: float):
    """Append r_new - r columns drawn N(0, std^2) from stream ``growth_index``."""
    n, r = U.shape
    extra = std * normal_matrix(stream_key(seed, growth_index), n, r_new - r)
    return np.concatenate([U, extra], axis=1)


def lralm(sdp: SDP, U0, p: Params, trace: Optional[list] = None, lam0=None, sigma0=None,
          refine: bool = False, growth0: int = 0):
    """Phase I: augmented Lagrangian on eq. prob:BM, L-BFGS inner solves, dynamic rank.

    With refine=True the same method continues from (U0, lam0, sigma0) -- Phase II's output --
    until the multiplier-updated pair meets the primal test and the stationarity of
    eq. def:eKKT: r_P <= tol and r_D = ||(C + A^T lambda) U||_F / (1 + ||C||_F) <= tol (after
    an inner solve, (C + A^T(lambda + sigma e)) U is half the gradient of phi, so r_D is read
    from it).  Rank growths draw from streams growth0 + 1, ..."""
    p = resolve_auto(sdp, p)
    U = U0.copy()
    lam = np.zeros(sdp.m) if lam0 is None else np.asarray(lam0, dtype=np.float64).copy()
    sigma = 1.0 / (1.0 + sdp.b_inf) if sigma0 is None else float(sigma0)
    cap = rank_cap(sdp.m, sdp.n, p)
    rp_prev = math.inf
    growths = growth0
    done = False
    inner_total = 0
    rp = primal_infeasibility(sdp, U, U)
    outer = 0
    for outer in range(1, p.max_outer + 1):
        S: list = []
        Y: list = []
        phi, g, e = bm_objective_and_gradient(sdp, U, lam, sigma)
        it = 0
        stalled = False
        while True:
            rp = float(np.linalg.norm(e) / (1.0 + sdp.b_inf))
            grel = float(np.linalg.norm(g) / (1.0 + sdp.C_fro))
            if grel <= max(p.inner_tol_abs, min(p.inner_tol_max, p.inner_tol_factor * rp)):
                break
            if it >= p.inner_max_iter:
                stalled = True
                break
            D = lbfgs_direction(g, S, Y)
            if float(np.vdot(D, g)) >= 0.0:
                D = -g
                S, Y = [], []
            a1, a2, a3, a4 = quartic_coefficients(sdp, U, D, lam, sigma, e)
            t = exact_line_search(a1, a2, a3, a4)
            if t <= 0.0:
                if S:                       # retry once along the steepest descent
                    S, Y = [], []
                    continue
                break
            U_new = U + t * D
            phi_new, g_new, e_new = bm_objective_and_gradient(sdp, U_new, lam, sigma)
            s = U_new - U
            y = g_new - g
            if float(np.vdot(s, y)) > 0.0:
                S.append(s)
                Y.append(y)
                if len(S) > p.lbfgs_mem:
                    S.pop(0)
                    Y.pop(0)
            U, phi, g, e = U_new, phi_new, g_new, e_new
            it += 1
        inner_total += it
        r = U.shape[1]
        if trace is not None:
            trace.append(dict(outer=outer, inner=it, rp=rp, sigma=sigma, rank=r, stalled=stalled))
        if refine:
            r_D = float(np.linalg.norm(g)) / (2.0 * (1.0 + sdp.C_fro))
            if rp <= p.tol and r_D <= p.tol:
                lam = lam + sigma * e
                done = True
                break
        elif rp <= p.switch_tol:
            lam = lam + sigma * e
            done = True
            break
        if stalled and r < cap:
            # Section 4.3: stop the subproblem, raise the rank, carry on
            growths += 1
            U = grow_rank(U, next_rank(r, cap, p), p.seed, growths, p.new_col_std)
            continue
        lam = lam + sigma * e
        if rp > p.sigma_decrease * rp_prev:
            sigma = min(sigma * p.sigma_factor, p.sigma_max)
        rp_prev = rp
    return dict(U=U, lam=lam, sigma=sigma, outer=outer, inner=inner_total,
                growths=growths - growth0, rp=rp, done=done)


# Phase III outside the sphere class runs the augmented Lagrangian method in chunks of this many
# outer iterations, with the dual test between chunks.
REFINE_CHUNK = 25


def alm_refine(sdp: SDP, U0, lam0, sigma0: float, p: Params, growth0: int) -> dict:
    """Phase III for problems outside the product-of-spheres class: the augmented Lagrangian
    method of Phase I continued from Phase II's output (U_hat, lambda) with Phase I's last
    penalty sigma, until r_P <= tol and r_D <= tol and the dual measure
    max(0, -lambda_min(C - A^T y)) / (1 + ||C||_inf) <= tol.  It runs in chunks of
    REFINE_CHUNK outer iterations with the dual measure taken after each: a dual measure above
    tol after a chunk that converged, or after one that did not but left the measure less than
    10% below the previous chunk's, means the rank is too small, and the escape of Phase II
    (tau z along the eigenvector of lambda_min, into a zero column or a grown rank) follows.
    At most max_outer outer iterations in all."""
    cap = rank_cap(sdp.m, sdp.n, p)
    U, lam, sigma = U0.copy(), np.asarray(lam0, dtype=np.float64).copy(), float(sigma0)
    outer = inner = growths = 0
    converged = False
    prev = None
    while outer < p.max_outer:
        q = dataclasses.replace(p, max_outer=min(REFINE_CHUNK, p.max_outer - outer))
        ph = lralm(sdp, U, q, lam0=lam, sigma0=sigma, refine=True, growth0=growth0 + growths)
        U, lam, sigma = ph["U"], ph["lam"], ph["sigma"]
        outer += ph["outer"]
        inner += ph["inner"]
        growths += ph["growths"]
        if not p.kkt_dinf:
            if ph["done"]:
                converged = True
                break
            continue
        d = dual_psd_measure(sdp, -lam)
        if ph["done"] and d <= p.tol:
            converged = True
            break
        if d <= p.tol or (not ph["done"] and (prev is None or d < 0.9 * prev)):
            prev = d
            continue
        Ws, grew = escape(sdp, [U], U, -lam, p, cap) if p.escape_scale > 0 else (None, False)
        if Ws is None:
            break
        U = Ws[0]
        growths += int(grew)
        prev = None
    return dict(U=U, lam=lam, sigma=sigma, converged=converged, outer=outer, inner=inner,
                growths=growths)


# ======================================================================================
# Algorithm 2 (LoRADS) and the KKT report
# ======================================================================================
def kkt_report(sdp: SDP, Uh, y, min_eig: Optional[float] = None) -> dict:
    """Appendix B measures plus BM stationarity.  y is the SDP dual (y = -lambda)."""
    pobj = sdp.C_inner(Uh, Uh)
    dobj = float(sdp.b @ y)
    rep = dict(
        objective=pobj, dual_objective=dobj,
        r_P=primal_infeasibility(sdp, Uh, Uh),
        r_D=dual_stationarity(sdp, Uh, -y),
        gap=(pobj - dobj) / (1.0 + abs(pobj) + abs(dobj)),
        p_infeas=float(np.linalg.norm(sdp.A_of(Uh, Uh) - sdp.b)) / (1.0 + sdp.b_one),
    )
    if min_eig is not None:
        rep["lambda_min"] = min_eig
        rep["d_infeas"] = max(0.0, -min_eig) / (1.0 + sdp.c_one)
        rep["dual_psd"] = max(0.0, -min_eig) / (1.0 + sdp.C_rowsum_max)
    return rep


def lorads(sdp: SDP, p: Params = Params(), U0=None, lam0=None, rho0=None,
           trace: Optional[dict] = None) -> dict:
    """Algorithm 2.  Returns U, V, U_hat, lambda, y and the KKT report."""
    p = resolve_auto(sdp, p)
    t0 = time.perf_counter()
    tr1: list = []
    tr2: list = []
    if p.phase1:
        r = initial_rank(sdp.m, sdp.n, p)
        U_init = initial_factor(sdp, r, p.seed) if U0 is None else U0
        ph1 = lralm(sdp, U_init, p, tr1)
        U_bm, lam_bm, sigma = ph1["U"], ph1["lam"], ph1["sigma"]
        rho = min(p.h * sigma, p.rho_max)
        sigma_last = sigma
    else:
        ph1 = dict(outer=0, inner=0, growths=0, rp=math.nan)
        U_bm = U0
        lam_bm = np.zeros(sdp.m) if lam0 is None else lam0
        rho = 100.0 if rho0 is None else rho0
        sigma_last = 1.0 / (1.0 + sdp.b_inf)
    t1 = time.perf_counter()
    st, converged = lradmm(sdp, U_bm, U_bm, lam_bm, rho, p, tr2)
    t2 = time.perf_counter()
    ph3 = dict(steps=0, cg=0, growths=0, outer=0, inner=0)
    if st.polish:
        Uh = 0.5 * (st.U + st.V)
        if polish_applies(sdp, p):
            ph3 = {**ph3, **bm_newton_polish(sdp, Uh, p)}
        else:
            ph3 = {**ph3, **alm_refine(sdp, Uh, st.lam, sigma_last, p,
                                       ph1["growths"] + st.growths)}
        st.U, st.V, st.lam = ph3["U"], ph3["U"].copy(), ph3["lam"]
        converged = ph3["converged"]
    t3 = time.perf_counter()
    Uh = 0.5 * (st.U + st.V)
    y = -st.lam
    rep = kkt_report(sdp, Uh, y, min_eig_dual_slack(sdp, y))
    if trace is not None:
        trace["phase1"] = tr1
        trace["phase2"] = tr2
    return dict(U=st.U, V=st.V, U_hat=Uh, lam=st.lam, y=y, rank=Uh.shape[1],
                converged=converged, admm_iters=st.k, cg_iters=st.cg_iters, rho=st.rho,
                alm_outer=ph1["outer"], lbfgs_iters=ph1["inner"],
                growths=ph1["growths"] + st.growths + ph3["growths"],
                polished=st.polish, newton_steps=ph3["steps"], newton_cg=ph3["cg"],
                refine_outer=ph3["outer"], refine_lbfgs=ph3["inner"],
                t_phase1=t1 - t0, t_phase2=t2 - t1, t_phase3=t3 - t2, **rep)
