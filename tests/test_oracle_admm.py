"""Pins for Phase II (Algorithm 1, Section 4.4): the CG step against closed forms and a
dense solve, and the ADMM identities of Proposition 1 and Section 2.2."""
import math

import numpy as np
import pytest

from oracle import SDP, Params
import oracle.lorads as L
from paper_2403_09133_gb300 import instances as I
from tests.helpers_sdp import random_general_sdp


def _tight():
    return Params(cg_rel_tol=1e-14, cg_abs_floor=1e-15, cg_max_iter=5000)


def test_cg_maxcut_matches_sherman_morrison(rng):
    """MaxCut: A_i = e_i e_i^T makes eq. linU block diagonal, (rho V_i V_i^T + gamma I) U_i = G_i,
    solved per row by Sherman-Morrison."""
    sdp = SDP.from_instance(I.maxcut_er(40, 5.0, seed=3))
    V = rng.standard_normal((40, 4)); lam = rng.standard_normal(40)
    rho, gamma = 7.0, 1.5
    G = L.subproblem_rhs(sdp, V, lam, rho, gamma)
    U, it = L.conjugate_gradient(lambda X: L.hessian_apply(sdp, V, X, rho, gamma), G, V,
                                 1e-14, 1e-16, 1000)
    vg = np.einsum("ij,ij->i", V, G)
    vv = np.einsum("ij,ij->i", V, V)
    want = (G - (rho * vg / (gamma + rho * vv))[:, None] * V) / gamma
    np.testing.assert_allclose(U, want, rtol=1e-10, atol=1e-10)


def _row_separable_sdp(rng):
    """n = 7, constraints on rows 0, 1, 2, 4, 6 with a = 1, 2, 0.5, 3, 1 (rows 3 and 5 have
    none), a random symmetric C."""
    rows = np.array([0, 1, 2, 4, 6])
    a = np.array([1.0, 2.0, 0.5, 3.0, 1.0])
    cr, cc = np.triu_indices(7)
    keep = rng.random(len(cr)) < 0.5
    return SDP(7, 5, cr[keep], cc[keep], rng.standard_normal(keep.sum()), np.arange(5), rows,
               rows, a, rng.standard_normal(5))


def test_row_block_solve_matches_dense_solve(rng):
    """The direct subproblem solve against a dense solve of the nr x nr system built column by
    column from hessian_apply (non-unit a_i, rows without a constraint)."""
    sdp = _row_separable_sdp(rng)
    assert L.row_separable(sdp)
    r, rho, gamma = 3, 6.0, 0.7
    W = rng.standard_normal((7, r)); lam = rng.standard_normal(5)
    G = L.subproblem_rhs(sdp, W, lam, rho, gamma)
    H = np.zeros((7 * r, 7 * r))
    for t in range(7 * r):
        E = np.zeros(7 * r); E[t] = 1.0
        H[:, t] = L.hessian_apply(sdp, W, E.reshape(7, r), rho, gamma).ravel()
    want = np.linalg.solve(H, G.ravel()).reshape(7, r)
    np.testing.assert_allclose(L.row_block_solve(sdp, W, G, rho, gamma), want,
                               rtol=1e-12, atol=1e-12)


def test_row_separable_detection(rng):
    assert L.row_separable(SDP.from_instance(I.maxcut_er(20, 3.0, seed=1)))
    assert not L.row_separable(SDP.from_instance(I.matrix_completion(5, 4, 1, 8, seed=1)))
    assert not L.row_separable(SDP.from_instance(random_general_sdp(6, 4, 2, rng)))
    with pytest.raises(ValueError):
        L.admm_iteration(SDP.from_instance(I.matrix_completion(5, 4, 1, 8, seed=1)),
                         L.AdmmState(U=np.ones((9, 2)), V=np.ones((9, 2)), lam=np.zeros(8),
                                     rho=1.0), Params(subsolver="row_direct"))


@pytest.mark.parametrize("case", ["K10", "torus6x8"])
def test_row_direct_whole_solve_closed_forms(case):
    """Algorithm 2 with the direct subproblem solve reaches the closed-form SDP values:
    K_n: n^2/4; a x b unit torus: n (lambda_max(C_a) + lambda_max(C_b)) / 4."""
    from oracle import solve
    if case == "K10":
        inst, want = I.maxcut_complete(10), 25.0
    else:
        inst = I.maxcut_torus(6, 8, seed=None)
        lmax = lambda k: 4.0 if k % 2 == 0 else 2.0 + 2.0 * math.cos(math.pi / k)
        want = 48 * (lmax(6) + lmax(8)) / 4
    sdp = SDP.from_instance(inst)
    res = solve(sdp, Params(subsolver="row_direct", tol=1e-9, max_admm_iter=6000))
    assert res["cg_iters"] == 0
    assert abs(-res["objective"] - want) <= 1e-7 * want


def test_cg_two_steps_when_rows_unit(rng):
    """With ||V_i|| = 1 for all i the spectrum is {gamma, gamma + rho}: CG ends in <= 2 steps."""
    sdp = SDP.from_instance(I.maxcut_er(60, 6.0, seed=4))
    V = rng.standard_normal((60, 5)); V /= np.linalg.norm(V, axis=1, keepdims=True)
    G = rng.standard_normal((60, 5))
    _, it = L.conjugate_gradient(lambda X: L.hessian_apply(sdp, V, X, 9.0, 2.0), G,
                                 np.zeros_like(G), 1e-12, 1e-16, 100)
    assert it <= 2


def test_cg_general_matches_dense_solve(rng):
    inst = random_general_sdp(n=8, m=6, nnz_per_con=3, rng=rng, rank1_terms=2)
    sdp = SDP.from_instance(inst)
    r = 3
    V = rng.standard_normal((8, r)); lam = rng.standard_normal(6); rho, gamma = 4.0, 0.9
    G = L.subproblem_rhs(sdp, V, lam, rho, gamma)
    H = gamma * np.eye(8 * r)
    for i in range(6):
        g = (sdp.dense_A(i) @ V).reshape(-1)
        H += rho * np.outer(g, g)
    want = np.linalg.solve(H, G.reshape(-1)).reshape(8, r)
    U, _ = L.conjugate_gradient(lambda X: L.hessian_apply(sdp, V, X, rho, gamma), G, V,
                                1e-14, 1e-16, 1000)
    np.testing.assert_allclose(U, want, rtol=1e-9, atol=1e-9)


def _one_iteration(sdp, rng, r=4):
    p = _tight()
    U0 = rng.standard_normal((sdp.n, r)) * 0.5
    V0 = U0 + 0.05 * rng.standard_normal((sdp.n, r))
    lam0 = 0.3 * rng.standard_normal(sdp.m)
    st = L.AdmmState(U=U0.copy(), V=V0.copy(), lam=lam0.copy(), rho=3.0, rp=1.0)
    info = L.admm_iteration(sdp, st, p)
    return p, U0, V0, lam0, st, info


@pytest.mark.parametrize("kind", ["maxcut", "general"])
def test_proposition1_identities(kind, rng):
    """eq. decrease1 (dual step raises L_rho by exactly ||dlambda||^2 / rho) and
    eq. decrease2 (exact U- and V-steps lower it by >= gamma/2 (||dU||^2 + ||dV||^2))."""
    if kind == "maxcut":
        sdp = SDP.from_instance(I.maxcut_er(50, 6.0, seed=5))
    else:
        sdp = SDP.from_instance(random_general_sdp(n=10, m=6, nnz_per_con=3, rng=rng, rank1_terms=2))
    p, U0, V0, lam0, st, info = _one_iteration(sdp, rng)
    rho, gamma = info["rho"], info["gamma"]
    U1, V1, lam1 = st.U, st.V, st.lam
    Lf = lambda U, V, lam: L.augmented_lagrangian(sdp, U, V, lam, rho, gamma)
    d1 = Lf(U1, V1, lam1) - Lf(U1, V1, lam0)
    assert abs(d1 - np.sum((lam1 - lam0) ** 2) / rho) <= 1e-9 * (1 + abs(d1))
    d2 = Lf(U1, V1, lam0) - Lf(U0, V0, lam0)
    bound = -0.5 * gamma * (np.sum((V1 - V0) ** 2) + np.sum((U1 - U0) ** 2))
    assert d2 <= bound + 1e-9 * (1 + abs(bound))


@pytest.mark.parametrize("kind", ["maxcut", "general"])
def test_kkt_identities_after_iteration(kind, rng):
    """eq. optv_revise with U^{k+1} in its first factor (the printed V^{k+1} there is a typo:
    it follows from eq. optV and the dual step):
        C U^{k+1} - gamma (U^{k+1} - V^{k+1}) + sum_i lambda_i^{k+1} A_i U^{k+1} = 0,
    and eq. optU_revise for linear f (the gradient-difference terms vanish)."""
    if kind == "maxcut":
        sdp = SDP.from_instance(I.maxcut_er(50, 6.0, seed=6))
    else:
        sdp = SDP.from_instance(random_general_sdp(n=10, m=6, nnz_per_con=3, rng=rng, rank1_terms=2))
    p, U0, V0, lam0, st, info = _one_iteration(sdp, rng)
    gamma, rho = info["gamma"], info["rho"]
    U1, V1, lam1 = st.U, st.V, st.lam
    resid_v = sdp.C_times(U1) - gamma * (U1 - V1) + sdp.At_times(lam1, U1)
    assert np.linalg.norm(resid_v) <= 1e-8 * (1 + np.linalg.norm(sdp.C_times(U1)))
    lhs = sdp.C_times(V1) + gamma * (U1 - V1) + sdp.At_times(lam1, V1)
    dV = V1 - V0
    rhs = (sdp.C_times(dV) + gamma * (V0 - V1)
           + rho * sdp.At_times(sdp.A_of(U1, dV), V0) + sdp.At_times(lam1, dV))
    assert np.linalg.norm(lhs - rhs) <= 1e-8 * (1 + np.linalg.norm(lhs))
