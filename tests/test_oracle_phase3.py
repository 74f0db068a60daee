"""Pins for the oracle's Phase III pieces (the refinement that is not in the paper) and its escape
from saddles, against what differential geometry and linear algebra fix independently of them:

  * the retraction lands on the spheres ||U_j|| = sqrt(b_j / a_j) and leaves points on them fixed;
  * the tangent projection is idempotent and row-wise orthogonal to U;
  * the multiplier minimises ||(C + A^T lambda) U||_F (checked against a least-squares solve of
    that residual over every lambda);
  * 2 (C U - mu U) is the Riemannian gradient: the first derivative of f(R(U + t Z)) at t = 0 along
    a tangent Z (central differences), f(U) = <C, U U^T>;
  * the Riemannian Hessian is symmetric on the tangent space and equals the second derivative of
    f(R(U + t Z)) at t = 0 (row normalisation is a second-order retraction on a sphere);
  * the truncated CG solves the Newton system inside the region (dense solve), stops on the
    boundary along the first direction for a small radius (the Cauchy direction -g) and along a
    direction of negative curvature;
  * the whole trust-region method reaches the closed-form values of K_n, an odd cycle and a torus;
  * the escape puts tau z, z the unit eigenvector of lambda_min(C - A^T y), into the first zero
    column, and grows the rank only when no zero column is left.
"""
import math

import numpy as np
import pytest

from oracle import SDP, Params
import oracle.lorads as L
from oracle.certify import min_eig_dual_slack
from paper_2403_09133_gb300 import instances as I


def lam_max_cycle(k):
    return 4.0 if k % 2 == 0 else 2.0 + 2.0 * math.cos(math.pi / k)


def _er_sdp(n=14, deg=4.0, seed=3):
    return SDP.from_instance(I.maxcut_er(n, deg, seed))


def _on_manifold(sdp, r, rng):
    rad, con, a = L.sphere_structure(sdp)
    U = L.retract(rng.standard_normal((sdp.n, r)), rad)
    return U, rad, con, a


def _tangent(U, rng):
    return L.tangent_project(U, rng.standard_normal(U.shape))


def _f(sdp, U):
    return sdp.C_inner(U, U)


def test_sphere_structure_matches_constraints():
    sdp = SDP.from_instance(I.maxcut_sdp(4, np.array([[0, 1], [1, 2], [2, 3]]),
                                         np.array([1.0, -2.0, 0.5])))
    rad, con, a = L.sphere_structure(sdp)
    np.testing.assert_allclose(rad, np.ones(4))          # X_jj = 1: unit spheres
    assert sorted(con.tolist()) == [0, 1, 2, 3]
    np.testing.assert_allclose(a, np.ones(4))


def test_retraction_lands_on_the_spheres(rng):
    sdp = _er_sdp()
    rad, _, _ = L.sphere_structure(sdp)
    rad = rad * rng.uniform(0.5, 2.0, size=rad.shape)    # any radii
    U = L.retract(rng.standard_normal((sdp.n, 3)), rad)
    np.testing.assert_allclose(np.linalg.norm(U, axis=1), rad, rtol=1e-14)
    np.testing.assert_allclose(L.retract(U, rad), U, rtol=1e-14)


def test_tangent_projection(rng):
    sdp = _er_sdp()
    U, *_ = _on_manifold(sdp, 4, rng)
    Z = rng.standard_normal(U.shape)
    T = L.tangent_project(U, Z)
    assert np.abs(np.einsum("ij,ij->i", T, U)).max() <= 1e-13
    np.testing.assert_allclose(L.tangent_project(U, T), T, atol=1e-14)
    # the removed part is along U_j
    N = Z - T
    cos = np.einsum("ij,ij->i", N, U) / (np.linalg.norm(N, axis=1) * np.linalg.norm(U, axis=1))
    np.testing.assert_allclose(np.abs(cos), 1.0, rtol=1e-12)


def test_multiplier_minimises_the_stationarity_residual(rng):
    sdp = _er_sdp()
    U, rad, con, a = _on_manifold(sdp, 3, rng)
    lam, mu, CU = L.manifold_multiplier(sdp, U, con, a)
    # vec((C + A^T lam) U) = vec(C U) + M lam, column i of M = vec(A_i U): least squares over lam
    M = np.stack([(sdp.dense_A(i) @ U).ravel() for i in range(sdp.m)], axis=1)
    ls = np.linalg.lstsq(M, -(sdp.dense_C() @ U).ravel(), rcond=None)[0]
    np.testing.assert_allclose(lam, ls, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(CU, sdp.dense_C() @ U, atol=1e-13)


def test_riemannian_gradient_by_finite_differences(rng):
    sdp = _er_sdp()
    U, rad, con, a = _on_manifold(sdp, 3, rng)
    _, mu, CU = L.manifold_multiplier(sdp, U, con, a)
    g = 2.0 * (CU - mu[:, None] * U)
    assert np.abs(np.einsum("ij,ij->i", g, U)).max() <= 1e-12        # tangent
    for _ in range(3):
        Z = _tangent(U, rng)
        h = 1e-5
        fd = (_f(sdp, L.retract(U + h * Z, rad)) - _f(sdp, L.retract(U - h * Z, rad))) / (2 * h)
        assert abs(fd - float(np.vdot(g, Z))) <= 1e-7 * (1 + abs(fd))


def test_riemannian_hessian_symmetric_and_second_derivative(rng):
    sdp = _er_sdp()
    U, rad, con, a = _on_manifold(sdp, 3, rng)
    _, mu, _ = L.manifold_multiplier(sdp, U, con, a)
    Z1, Z2 = _tangent(U, rng), _tangent(U, rng)
    H1 = L.riemannian_hessian(sdp, U, mu, Z1)
    H2 = L.riemannian_hessian(sdp, U, mu, Z2)
    assert np.abs(np.einsum("ij,ij->i", H1, U)).max() <= 1e-12       # maps into the tangent
    assert abs(np.vdot(Z1, H2) - np.vdot(H1, Z2)) <= 1e-12 * np.linalg.norm(H1) * np.linalg.norm(Z2)
    for Z in (Z1, Z2):
        h = 1e-4
        f0 = _f(sdp, U)
        fp = _f(sdp, L.retract(U + h * Z, rad))
        fm = _f(sdp, L.retract(U - h * Z, rad))
        fd2 = (fp - 2 * f0 + fm) / (h * h)
        want = float(np.vdot(Z, L.riemannian_hessian(sdp, U, mu, Z)))
        assert abs(fd2 - want) <= 1e-5 * (1 + abs(want)), (fd2, want)


def test_boundary_step_root(rng):
    d = rng.standard_normal(7) * 0.1
    p = rng.standard_normal(7)
    tau = L.boundary_step(d, p, 2.0)
    assert tau >= 0
    assert abs(np.linalg.norm(d + tau * p) - 2.0) <= 1e-13


def _spd(k, rng, cond=30.0):
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    return Q @ np.diag(np.geomspace(1.0, cond, k)) @ Q.T


def test_truncated_cg_interior_solution(rng):
    k = 12
    H = _spd(k, rng)
    g = rng.standard_normal(k)
    g *= 1e-12 / np.linalg.norm(g)              # eta = sqrt(||g||) = 1e-6: a near-exact solve
    d, used, on_b = L.truncated_cg(lambda x: H @ x, g, 1.0, 100)
    assert not on_b and used <= k + 1
    np.testing.assert_allclose(d, -np.linalg.solve(H, g), rtol=1e-4)
    # the stopping rule itself: ||H d + g|| <= min(0.5, sqrt(||g||)) ||g||, with a looser eta
    g2 = rng.standard_normal(k) * 1e-2
    d2, _, on_b2 = L.truncated_cg(lambda x: H @ x, g2, 1e3, 100)
    gn = np.linalg.norm(g2)
    assert not on_b2
    assert np.linalg.norm(H @ d2 + g2) <= min(0.5, math.sqrt(gn)) * gn


def test_truncated_cg_small_radius_takes_the_cauchy_direction(rng):
    H = _spd(10, rng)
    g = rng.standard_normal(10)
    d, used, on_b = L.truncated_cg(lambda x: H @ x, g, 1e-6, 100)
    assert on_b and used == 1
    np.testing.assert_allclose(d, -1e-6 * g / np.linalg.norm(g), rtol=1e-12)


def test_truncated_cg_negative_curvature_goes_to_the_boundary(rng):
    k = 8
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    H = Q @ np.diag([-1.0] + [2.0] * (k - 1)) @ Q.T
    g = Q[:, 0] * 0.3 + 1e-3 * Q[:, 1]           # mostly along the negative direction
    d, _, on_b = L.truncated_cg(lambda x: H @ x, g, 0.7, 100)
    assert on_b
    assert abs(np.linalg.norm(d) - 0.7) <= 1e-12
    # the first direction -g already has negative curvature: the boundary point along it
    np.testing.assert_allclose(d, -0.7 * g / np.linalg.norm(g), rtol=1e-12)
    assert float(g @ d + 0.5 * d @ H @ d) < 0


@pytest.mark.parametrize("case", ["K8", "C11", "T6x8"])
def test_trust_region_newton_reaches_closed_forms(case):
    if case == "K8":
        inst, want = I.maxcut_complete(8), 8 * 8 / 4
    elif case == "C11":
        inst, want = I.maxcut_cycle(11), 11 * lam_max_cycle(11) / 4
    else:
        inst, want = I.maxcut_torus(6, 8, seed=None), 48 * (lam_max_cycle(6) + lam_max_cycle(8)) / 4
    sdp = SDP.from_instance(inst)
    p = L.resolve_auto(sdp, Params(tol=1e-9))
    r = 4
    rng = np.random.default_rng(11)
    out = L.bm_newton_polish(sdp, rng.standard_normal((sdp.n, r)), p)
    assert out["converged"]
    U = out["U"]
    assert abs(-_f(sdp, U) - want) <= 1e-9 * want
    np.testing.assert_allclose(np.linalg.norm(U, axis=1), 1.0, rtol=1e-13)
    y = -out["lam"]
    assert min_eig_dual_slack(sdp, y) >= -1e-7
    assert abs(float(sdp.b @ y) - _f(sdp, U)) <= 1e-9 * want     # the gap vanishes on the manifold


def test_escape_fills_the_first_zero_column_with_the_eigenvector(rng):
    sdp = _er_sdp(n=12, deg=4.0, seed=5)
    p = L.resolve_auto(sdp, Params())
    U = rng.standard_normal((sdp.n, 4))
    U[:, 2] = 0.0
    U[:, 3] = 0.0
    y = -np.abs(rng.standard_normal(sdp.m)) * 0.1       # S = C - A^T y has a negative eigenvalue
    Ws, grew = L.escape(sdp, [U, U.copy()], U, y, p, cap=L.rank_cap(sdp.m, sdp.n, p))
    assert not grew
    S = sdp.dual_slack(y)
    S = S.toarray() if hasattr(S, "toarray") else np.asarray(S)
    w, Q = np.linalg.eigh(S)
    assert w[0] < 0
    tau = p.escape_scale * np.linalg.norm(U) / math.sqrt(4)
    for W in Ws:
        np.testing.assert_array_equal(W[:, :2], U[:, :2])
        z = W[:, 2] / tau
        assert abs(np.linalg.norm(z) - 1.0) <= 1e-10
        assert abs(abs(float(z @ Q[:, 0])) - 1.0) <= 1e-8
        np.testing.assert_array_equal(W[:, 3], 0.0)
    assert L.first_zero_column(Ws[0]) == 3


def test_escape_grows_the_rank_only_without_a_zero_column(rng):
    sdp = _er_sdp(n=12, deg=4.0, seed=5)
    p = L.resolve_auto(sdp, Params())
    cap = L.rank_cap(sdp.m, sdp.n, p)
    U = rng.standard_normal((sdp.n, 2))
    y = -np.abs(rng.standard_normal(sdp.m)) * 0.1
    Ws, grew = L.escape(sdp, [U], U, y, p, cap)
    assert grew
    W = Ws[0]
    assert W.shape[1] == max(L.next_rank(2, cap, p), 3)
    np.testing.assert_array_equal(W[:, :2], U)
    assert np.linalg.norm(W[:, 2]) > 0
    assert np.all(W[:, 3:] == 0)
    Ufull = rng.standard_normal((sdp.n, cap))
    assert L.escape(sdp, [Ufull], Ufull, y, p, cap) == (None, False)
