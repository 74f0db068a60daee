"""The pins catch plausible mistakes: each test plants one mistake in the oracle (on the CPU,
through monkeypatch) and checks that the pin that guards that step then fails, while it
passes on the oracle as written.  Mistakes: a dropped symmetric term in A(U V^T), a dropped
gamma term in the Hessian, a instead of a^2 in the row-block solve, the sign of lambda in the
subproblem right-hand side, y = +lambda in the output, in Phase III the dropped curvature
term of the Riemannian Hessian and the sign of the sphere multiplier, and in Phase I a dropped
cubic term of the exact line search's quartic, L-BFGS without its initial scaling s'y / y'y,
the Burer-Monteiro gradient without its factor 2, and a rank-one constraint s a a^T whose
scale s is dropped from A^T(w) V."""
import dataclasses
import math

import numpy as np

from oracle import SDP, Params, solve
import oracle.lorads as L
from oracle import sdp as S
from paper_2403_09133_gb300 import instances as I
from tests.helpers_sdp import random_general_sdp


def _A_of_error(sdp, rng):
    U = rng.standard_normal((sdp.n, 3))
    V = rng.standard_normal((sdp.n, 3))
    want = np.array([np.trace(sdp.dense_A(i).T @ (U @ V.T)) for i in range(sdp.m)])
    return np.abs(sdp.A_of(U, V) - want).max()


def test_dropped_symmetric_term_in_A_of(rng, monkeypatch):
    sdp = SDP.from_instance(random_general_sdp(n=9, m=7, nnz_per_con=3, rng=rng))
    assert _A_of_error(sdp, rng) <= 1e-12

    def planted(self, U, V):                       # U_r.V_c only, also off the diagonal
        term = np.einsum("ij,ij->i", U[self.A_row], V[self.A_col])
        return np.bincount(self.A_con, weights=self.A_val * term, minlength=self.m)

    monkeypatch.setattr(S.SDP, "A_of", planted)
    assert _A_of_error(sdp, rng) > 1e-3


def _hessian_error(sdp, rng, rho=2.5, gamma=0.8, r=3):
    W = rng.standard_normal((sdp.n, r))
    P = rng.standard_normal((sdp.n, r))
    # the matrix of eq. linU from the definition: rho sum_i vec(A_i W) vec(A_i W)^T + gamma I
    H = gamma * np.eye(sdp.n * r)
    for i in range(sdp.m):
        a = (sdp.dense_A(i) @ W).ravel()
        H += rho * np.outer(a, a)
    return np.abs(L.hessian_apply(sdp, W, P, rho, gamma).ravel() - H @ P.ravel()).max()


def test_dropped_gamma_in_hessian(rng, monkeypatch):
    sdp = SDP.from_instance(random_general_sdp(n=8, m=5, nnz_per_con=3, rng=rng))
    assert _hessian_error(sdp, rng) <= 1e-10
    monkeypatch.setattr(L, "hessian_apply",
                        lambda sdp, W, P, rho, gamma: rho * sdp.At_times(sdp.A_of(P, W), W))
    assert _hessian_error(sdp, rng) > 1e-2


def _row_solve_error(sdp, rng):
    r, rho, gamma = 3, 6.0, 0.7
    W = rng.standard_normal((sdp.n, r))
    G = rng.standard_normal((sdp.n, r))
    X = L.row_block_solve(sdp, W, G, rho, gamma)
    return np.abs(L.hessian_apply(sdp, W, X, rho, gamma) - G).max()


def test_a_instead_of_a_squared_in_row_block_solve(rng, monkeypatch):
    rows = np.array([0, 1, 2, 4, 6])
    sdp = SDP(7, 5, [0, 1], [1, 2], [1.0, -1.0], np.arange(5), rows, rows,
              np.array([1.0, 2.0, 0.5, 3.0, 1.0]), np.ones(5))
    assert _row_solve_error(sdp, rng) <= 1e-12

    def planted(sdp, W, G, rho, gamma):
        s = np.bincount(sdp.A_row, weights=sdp.A_val, minlength=sdp.n)   # a, not a^2
        w2 = np.einsum("ij,ij->i", W, W)
        wg = np.einsum("ij,ij->i", W, G)
        c = rho * s / (gamma + rho * s * w2)
        return (G - (c * wg)[:, None] * W) / gamma

    monkeypatch.setattr(L, "row_block_solve", planted)
    assert _row_solve_error(sdp, rng) > 1e-3


def _optv_residual(sdp, rng):
    """eq. optv_revise after one ADMM iteration (the KKT identity pinned in test_oracle_admm)."""
    p = Params(cg_rel_tol=1e-14, cg_abs_floor=1e-15, cg_max_iter=5000)
    U0 = rng.standard_normal((sdp.n, 3))
    st = L.AdmmState(U=U0.copy(), V=U0.copy(), lam=0.3 * rng.standard_normal(sdp.m), rho=3.0)
    info = L.admm_iteration(sdp, st, p)
    U1, V1, lam1 = st.U, st.V, st.lam
    res = sdp.C_times(U1) - info["gamma"] * (U1 - V1) + sdp.At_times(lam1, U1)
    return np.linalg.norm(res) / (1 + np.linalg.norm(sdp.C_times(U1)))


def test_lambda_sign_in_rhs(rng, monkeypatch):
    sdp = SDP.from_instance(I.maxcut_er(40, 5.0, seed=8))
    assert _optv_residual(sdp, np.random.default_rng(1)) <= 1e-8
    monkeypatch.setattr(L, "subproblem_rhs", lambda sdp, W, lam, rho, gamma:
                        sdp.At_times(rho * sdp.b + lam, W) - sdp.C_times(W) + gamma * W)
    assert _optv_residual(sdp, np.random.default_rng(1)) > 1e-3


def test_dual_sign_in_output(monkeypatch):
    """K_n: the dual is y = -(n/4) 1 (closed form); y = +lambda fails it."""
    n = 8
    sdp = SDP.from_instance(I.maxcut_complete(n))
    good = solve(sdp, Params(tol=1e-9, max_admm_iter=4000))
    assert np.abs(good["y"] + n / 4).max() <= 1e-4 * n
    real = L.kkt_report

    def planted(sdp, Uh, y, min_eig=None):
        return real(sdp, Uh, -y, min_eig)

    monkeypatch.setattr(L, "kkt_report", planted)
    bad = solve(sdp, Params(tol=1e-9, max_admm_iter=4000))
    # the report built from the wrong sign no longer closes the gap at the K_n optimum
    assert abs(bad["gap"]) > 1e-3 and abs(good["gap"]) <= 1e-6
    assert math.isclose(bad["objective"], good["objective"], rel_tol=1e-9)


def _hessian_fd_error(sdp, seed):
    """|second derivative of f(R(U + tZ)) - <Z, Hess Z>| at a random point of the spheres."""
    rng = np.random.default_rng(seed)
    rad, con, a = L.sphere_structure(sdp)
    U = L.retract(rng.standard_normal((sdp.n, 3)), rad)
    _, mu, _ = L.manifold_multiplier(sdp, U, con, a)
    Z = L.tangent_project(U, rng.standard_normal(U.shape))
    h = 1e-4
    f = lambda W: sdp.C_inner(W, W)
    fd2 = (f(L.retract(U + h * Z, rad)) - 2 * f(U) + f(L.retract(U - h * Z, rad))) / (h * h)
    return abs(fd2 - float(np.vdot(Z, L.riemannian_hessian(sdp, U, mu, Z)))) / (1 + abs(fd2))


def test_dropped_curvature_term_in_riemannian_hessian(monkeypatch):
    sdp = SDP.from_instance(I.maxcut_er(14, 4.0, seed=3))
    assert _hessian_fd_error(sdp, 2) <= 1e-5
    monkeypatch.setattr(L, "riemannian_hessian",
                        lambda sdp, U, mu, Z: 2.0 * L.tangent_project(U, sdp.C_times(Z)))
    assert _hessian_fd_error(sdp, 2) > 1e-2


def test_multiplier_sign_in_phase3(monkeypatch):
    """K_8 from a random start: the trust-region Newton method reaches n^2/4 with y = -(n/4) 1;
    a multiplier of the wrong sign makes the gradient 2(CU + mu U), which is not tangent, and
    the method no longer reaches the optimum."""
    n = 8
    sdp = SDP.from_instance(I.maxcut_complete(n))
    p = L.resolve_auto(sdp, Params(tol=1e-9))
    U0 = np.random.default_rng(4).standard_normal((n, 3))
    good = L.bm_newton_polish(sdp, U0, p)
    assert good["converged"] and abs(-sdp.C_inner(good["U"], good["U"]) - n * n / 4) <= 1e-9 * n * n
    real = L.manifold_multiplier

    def planted(sdp, U, con, a):
        lam, mu, CU = real(sdp, U, con, a)
        return -lam, -mu, CU

    monkeypatch.setattr(L, "manifold_multiplier", planted)
    bad = L.bm_newton_polish(sdp, U0, dataclasses.replace(p, newton_max=30))
    assert not bad["converged"]


def _quartic_error(sdp, rng):
    """max over t of |phi(U + tD) - phi(U) - (a1 t + a2 t^2 + a3 t^3 + a4 t^4)| (Phase I's
    exact line search, Algorithm 1)."""
    U = rng.standard_normal((sdp.n, 3))
    D = rng.standard_normal((sdp.n, 3))
    lam = rng.standard_normal(sdp.m)
    sigma = 1.3
    phi0, _, e0 = L.bm_objective_and_gradient(sdp, U, lam, sigma)
    a1, a2, a3, a4 = L.quartic_coefficients(sdp, U, D, lam, sigma, e0)
    err = 0.0
    for t in [-0.7, 0.1, 0.5, 2.0]:
        phit, _, _ = L.bm_objective_and_gradient(sdp, U + t * D, lam, sigma)
        got = a1 * t + a2 * t ** 2 + a3 * t ** 3 + a4 * t ** 4
        err = max(err, abs(got - (phit - phi0)) / (1 + abs(phit - phi0)))
    return err


def test_dropped_cubic_term_in_line_search(rng, monkeypatch):
    sdp = SDP.from_instance(random_general_sdp(n=9, m=7, nnz_per_con=3, rng=rng))
    assert _quartic_error(sdp, np.random.default_rng(3)) <= 1e-9
    real = L.quartic_coefficients

    def planted(sdp, U, D, lam, sigma, e0):
        a1, a2, _, a4 = real(sdp, U, D, lam, sigma, e0)
        return a1, a2, 0.0, a4

    monkeypatch.setattr(L, "quartic_coefficients", planted)
    assert _quartic_error(sdp, np.random.default_rng(3)) > 1e-6      # the pin holds to 1e-9


def _lbfgs_error(rng):
    """The two-loop recursion against H_k g, H_k from the dense BFGS inverse updates of
    H_0 = (s'y / y'y) I (Nocedal and Wright, eq. 7.19-7.20)."""
    d = 6
    A = rng.standard_normal((d, d))
    A = A @ A.T + d * np.eye(d)
    S = [rng.standard_normal((3, 2)) for _ in range(4)]
    Y = [(A @ s.reshape(-1)).reshape(3, 2) for s in S]
    g = rng.standard_normal((3, 2))
    s_, y_ = S[-1].reshape(-1), Y[-1].reshape(-1)
    H = (s_ @ y_) / (y_ @ y_) * np.eye(d)
    for s, y in zip(S, Y):
        s, y = s.reshape(-1), y.reshape(-1)
        rho = 1.0 / (y @ s)
        Vm = np.eye(d) - rho * np.outer(y, s)
        H = Vm.T @ H @ Vm + rho * np.outer(s, s)
    want = -(H @ g.reshape(-1)).reshape(3, 2)
    return np.abs(L.lbfgs_direction(g, S, Y) - want).max() / np.abs(want).max()


def test_lbfgs_without_initial_scaling(monkeypatch):
    assert _lbfgs_error(np.random.default_rng(5)) <= 1e-10

    def planted(g, S, Y):                      # H_0 = I instead of (s'y / y'y) I
        q = g.copy()
        alphas = []
        for s, y in zip(reversed(S), reversed(Y)):
            rho_i = 1.0 / float(np.vdot(y, s))
            a = rho_i * float(np.vdot(s, q))
            q = q - a * y
            alphas.append((rho_i, a))
        for (s, y), (rho_i, a) in zip(zip(S, Y), reversed(alphas)):
            q = q + (a - rho_i * float(np.vdot(y, q))) * s
        return -q

    monkeypatch.setattr(L, "lbfgs_direction", planted)
    assert _lbfgs_error(np.random.default_rng(5)) > 1e-2


def _bm_gradient_error(sdp, rng):
    """Central differences of phi against grad phi = 2 (C + A^T(lam + sigma e)) U."""
    U = rng.standard_normal((sdp.n, 2))
    lam = rng.standard_normal(sdp.m)
    sigma = 0.8
    _, g, _ = L.bm_objective_and_gradient(sdp, U, lam, sigma)
    h = 1e-6
    err = 0.0
    for j in range(sdp.n):
        for c in range(2):
            E = np.zeros_like(U)
            E[j, c] = h
            fp, _, _ = L.bm_objective_and_gradient(sdp, U + E, lam, sigma)
            fm, _, _ = L.bm_objective_and_gradient(sdp, U - E, lam, sigma)
            err = max(err, abs((fp - fm) / (2 * h) - g[j, c]) / (1 + abs(g[j, c])))
    return err


def test_bm_gradient_without_factor_two(rng, monkeypatch):
    sdp = SDP.from_instance(random_general_sdp(n=8, m=6, nnz_per_con=3, rng=rng))
    assert _bm_gradient_error(sdp, np.random.default_rng(6)) <= 1e-5
    real = L.bm_objective_and_gradient

    def planted(sdp, U, lam, sigma):
        phi, g, e = real(sdp, U, lam, sigma)
        return phi, 0.5 * g, e

    monkeypatch.setattr(L, "bm_objective_and_gradient", planted)
    assert _bm_gradient_error(sdp, np.random.default_rng(6)) > 1e-2


def _At_error(sdp, rng):
    """A^T(w) V against sum_i w_i A_i V with each A_i written out densely (Section 1)."""
    V = rng.standard_normal((sdp.n, 3))
    w = rng.standard_normal(sdp.m)
    want = sum(w[i] * (sdp.dense_A(i) @ V) for i in range(sdp.m))
    return np.abs(sdp.At_times(w, V) - want).max() / np.abs(want).max()


def test_rank_one_scale_dropped_in_At(monkeypatch):
    idx = np.array([0, 3, 5])
    sdp = SDP(7, 3, [0], [0], [1.0], [0, 2], [1, 2], [4, 6], [1.0, -0.5], np.ones(3),
              rank1=[(1, idx, np.array([0.5, -2.0, 1.5]), 1.7)])
    assert _At_error(sdp, np.random.default_rng(8)) <= 1e-13

    def planted(self, w, V):
        out = self.At_matrix(w) @ V
        aV = self.R1 @ V
        return np.asarray(out + self.R1.T @ (w[self.r1_con][:, None] * aV))

    monkeypatch.setattr(S.SDP, "At_times", planted)
    assert _At_error(sdp, np.random.default_rng(8)) > 1e-2
