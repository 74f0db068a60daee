"""Pins for the oracle's linear maps: each against a dense brute-force evaluation of its
definition (Section 1, eq. prob:linear-SDP; eq. linU of Section 4.4)."""
import numpy as np
import pytest

from oracle import SDP
import oracle.lorads as L
from tests.helpers_sdp import random_general_sdp


@pytest.fixture
def small(rng):
    inst = random_general_sdp(n=9, m=7, nnz_per_con=3, rng=rng, rank1_terms=4)
    return SDP.from_instance(inst)


def test_A_of_matches_dense_trace(small, rng):
    U = rng.standard_normal((small.n, 3))
    V = rng.standard_normal((small.n, 3))
    X = U @ V.T
    want = np.array([np.trace(small.dense_A(i).T @ X) for i in range(small.m)])
    np.testing.assert_allclose(small.A_of(U, V), want, rtol=1e-12, atol=1e-12)


def test_At_times_matches_dense_sum(small, rng):
    V = rng.standard_normal((small.n, 4))
    w = rng.standard_normal(small.m)
    want = sum(w[i] * small.dense_A(i) for i in range(small.m)) @ V
    np.testing.assert_allclose(small.At_times(w, V), want, rtol=1e-12, atol=1e-12)


def test_adjoint_identity(small, rng):
    """<A^T(w) V, P> = <w, A(P V^T)> for symmetric A_i."""
    V = rng.standard_normal((small.n, 3))
    P = rng.standard_normal((small.n, 3))
    w = rng.standard_normal(small.m)
    lhs = np.sum(small.At_times(w, V) * P)
    rhs = w @ small.A_of(P, V)
    assert abs(lhs - rhs) <= 1e-11 * (1 + abs(lhs))


def test_rank_one_equals_triplet_expansion(rng):
    """A_i = s a a^T given as a rank-one term gives the same maps as its upper triplets."""
    n, m = 8, 3
    idx = np.array([1, 4, 6])
    a = np.array([0.5, -2.0, 1.5])
    s = 1.7
    base = dict(n=n, m=m, C_row=[0], C_col=[0], C_val=[1.0], b=np.ones(m))
    r1 = SDP(**base, A_con=[0, 2], A_row=[0, 3], A_col=[2, 5], A_val=[1.0, -1.0],
             rank1=[(1, idx, a, s)])
    con, row, col, val = [0, 2], [0, 3], [2, 5], [1.0, -1.0]
    for p in range(3):
        for q in range(p, 3):
            con.append(1); row.append(idx[p]); col.append(idx[q]); val.append(s * a[p] * a[q])
    tr = SDP(**base, A_con=con, A_row=row, A_col=col, A_val=val)
    U = rng.standard_normal((n, 2)); V = rng.standard_normal((n, 2))
    w = rng.standard_normal(m)
    np.testing.assert_allclose(r1.A_of(U, V), tr.A_of(U, V), rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(r1.At_times(w, V), tr.At_times(w, V), rtol=1e-13, atol=1e-13)


def test_C_inner_matches_trace(small, rng):
    U = rng.standard_normal((small.n, 3)); V = rng.standard_normal((small.n, 3))
    assert abs(small.C_inner(U, V) - np.trace(small.dense_C() @ V @ U.T)) < 1e-11


def _vec(M):
    return M.reshape(-1)          # row-major vec; H below is built in the same order


def test_hessian_apply_matches_explicit_nr_matrix(small, rng):
    """eq. linU: H = rho sum_i vec(A_i V) vec(A_i V)^T + gamma I, formed densely."""
    r = 3
    V = rng.standard_normal((small.n, r)); P = rng.standard_normal((small.n, r))
    rho, gamma = 3.0, 0.7
    H = gamma * np.eye(small.n * r)
    for i in range(small.m):
        g = _vec(small.dense_A(i) @ V)
        H += rho * np.outer(g, g)
    want = (H @ _vec(P)).reshape(small.n, r)
    np.testing.assert_allclose(L.hessian_apply(small, V, P, rho, gamma), want, rtol=1e-11, atol=1e-11)


def test_rhs_matches_eq_linU(small, rng):
    r = 2
    V = rng.standard_normal((small.n, r)); lam = rng.standard_normal(small.m)
    rho, gamma = 2.0, 0.5
    C = small.dense_C()
    Ai = [small.dense_A(i) for i in range(small.m)]
    want = -(C @ V - gamma * V + sum(lam[i] * Ai[i] @ V for i in range(small.m))
             - rho * sum(small.b[i] * Ai[i] @ V for i in range(small.m)))
    np.testing.assert_allclose(L.subproblem_rhs(small, V, lam, rho, gamma), want, rtol=1e-11, atol=1e-11)


def test_quartic_coefficients_reproduce_phi(small, rng):
    """phi(U + tD) - phi(U) equals the quartic at several t (exact up to rounding)."""
    U = rng.standard_normal((small.n, 3)); D = rng.standard_normal((small.n, 3))
    lam = rng.standard_normal(small.m); sigma = 1.3
    phi0, _, e0 = L.bm_objective_and_gradient(small, U, lam, sigma)
    a1, a2, a3, a4 = L.quartic_coefficients(small, U, D, lam, sigma, e0)
    for t in [-0.7, 0.1, 0.5, 2.0]:
        phit, _, _ = L.bm_objective_and_gradient(small, U + t * D, lam, sigma)
        want = phit - phi0
        got = a1 * t + a2 * t ** 2 + a3 * t ** 3 + a4 * t ** 4
        assert abs(got - want) <= 1e-9 * (1 + abs(want))


def test_bm_gradient_finite_differences(small, rng):
    U = rng.standard_normal((small.n, 2)); lam = rng.standard_normal(small.m); sigma = 0.8
    _, g, _ = L.bm_objective_and_gradient(small, U, lam, sigma)
    h = 1e-6
    for _ in range(6):
        j, c = rng.integers(0, small.n), rng.integers(0, 2)
        E = np.zeros_like(U); E[j, c] = h
        fp, _, _ = L.bm_objective_and_gradient(small, U + E, lam, sigma)
        fm, _, _ = L.bm_objective_and_gradient(small, U - E, lam, sigma)
        fd = (fp - fm) / (2 * h)
        assert abs(fd - g[j, c]) <= 1e-5 * (1 + abs(g[j, c]))


def test_exact_line_search_vs_grid(rng):
    for _ in range(20):
        a4 = rng.uniform(0.01, 2.0); a3 = rng.standard_normal(); a2 = rng.standard_normal()
        a1 = -abs(rng.standard_normal())          # descent direction
        t = L.exact_line_search(a1, a2, a3, a4)
        grid = np.linspace(0, 10, 200001)
        vals = a1 * grid + a2 * grid ** 2 + a3 * grid ** 3 + a4 * grid ** 4
        tg = grid[np.argmin(vals)]
        ft = a1 * t + a2 * t ** 2 + a3 * t ** 3 + a4 * t ** 4
        assert ft <= vals.min() + 1e-9
        assert abs(t - tg) < 1e-3 or abs(ft - vals.min()) < 1e-9


def test_lbfgs_two_loop_matches_dense_bfgs(rng):
    """Two-loop recursion = H_k g with H_k from the BFGS inverse update of H_0 = s'y/y'y I."""
    d = 6
    A = rng.standard_normal((d, d)); A = A @ A.T + d * np.eye(d)
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
    np.testing.assert_allclose(L.lbfgs_direction(g, S, Y), want, rtol=1e-10, atol=1e-12)
