"""Pins for the oracle's learned warm start: its backward pass against central finite
differences of the loss (every parameter block), the output constraint X_jj = 1, and the
definitions of the normalised adjacency, the node features and the forward pass against values
worked out by hand on a four-node graph."""
import numpy as np
import pytest

import oracle.gnn as G
from paper_2403_09133_gb300 import instances as I


@pytest.fixture(scope="module")
def setup():
    inst = I.maxcut_er(40, 5.0, seed=3)
    ei, ej, w = G.graph_of(inst)
    A, _ = G.normalized_adjacency(inst.n, ei, ej, w)
    X0 = G.features(inst.n, ei, ej, w, seed=7)
    P = G.init_params(seed=11)
    rng = np.random.default_rng(0)
    Xs = rng.uniform(-1, 1, len(ei))
    ys = rng.standard_normal(inst.n)
    return inst, ei, ej, A, X0, P, Xs, ys


def test_rows_on_unit_sphere(setup):
    inst, ei, ej, A, X0, P, Xs, ys = setup
    U, y, _ = G.forward(P, X0, A, r=6)
    np.testing.assert_allclose(np.sum(U * U, axis=1), 1.0, rtol=1e-13)


@pytest.mark.parametrize("name", ["theta0", "b0", "theta1", "b1", "theta2", "b2", "theta_u", "theta_y", "b_y"])
def test_gradient_finite_differences(setup, name):
    inst, ei, ej, A, X0, P, Xs, ys = setup
    r = 6
    loss, Gr, _, _ = G.loss_and_grad(P, X0, A, ei, ej, Xs, ys, r)
    rng = np.random.default_rng(hash(name) % 2**32)
    flat = P[name].reshape(-1)
    idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
    if name == "theta_u":
        idx = np.array([i for i in range(flat.size) if i % G.RMAX < r])[:6]
    h = 1e-6
    for k in idx:
        Pp = {kk: v.copy() for kk, v in P.items()}
        Pm = {kk: v.copy() for kk, v in P.items()}
        Pp[name].reshape(-1)[k] += h
        Pm[name].reshape(-1)[k] -= h
        lp = G.loss_and_grad(Pp, X0, A, ei, ej, Xs, ys, r)[0]
        lm = G.loss_and_grad(Pm, X0, A, ei, ej, Xs, ys, r)[0]
        fd = (lp - lm) / (2 * h)
        an = Gr[name].reshape(-1)[k]
        assert abs(fd - an) <= 1e-6 * (1 + abs(an)), (name, k, fd, an)


# ---- hand-computed pins of the definitions (not of the oracle's own arithmetic) ----------
# Graph: edges (0,1), (1,2), (0,2), (2,3) with MaxCut weights 4, -4, 8, 4, so the
# off-diagonal entries of C = -L/4 are w = 1, -1, 2, 1.
#   d = 1 + sum |w|:      d0 = 1+1+2 = 4, d1 = 1+1+1 = 3, d2 = 1+1+2+1 = 5, d3 = 1+1 = 2
#   A_hat_ij = w_ij/sqrt(d_i d_j):
#     A01 = 1/sqrt(12) = 0.28867513459481287,  A12 = -1/sqrt(15) = -0.2581988897471611,
#     A02 = 2/sqrt(20) = 0.4472135954999579,   A23 = 1/sqrt(10) = 0.31622776601683794
#   features (columns 8..11): 1, log(1+deg) with deg = 2, 2, 3, 1, d/10, s = sum w / d:
#     s0 = (1+2)/4 = 0.75, s1 = (1-1)/3 = 0, s2 = (2-1+1)/5 = 0.4, s3 = 1/2 = 0.5
def _tiny():
    inst = I.maxcut_sdp(4, np.array([[0, 1], [1, 2], [0, 2], [2, 3]]),
                        np.array([4.0, -4.0, 8.0, 4.0]))
    return inst, G.graph_of(inst)


def test_normalized_adjacency_by_hand():
    inst, (ei, ej, w) = _tiny()
    A, d = G.normalized_adjacency(inst.n, ei, ej, w)
    np.testing.assert_allclose(d, [4.0, 3.0, 5.0, 2.0], rtol=0, atol=1e-15)
    a01, a12, a02, a23 = 0.28867513459481287, -0.2581988897471611, 0.4472135954999579, 0.31622776601683794
    want = np.array([[0.0, a01, a02, 0.0],
                     [a01, 0.0, a12, 0.0],
                     [a02, a12, 0.0, a23],
                     [0.0, 0.0, a23, 0.0]])
    np.testing.assert_allclose(A.toarray(), want, rtol=1e-15, atol=1e-16)


def test_features_by_hand():
    inst, (ei, ej, w) = _tiny()
    X = G.features(inst.n, ei, ej, w, seed=7)
    assert X.shape == (4, G.HIDDEN)
    np.testing.assert_array_equal(X[:, 8], 1.0)
    np.testing.assert_allclose(X[:, 9], [1.0986122886681098, 1.0986122886681098,
                                         1.3862943611198906, 0.6931471805599453], rtol=1e-15)
    np.testing.assert_allclose(X[:, 10], [0.4, 0.3, 0.5, 0.2], rtol=1e-15)
    np.testing.assert_allclose(X[:, 11], [0.75, 0.0, 0.4, 0.5], rtol=1e-15, atol=1e-16)
    np.testing.assert_array_equal(X[:, 12:], 0.0)


def test_forward_by_hand():
    """Weights chosen so that each step can be followed by hand: layer 1 copies the constant
    feature (input column 8) to hidden unit 0 and the aggregated constant (A_hat 1, input column
    64 + 8) to unit 1; layers 2 and 3 copy units 0 and 1 through the H half of [H, A_hat H]; the
    heads read Z_i = (1, t_i) and y_i = 2 + 3 t_i + 0.5, with t = A_hat 1 (row sums):
      t0 = A01 + A02 = 0.7358887300947708,   t1 = A01 + A12 = 0.030476244847651746,
      t2 = A02 + A12 + A23 = 0.5052424717696348,  t3 = A23 = 0.31622776601683794."""
    inst, (ei, ej, w) = _tiny()
    A, _ = G.normalized_adjacency(inst.n, ei, ej, w)
    X = G.features(inst.n, ei, ej, w, seed=7)
    P = {k: np.zeros_like(v) for k, v in G.init_params(1).items()}
    P["theta0"][8, 0] = 1.0
    P["theta0"][G.HIDDEN + 8, 1] = 1.0
    for l in (1, 2):
        P[f"theta{l}"][0, 0] = 1.0
        P[f"theta{l}"][1, 1] = 1.0
    P["theta_u"][0, 0] = 1.0
    P["theta_u"][1, 1] = 1.0
    P["theta_y"][0] = 2.0
    P["theta_y"][1] = 3.0
    P["b_y"][0] = 0.5
    U, y, _ = G.forward(P, X, A, r=3)
    t = np.array([0.7358887300947708, 0.030476244847651746, 0.5052424717696348,
                  0.31622776601683794])
    nrm = np.sqrt(1.0 + t * t)
    np.testing.assert_allclose(U[:, 0], 1.0 / nrm, rtol=1e-14)
    np.testing.assert_allclose(U[:, 1], t / nrm, rtol=1e-14)
    np.testing.assert_array_equal(U[:, 2], 0.0)
    np.testing.assert_allclose(y, 2.0 + 3.0 * t + 0.5, rtol=1e-14)
