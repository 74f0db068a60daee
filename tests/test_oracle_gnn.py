"""Pins for the oracle's learned warm start: its backward pass against central finite
differences of the loss (every parameter block), and the output constraint X_jj = 1."""
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


@pytest.mark.parametrize("name", ["theta0", "b0", "theta1", "theta2", "b2", "theta_u", "theta_y", "b_y"])
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
