"""Learned warm start on the GPU (tensor-core GEMMs, BF16 weights, FP32 accumulation) against
the FP64 oracle network with the same parameters: forward outputs and gradients."""
import numpy as np
import pytest

import oracle.gnn as G
from paper_2403_09133_gb300 import instances as I
from paper_2403_09133_gb300 import lorads as L

pytestmark = pytest.mark.gpu


def _bf16(x):
    """Round to BF16 (round to nearest even) and back, in numpy."""
    a = np.asarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def setup(cuda):
    inst = I.maxcut_er(300, 6.0, seed=5)         # 3 row tiles, the last one ragged
    ei, ej, w = G.graph_of(inst)
    A, _ = G.normalized_adjacency(inst.n, ei, ej, w)
    X0 = G.features(inst.n, ei, ej, w, seed=9)
    P = G.init_params(seed=4)
    # the GPU keeps BF16 operands: give both sides the same BF16-representable weights
    flat = _bf16(G.flatten(P)).astype(np.float32)
    P = G.unflatten(flat)
    g = L.lorads_gnn_create(1)
    assert L.lorads_gnn_set_params(g, flat) == 0
    assert L.lorads_gnn_load_graph(g, inst.n, ei, ej, w, 9) == 0
    yield inst, ei, ej, A, X0, P, g
    L.lorads_gnn_destroy(g)


def test_params_roundtrip(setup):
    *_, g = setup
    p = L.lorads_gnn_get_params(g)
    assert p.size == L.lorads_gnn_param_count() == G.flatten(G.init_params(1)).size


@pytest.mark.parametrize("r", [9, 16])
def test_forward_matches_oracle(setup, r):
    inst, ei, ej, A, X0, P, g = setup
    U, y = L.lorads_gnn_forward(g, inst.n, r)
    Uo, yo, _ = G.forward(P, X0, A, r)
    np.testing.assert_allclose(np.sum(U * U, axis=1), 1.0, rtol=1e-5)
    # about five BF16 roundings (2^-9 each) in sequence: measured 0.3-0.6 %
    assert np.linalg.norm(U - Uo) <= 2e-2 * np.linalg.norm(Uo)
    assert np.linalg.norm(y - yo) <= 2e-2 * np.linalg.norm(yo)


def test_gradients_match_oracle(setup):
    inst, ei, ej, A, X0, P, g = setup
    r = 9
    rng = np.random.default_rng(2)
    Xs = rng.uniform(-1, 1, len(ei))
    ys = rng.standard_normal(inst.n)
    loss, grads = L.lorads_gnn_train_step(g, r, Xs, ys, 0.0, want_grads=True)
    lo, Go, _, _ = G.loss_and_grad(P, X0, A, ei, ej, Xs, ys, r)
    assert abs(loss - lo) <= 2e-3 * abs(lo)           # measured <= 3e-4: the errors average out
    Gg = G.unflatten(grads)
    for name in ["theta0", "b0", "theta1", "b1", "theta2", "b2", "theta_u", "theta_y", "b_y"]:
        a, b = Gg[name], Go[name]
        if name == "theta_u":
            a, b = a[:, :r], b[:, :r]
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-12)
        # the first two layers' gradients cross every BF16 layer back (~15 roundings,
        # measured <= 2.1e-2); the rest pass through as many as the forward pass again
        tol = 3e-2 if name in ("theta0", "b0", "theta1", "b1") else 2e-2
        assert rel <= tol, (name, rel)


def test_training_reduces_loss(setup):
    inst, ei, ej, A, X0, P, g = setup
    r = 9
    rng = np.random.default_rng(3)
    Xs = rng.uniform(-0.5, 0.5, len(ei))
    ys = -1.0 - rng.uniform(0, 1, inst.n)
    l0, _ = L.lorads_gnn_train_step(g, r, Xs, ys, 0.0)
    for _ in range(60):
        L.lorads_gnn_train_step(g, r, Xs, ys, 3e-3)
    l1, _ = L.lorads_gnn_train_step(g, r, Xs, ys, 0.0)
    assert l1 < 0.7 * l0
