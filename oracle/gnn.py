"""FP64 CPU oracle -- the learned warm start (message-passing network) and its gradients.

TEST INFRASTRUCTURE ONLY (imported by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``).

The paper's Phase I is the Burer-Monteiro method (Section 4.1) and its conclusion names
better warm starts as future work (Section 6).  This network proposes the Phase II start
(U_0, y_0) for a MaxCut graph instead; Phase II (Algorithm 1) then runs unchanged from
U = V = U_0, lambda = -y_0.  Definitions (written out plainly; the CUDA side implements the
same definitions independently):

  graph        w_ij = C_ij for the off-diagonal entries of C (MaxCut: C = -L/4, so w = w_graph/4)
  normalised   A_hat_ij = w_ij / sqrt(d_i d_j),  d_i = 1 + sum_j |w_ij|
  features     X0_i = [z_i (8 standard normals, SplitMix64 stream of the seed),
                       1, log(1 + deg_i), d_i / 10, s_i, 0 ...] in R^64, s_i = sum_j w_ij / d_i
  layers l=1..3  H_l = relu([H_{l-1}, A_hat H_{l-1}] Theta_l + b_l),  Theta_l in R^{128 x 64}
  heads        Z = H_3 Theta_u (64 x r), U0_i = Z_i / ||Z_i||;  y0 = H_3 theta_y + b_y
  loss         (1/|E|) sum_{(i,j) in E} (U0_i . U0_j - Xs_ij)^2 + beta (1/n) sum_i (y0_i - ys_i)^2
               (E = the off-diagonal entries of C; Xs = U_hat U_hat^T of a solved instance,
               ys its dual: rotation-invariant targets, since U_0 is defined up to rotation)
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from .lorads import normal_matrix, stream_key

HIDDEN = 64
LAYERS = 3
RMAX = 16
NRAND = 8
BETA = 0.1


def graph_of(inst):
    """Edge list (i < j) and weights w_ij = C_ij from the off-diagonal triplets of C."""
    off = inst.C_row != inst.C_col
    return (np.asarray(inst.C_row[off], np.int64), np.asarray(inst.C_col[off], np.int64),
            np.asarray(inst.C_val[off], np.float64))


def normalized_adjacency(n, ei, ej, w):
    d = 1.0 + np.bincount(ei, np.abs(w), n) + np.bincount(ej, np.abs(w), n)
    vals = w / np.sqrt(d[ei] * d[ej])
    A = sp.coo_matrix((np.concatenate([vals, vals]), (np.concatenate([ei, ej]),
                                                       np.concatenate([ej, ei]))), shape=(n, n))
    return A.tocsr(), d


def features(n, ei, ej, w, seed):
    d = 1.0 + np.bincount(ei, np.abs(w), n) + np.bincount(ej, np.abs(w), n)
    deg = np.bincount(ei, minlength=n) + np.bincount(ej, minlength=n)
    s = (np.bincount(ei, w, n) + np.bincount(ej, w, n)) / d
    X = np.zeros((n, HIDDEN))
    X[:, :NRAND] = normal_matrix(stream_key(seed, 1000), n, NRAND)
    X[:, NRAND] = 1.0
    X[:, NRAND + 1] = np.log1p(deg)
    X[:, NRAND + 2] = d / 10.0
    X[:, NRAND + 3] = s
    return X


def init_params(seed):
    """Weights ~ N(0, 1/fan_in) from the SplitMix64 stream (stream ids 2000+), biases 0."""
    P = {}
    for l in range(LAYERS):
        P[f"theta{l}"] = normal_matrix(stream_key(seed, 2000 + l), 2 * HIDDEN, HIDDEN) / math.sqrt(2 * HIDDEN)
        P[f"b{l}"] = np.zeros(HIDDEN)
    P["theta_u"] = normal_matrix(stream_key(seed, 2100), HIDDEN, RMAX) / math.sqrt(HIDDEN)
    P["theta_y"] = normal_matrix(stream_key(seed, 2101), HIDDEN, 1)[:, 0] / math.sqrt(HIDDEN)
    P["b_y"] = np.zeros(1)
    return P


def forward(P, X0, A, r):
    cache = {"H": [X0], "S": [], "AH": []}
    H = X0
    for l in range(LAYERS):
        AH = A @ H
        S = np.concatenate([H, AH], axis=1) @ P[f"theta{l}"] + P[f"b{l}"]
        H = np.maximum(S, 0.0)
        cache["AH"].append(AH)
        cache["S"].append(S)
        cache["H"].append(H)
    Z = H @ P["theta_u"][:, :r]
    nz = np.linalg.norm(Z, axis=1)
    U = Z / nz[:, None]
    y = H @ P["theta_y"] + P["b_y"][0]
    cache.update(Z=Z, nz=nz, U=U, y=y)
    return U, y, cache


def loss_and_grad(P, X0, A, ei, ej, Xs, ys, r):
    U, y, c = forward(P, X0, A, r)
    n = U.shape[0]
    E = len(ei)
    g = np.einsum("ij,ij->i", U[ei], U[ej]) - Xs
    ry = y - ys
    loss = float(g @ g) / E + BETA * float(ry @ ry) / n
    # d loss / d U
    dU = np.zeros_like(U)
    coef = 2.0 * g / E
    np.add.at(dU, ei, coef[:, None] * U[ej])
    np.add.at(dU, ej, coef[:, None] * U[ei])
    # through U = Z / ||Z||
    dZ = (dU - U * np.sum(U * dU, axis=1, keepdims=True)) / c["nz"][:, None]
    H3 = c["H"][-1]
    G = {}
    G["theta_u"] = np.zeros_like(P["theta_u"])
    G["theta_u"][:, :r] = H3.T @ dZ
    dy = 2.0 * BETA * ry / n
    G["theta_y"] = H3.T @ dy
    G["b_y"] = np.array([dy.sum()])
    dH = dZ @ P["theta_u"][:, :r].T + np.outer(dy, P["theta_y"])
    for l in reversed(range(LAYERS)):
        dS = dH * (c["S"][l] > 0)
        Hin = c["H"][l]
        cat = np.concatenate([Hin, c["AH"][l]], axis=1)
        G[f"theta{l}"] = cat.T @ dS
        G[f"b{l}"] = dS.sum(axis=0)
        dcat = dS @ P[f"theta{l}"].T
        dH = dcat[:, :HIDDEN] + A.T @ dcat[:, HIDDEN:]
    return loss, G, U, y


def flatten(P):
    """Parameter dict -> the flat FP32 layout of the C ABI (Theta_l, b_l, Theta_u, theta_y, b_y)."""
    parts = []
    for l in range(LAYERS):
        parts += [P[f"theta{l}"].reshape(-1), P[f"b{l}"]]
    parts += [P["theta_u"].reshape(-1), P["theta_y"], P["b_y"]]
    return np.concatenate(parts)


def unflatten(v):
    P = {}
    o = 0
    for l in range(LAYERS):
        P[f"theta{l}"] = v[o:o + 2 * HIDDEN * HIDDEN].reshape(2 * HIDDEN, HIDDEN).astype(np.float64)
        o += 2 * HIDDEN * HIDDEN
        P[f"b{l}"] = v[o:o + HIDDEN].astype(np.float64)
        o += HIDDEN
    P["theta_u"] = v[o:o + HIDDEN * RMAX].reshape(HIDDEN, RMAX).astype(np.float64)
    o += HIDDEN * RMAX
    P["theta_y"] = v[o:o + HIDDEN].astype(np.float64)
    o += HIDDEN
    P["b_y"] = v[o:o + 1].astype(np.float64)
    return P
