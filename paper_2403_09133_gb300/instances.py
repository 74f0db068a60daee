"""Seeded synthetic SDP instances shaped like the paper's workloads.

This module only *generates problem data* (graphs, weights, samples) and writes
them as the linear-SDP triple (C, {A_i}, b) of Section 1 (eq. prob:linear-SDP).
It holds none of the solver's arithmetic, so both the CUDA library's tests and
the FP64 CPU oracle can draw identical inputs from it.

Conventions (shared by the C ABI and the oracle):
  * symmetric matrices are given as upper triplets (row <= col); an off-diagonal
    triplet (i, j, a) stands for both (i, j) and (j, i), so
    <A, X> = sum_diag a_ii X_ii + 2 sum_{i<j} a_ij X_ij;
  * constraint k is the set of triplets whose ``con`` equals k.

Workload families:
  * MaxCut SDP (Section 5.3): C = -L(G, w)/4, A_i = e_i e_i^T, b = 1.  The paper
    states the max form <L/4, X>; the min form used here has objective
    -(SDP value).
  * Matrix completion (Section 5.4): X in S^{n1+n2}, constraint k fixes the entry
    (p, n1+q) of the off-diagonal block through <A_k, X> = 2 X_{p,n1+q} = 2 M_pq,
    C = I.
  * General constraints: the Lovasz theta SDP (tr X = 1 has n entries), the minimum
    bisection relaxation (<e e^T, X> = 0 as a rank-one term) and sensor network
    localisation (rank-one distance constraints, Section 2.3).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np


@dataclass
class SDPInstance:
    """Linear SDP data as upper-triangular triplets (see module docstring)."""

    n: int
    m: int
    C_row: np.ndarray
    C_col: np.ndarray
    C_val: np.ndarray
    A_con: np.ndarray
    A_row: np.ndarray
    A_col: np.ndarray
    A_val: np.ndarray
    b: np.ndarray
    # rank-one terms: A_con += scale * a a^T with a given sparsely by (idx, vals)
    rank1: List[Tuple[int, np.ndarray, np.ndarray, float]] = field(default_factory=list)
    kind: str = "general"          # "maxcut" | "mc" | "general"
    name: str = ""
    # graph data kept for certificates (MaxCut only)
    edges: Optional[np.ndarray] = None
    weights: Optional[np.ndarray] = None
    # matrix-completion ground truth (MC only)
    mc_P: Optional[np.ndarray] = None
    mc_Q: Optional[np.ndarray] = None
    mc_n1: int = 0

    def __post_init__(self):
        self.C_row = np.ascontiguousarray(self.C_row, dtype=np.int32)
        self.C_col = np.ascontiguousarray(self.C_col, dtype=np.int32)
        self.C_val = np.ascontiguousarray(self.C_val, dtype=np.float64)
        self.A_con = np.ascontiguousarray(self.A_con, dtype=np.int32)
        self.A_row = np.ascontiguousarray(self.A_row, dtype=np.int32)
        self.A_col = np.ascontiguousarray(self.A_col, dtype=np.int32)
        self.A_val = np.ascontiguousarray(self.A_val, dtype=np.float64)
        self.b = np.ascontiguousarray(self.b, dtype=np.float64)


# --------------------------------------------------------------------------------------
# graphs
# --------------------------------------------------------------------------------------
def _sorted_unique(x: np.ndarray) -> np.ndarray:
    """Sorted distinct values (the same set np.unique returns; sort + adjacent difference)."""
    s = np.sort(x, kind="stable")
    if s.size == 0:
        return s
    keep = np.empty(s.size, dtype=bool)
    keep[0] = True
    np.not_equal(s[1:], s[:-1], out=keep[1:])
    return s[keep]


def erdos_renyi_edges(n: int, num_edges: int, rng: np.random.Generator) -> np.ndarray:
    """G(n, M): ``num_edges`` distinct unordered pairs drawn uniformly (i < j)."""
    total = n * (n - 1) // 2
    if num_edges > total:
        raise ValueError("too many edges for G(n, M)")
    chosen = np.empty(0, dtype=np.int64)
    while chosen.size < num_edges:
        need = num_edges - chosen.size
        i = rng.integers(0, n, size=2 * need + 16, dtype=np.int64)
        j = rng.integers(0, n, size=2 * need + 16, dtype=np.int64)
        keep = i != j
        lo = np.minimum(i[keep], j[keep])
        hi = np.maximum(i[keep], j[keep])
        chosen = _sorted_unique(np.concatenate([chosen, lo * n + hi]))
    # a uniformly random M-subset of the distinct pairs found
    pick = rng.permutation(chosen.size)[:num_edges]
    codes = np.sort(chosen[pick])
    return np.stack([codes // n, codes % n], axis=1).astype(np.int64)


def torus_edges(a: int, b: int) -> np.ndarray:
    """Edges of the a x b toroidal grid (Cartesian product of two cycles), i < j."""
    idx = np.arange(a * b).reshape(a, b)
    right = np.stack([idx.ravel(), np.roll(idx, -1, axis=1).ravel()], axis=1)
    down = np.stack([idx.ravel(), np.roll(idx, -1, axis=0).ravel()], axis=1)
    e = np.concatenate([right, down])
    e = np.stack([e.min(1), e.max(1)], axis=1)
    e = np.unique(e, axis=0)          # a or b equal to 2 would create duplicates
    return e[e[:, 0] != e[:, 1]]


def cycle_edges(n: int) -> np.ndarray:
    i = np.arange(n)
    e = np.stack([i, (i + 1) % n], axis=1)
    e = np.stack([e.min(1), e.max(1)], axis=1)
    return np.unique(e, axis=0)


def complete_edges(n: int) -> np.ndarray:
    i, j = np.triu_indices(n, 1)
    return np.stack([i, j], axis=1).astype(np.int64)


# --------------------------------------------------------------------------------------
# MaxCut SDP (Section 5.3)
# --------------------------------------------------------------------------------------
def maxcut_sdp(n: int, edges: np.ndarray, w: np.ndarray, name: str = "") -> SDPInstance:
    """min <C,X> with C = -L(G,w)/4, X_ii = 1 (A_i = e_i e_i^T, b_i = 1)."""
    edges = np.asarray(edges, dtype=np.int64)
    w = np.asarray(w, dtype=np.float64)
    deg = np.zeros(n)
    np.add.at(deg, edges[:, 0], w)
    np.add.at(deg, edges[:, 1], w)
    # Laplacian: L_ii = sum_k w_ik, L_ij = -w_ij  ->  C = -L/4
    diag_rows = np.arange(n)
    C_row = np.concatenate([diag_rows, edges[:, 0]])
    C_col = np.concatenate([diag_rows, edges[:, 1]])
    C_val = np.concatenate([-deg / 4.0, w / 4.0])
    keep = C_val != 0.0
    return SDPInstance(
        n=n, m=n,
        C_row=C_row[keep], C_col=C_col[keep], C_val=C_val[keep],
        A_con=np.arange(n), A_row=np.arange(n), A_col=np.arange(n), A_val=np.ones(n),
        b=np.ones(n), kind="maxcut", name=name, edges=edges, weights=w,
    )


def maxcut_er(n: int, avg_degree: float, seed: int, name: str = "") -> SDPInstance:
    """Erdos-Renyi G(n, M = floor(n d / 2)) with unit weights."""
    rng = np.random.default_rng(seed)
    M = int(np.floor(n * avg_degree / 2))
    e = erdos_renyi_edges(n, M, rng)
    return maxcut_sdp(n, e, np.ones(len(e)), name or f"er_n{n}_d{avg_degree:g}_s{seed}")


def maxcut_torus(a: int, b: int, seed: Optional[int], name: str = "") -> SDPInstance:
    """a x b toroidal grid; weights uniform in {-1,+1} (seed given) or all 1 (seed None)."""
    e = torus_edges(a, b)
    if seed is None:
        w = np.ones(len(e))
    else:
        rng = np.random.default_rng(seed)
        w = rng.choice(np.array([-1.0, 1.0]), size=len(e))
    return maxcut_sdp(a * b, e, w, name or f"torus_{a}x{b}_s{seed}")


def maxcut_complete(n: int) -> SDPInstance:
    e = complete_edges(n)
    return maxcut_sdp(n, e, np.ones(len(e)), f"K{n}")


def maxcut_cycle(n: int) -> SDPInstance:
    e = cycle_edges(n)
    return maxcut_sdp(n, e, np.ones(len(e)), f"C{n}")


# --------------------------------------------------------------------------------------
# Matrix completion SDP (Section 5.4)
# --------------------------------------------------------------------------------------
def matrix_completion(n1: int, n2: int, rank: int, num_samples: int, seed: int,
                      name: str = "") -> SDPInstance:
    """Z block fixed to samples of M = P Q^T, P, Q i.i.d. N(0,1); C = I.

    Sampled positions are distinct, uniform over the n1*n2 grid, sorted row-major.
    """
    rng = np.random.default_rng(seed)
    P = rng.standard_normal((n1, rank))
    Q = rng.standard_normal((n2, rank))
    total = n1 * n2
    if num_samples > total:
        raise ValueError("more samples than entries")
    codes = np.empty(0, dtype=np.int64)
    while codes.size < num_samples:
        need = num_samples - codes.size
        draw = rng.integers(0, total, size=need + need // 8 + 16, dtype=np.int64)
        codes = _sorted_unique(np.concatenate([codes, draw]))
    codes = np.sort(codes[rng.permutation(codes.size)[:num_samples]])
    p = codes // n2
    q = codes % n2
    Mpq = np.einsum("ij,ij->i", P[p], Q[q])
    n = n1 + n2
    m = num_samples
    return SDPInstance(
        n=n, m=m,
        C_row=np.arange(n), C_col=np.arange(n), C_val=np.ones(n),
        A_con=np.arange(m), A_row=p, A_col=n1 + q, A_val=np.ones(m),
        b=2.0 * Mpq, kind="mc", name=name or f"mc_{n1}x{n2}_r{rank}_m{m}_s{seed}",
        mc_P=P, mc_Q=Q, mc_n1=n1,
    )


# --------------------------------------------------------------------------------------
# General constraints: multi-entry (theta), rank-one with a long vector (bisection) and
# rank-one with short vectors (sensor network localisation, Section 2.3)
# --------------------------------------------------------------------------------------
def lovasz_theta(n: int, edges: np.ndarray, name: str = "") -> SDPInstance:
    """min <-J, X> s.t. tr X = 1 (one constraint with n diagonal entries), X_ij = 0 for every
    edge (i, j) (b = 0), X PSD: minus the Lovasz theta number of G (the SDPLIB theta family of
    Section 5.5's general benchmarks).  C = -J is dense: every upper triplet has value -1."""
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    iu, ju = np.triu_indices(n)
    m = 1 + len(edges)
    return SDPInstance(
        n=n, m=m,
        C_row=iu, C_col=ju, C_val=-np.ones(len(iu)),
        A_con=np.concatenate([np.zeros(n, dtype=np.int64), 1 + np.arange(len(edges))]),
        A_row=np.concatenate([np.arange(n), edges[:, 0]]),
        A_col=np.concatenate([np.arange(n), edges[:, 1]]),
        A_val=np.ones(n + len(edges)),
        b=np.concatenate([[1.0], np.zeros(len(edges))]),
        kind="general", name=name or f"theta_n{n}_e{len(edges)}", edges=edges,
    )


def graph_bisection(n: int, edges: np.ndarray, w: np.ndarray, name: str = "",
                    small_side: Optional[int] = None) -> SDPInstance:
    """min <L(G, w)/4, X> s.t. X_ii = 1 and <e e^T / n^2, X> = ((n - 2k) / n)^2 (a rank-one
    constraint whose vector is all ones, scaled like the diagonal ones), X PSD: the relaxation
    of the minimum cut into sides of k and n - k vertices (x in {-1, 1}^n with e^T x = n - 2k).
    k = n/2 (the default) is the bisection of the SDPLIB gpp family (Section 5.5); there
    <e e^T, X> = 0 leaves no strictly feasible X."""
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    w = np.asarray(w, dtype=np.float64)
    k = n // 2 if small_side is None else int(small_side)
    deg = np.zeros(n)
    np.add.at(deg, edges[:, 0], w)
    np.add.at(deg, edges[:, 1], w)
    C_row = np.concatenate([np.arange(n), edges[:, 0]])
    C_col = np.concatenate([np.arange(n), edges[:, 1]])
    C_val = np.concatenate([deg / 4.0, -w / 4.0])
    keep = C_val != 0.0
    return SDPInstance(
        n=n, m=n + 1,
        C_row=C_row[keep], C_col=C_col[keep], C_val=C_val[keep],
        A_con=np.arange(n), A_row=np.arange(n), A_col=np.arange(n), A_val=np.ones(n),
        b=np.concatenate([np.ones(n), [(float(n - 2 * k) / n) ** 2]]),
        rank1=[(n, np.arange(n), np.ones(n), 1.0 / (float(n) * n))],
        kind="general", name=name or f"partition_n{n}_k{k}", edges=edges, weights=w,
    )


def maxcut_rank_one(n: int, avg_degree: float, count: int, support: int, seed: int,
                    name: str = "") -> SDPInstance:
    """The Erdos-Renyi MaxCut SDP of `maxcut_er` plus `count` rank-one constraints
    <a_t a_t^T, X> / ||a_t||^2 = 1, a_t Gaussian on `support` random rows: X = I meets them
    strictly inside the cone.  Rank-one constraints with long vectors (the `support` entries of
    a_t expand into support (support + 1) / 2 matrix entries)."""
    base = maxcut_er(n, avg_degree, seed)
    rng = np.random.default_rng(seed + 1000)
    rank1 = []
    for t in range(count):
        idx = np.sort(rng.choice(n, size=support, replace=False))
        a = rng.standard_normal(support)
        rank1.append((n + t, idx, a, 1.0 / float(a @ a)))
    base.rank1 = rank1
    base.m = n + count
    base.b = np.concatenate([base.b, np.ones(count)])
    base.kind = "general"
    base.name = name or f"maxcut_r1_n{n}_q{count}_s{support}_seed{seed}"
    return base


def sensor_network(num_sensors: int, num_anchors: int, dim: int, radius: float, seed: int,
                   name: str = "") -> SDPInstance:
    """The SDP relaxation of sensor network localisation in the form Section 2.3 gives with its
    escape example: Z in S^{d+n} = [[I, X], [X^T, Y]], Z_{1:d,1:d} = I (d diagonal and
    d(d-1)/2 zero off-diagonal constraints), <(0; e_i - e_j)(0; e_i - e_j)^T, Z> = d_ij^2 for
    sensor pairs closer than `radius`, <(a_k; -e_j)(a_k; -e_j)^T, Z> = d_kj^2 for
    anchor-sensor pairs closer than `radius` (rank-one constraints), C = 0.  Sensors and
    anchors uniform in [-0.5, 0.5]^d; distances exact, so Z with X the true positions and
    Y = X^T X is feasible.  The true positions are kept in mc_P (d x n) for checks."""
    rng = np.random.default_rng(seed)
    d, ns = dim, num_sensors
    x = rng.uniform(-0.5, 0.5, size=(ns, d))
    a = rng.uniform(-0.5, 0.5, size=(num_anchors, d))
    A_con, A_row, A_col, A_val, b = [], [], [], [], []
    m = 0
    for k in range(d):
        for l in range(k, d):
            A_con.append(m); A_row.append(k); A_col.append(l); A_val.append(1.0)
            b.append(1.0 if k == l else 0.0)
            m += 1
    rank1 = []
    for i in range(ns):
        for j in range(i + 1, ns):
            dist2 = float(np.sum((x[i] - x[j]) ** 2))
            if dist2 < radius * radius:
                rank1.append((m, np.array([d + i, d + j]), np.array([1.0, -1.0]), 1.0))
                b.append(dist2)
                m += 1
    for k in range(num_anchors):
        for j in range(ns):
            dist2 = float(np.sum((a[k] - x[j]) ** 2))
            if dist2 < radius * radius:
                idx = np.concatenate([np.arange(d), [d + j]])
                rank1.append((m, idx, np.concatenate([a[k], [-1.0]]), 1.0))
                b.append(dist2)
                m += 1
    n = d + ns
    return SDPInstance(
        n=n, m=m,
        C_row=np.zeros(0), C_col=np.zeros(0), C_val=np.zeros(0),
        A_con=np.array(A_con), A_row=np.array(A_row), A_col=np.array(A_col),
        A_val=np.array(A_val), b=np.array(b), rank1=rank1,
        kind="general", name=name or f"snl_n{ns}_a{num_anchors}_d{d}_s{seed}",
        mc_P=x.T.copy(),
    )


# --------------------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------------------
def workload_er500() -> SDPInstance:
    """MaxCut, Erdos-Renyi n=500, average degree 8 (M=2000), unit weights, seed 1."""
    return maxcut_er(500, 8.0, seed=1, name="maxcut_er_n500_d8")


def workload_torus141() -> SDPInstance:
    """MaxCut, 141x141 toroidal grid (n=m=19,881), weights uniform in {-1,+1}, seed 2."""
    return maxcut_torus(141, 141, seed=2, name="maxcut_torus_141x141_pm1")


def workload_batch(count: int = 512, seed0: int = 1000, n_lo: int = 64, n_hi: int = 2048,
                   d_lo: float = 3.0, d_hi: float = 12.0) -> List[SDPInstance]:
    """Uneven batch of ER MaxCuts: n ~ U[n_lo, n_hi], degree ~ U[d_lo, d_hi], seeds seed0+i."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        n = int(rng.integers(n_lo, n_hi + 1))
        d = float(rng.uniform(d_lo, d_hi))
        out.append(maxcut_er(n, d, seed=seed0 + i, name=f"batch_{i}"))
    return out


def workload_mc(n1: int = 20000, n2: int = 20000, rank: int = 5,
                num_samples: int = 15_694_167, seed: int = 5) -> SDPInstance:
    """Matrix completion, n = n1 + n2; the full size is n = 40,000 with 15,694,167 samples."""
    return matrix_completion(n1, n2, rank, num_samples, seed, name=f"mc_{n1 + n2}")
