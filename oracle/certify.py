"""FP64 CPU oracle -- certificates used to pin the solver's output.

TEST INFRASTRUCTURE ONLY (imported by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``).

  * lambda_min(C - A^T y): the dual-infeasibility measure of Appendix B (its "sigma_min"
    of a symmetric matrix read as the smallest eigenvalue); dense LAPACK for small n,
    ARPACK Lanczos otherwise (shift-invert where plain Lanczos does not converge).
  * exhaustive max cut for n <= 20 (the Goemans-Williamson sandwich
    0.878 SDP <= maxcut <= SDP needs nonnegative weights).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .sdp import SDP


def _sparse_min_eig(S):
    """Smallest eigenpair of a large sparse symmetric S: implicitly restarted Lanczos (ARPACK)
    with a 128-vector basis; where it does not converge (a cluster of eigenvalues at the bottom
    of the spectrum, as at the dual of a degenerate SDP), ARPACK in shift-invert mode about a
    shift 1e-2 below the best estimate, which returns the eigenvalue nearest the shift."""
    n = S.shape[0]
    ncv = min(n - 1, 128)
    try:
        w, Z = spla.eigsh(S, k=1, which="SA", ncv=ncv, tol=1e-10, maxiter=20000)
        return float(w[0]), Z[:, 0]
    except spla.ArpackNoConvergence as err:
        est = float(err.eigenvalues[0]) if len(err.eigenvalues) else 0.0
    sigma = min(est, 0.0) - 1e-2
    w, Z = spla.eigsh(sp.csc_matrix(S), k=1, sigma=sigma, which="LM", tol=1e-12)
    return float(w[0]), Z[:, 0]


def min_eig_dual_slack(sdp: SDP, y, dense_limit: int = 2500) -> float:
    S = sdp.dual_slack(y)
    if sdp.n <= dense_limit:
        Sd = S.toarray() if sp.issparse(S) else np.asarray(S)
        return float(np.linalg.eigvalsh(0.5 * (Sd + Sd.T))[0])
    return _sparse_min_eig(S)[0]


def min_eig_pair_dual_slack(sdp: SDP, y, dense_limit: int = 2500):
    """(lambda_min, unit eigenvector) of S = C - A^T y."""
    S = sdp.dual_slack(y)
    if sdp.n <= dense_limit:
        Sd = S.toarray() if sp.issparse(S) else np.asarray(S)
        w, Z = np.linalg.eigh(0.5 * (Sd + Sd.T))
        return float(w[0]), Z[:, 0]
    lam, z = _sparse_min_eig(S)
    return lam, z / np.linalg.norm(z)


def exhaustive_maxcut(n: int, edges, w) -> float:
    """max over x in {-1,1}^n of sum_{(i,j)} w_ij (1 - x_i x_j)/2, with x_0 fixed."""
    if n > 22:
        raise ValueError("exhaustive max cut is for tiny graphs only")
    edges = np.asarray(edges, dtype=np.int64)
    w = np.asarray(w, dtype=np.float64)
    best = -np.inf
    # enumerate the 2^(n-1) cuts with vertex 0 on side +1, in chunks
    free = n - 1
    chunk_bits = min(free, 16)
    low = np.arange(1 << chunk_bits, dtype=np.int64)
    for hi in range(1 << (free - chunk_bits)):
        codes = (hi << chunk_bits) | low
        bits = (codes[:, None] >> np.arange(free)[None, :]) & 1
        x = np.concatenate([np.ones((len(codes), 1)), 1.0 - 2.0 * bits], axis=1)
        cut = ((1.0 - x[:, edges[:, 0]] * x[:, edges[:, 1]]) * 0.5) @ w
        best = max(best, float(cut.max()))
    return best
