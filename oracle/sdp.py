"""FP64 CPU oracle -- the linear maps of the linear SDP.

TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow, obviously-correct restatement
of the paper, used to check the CUDA library.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the library never does.

Problem (Section 1, eq. prob:linear-SDP):
    min <C, X>  s.t.  A(X) = b,  X PSD,   A(X) = (<A_1, X>, ..., <A_m, X>).
With the bilinear split X = U V^T (Section 2.1, eq. prob:split) the method only ever
needs three linear maps, written here as their definitions:

    A(U V^T)_i     = <A_i, U V^T>                (sampled dense-dense product)
    A^T(w) V       = (sum_i w_i A_i) V           (sparse times dense)
    <C, U V^T>     = sum_jk C_jk U_j . V_k

Every A_i and C is symmetric, stored as upper triplets (row <= col); an off-diagonal
triplet (r, c, a) stands for a at (r, c) and at (c, r).  Rank-one terms
A_i += s a a^T (the sensor-localisation constraints of Section 2.3) are kept as
(con, idx, vals, s).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


class SDP:
    """Container for (C, {A_i}, b) with the definitional linear maps."""

    def __init__(self, n, m, C_row, C_col, C_val, A_con, A_row, A_col, A_val, b,
                 rank1=()):
        self.n = int(n)
        self.m = int(m)
        self.C_row = np.asarray(C_row, dtype=np.int64)
        self.C_col = np.asarray(C_col, dtype=np.int64)
        self.C_val = np.asarray(C_val, dtype=np.float64)
        self.A_con = np.asarray(A_con, dtype=np.int64)
        self.A_row = np.asarray(A_row, dtype=np.int64)
        self.A_col = np.asarray(A_col, dtype=np.int64)
        self.A_val = np.asarray(A_val, dtype=np.float64)
        self.b = np.asarray(b, dtype=np.float64)
        if np.any(self.C_row > self.C_col) or np.any(self.A_row > self.A_col):
            raise ValueError("symmetric triplets must satisfy row <= col")
        self.A_off = self.A_row != self.A_col
        # C as a full symmetric sparse matrix (both triangles)
        off = self.C_row != self.C_col
        rows = np.concatenate([self.C_row, self.C_col[off]])
        cols = np.concatenate([self.C_col, self.C_row[off]])
        vals = np.concatenate([self.C_val, self.C_val[off]])
        self.C = sp.csr_matrix((vals, (rows, cols)), shape=(self.n, self.n))
        # rank-one terms as a sparse (terms x n) matrix whose row t is a_t^T
        self.r1_con = np.array([t[0] for t in rank1], dtype=np.int64)
        self.r1_scale = np.array([t[3] for t in rank1], dtype=np.float64)
        if len(rank1):
            rr = np.concatenate([np.full(len(t[1]), k) for k, t in enumerate(rank1)])
            cc = np.concatenate([np.asarray(t[1], dtype=np.int64) for t in rank1])
            vv = np.concatenate([np.asarray(t[2], dtype=np.float64) for t in rank1])
            self.R1 = sp.csr_matrix((vv, (rr, cc)), shape=(len(rank1), self.n))
        else:
            self.R1 = None

    @classmethod
    def from_instance(cls, inst):
        return cls(inst.n, inst.m, inst.C_row, inst.C_col, inst.C_val, inst.A_con,
                   inst.A_row, inst.A_col, inst.A_val, inst.b, inst.rank1)

    # ---------------------------------------------------------------- norms of the data
    @property
    def b_inf(self):
        return float(np.max(np.abs(self.b))) if self.m else 0.0

    @property
    def b_one(self):
        return float(np.sum(np.abs(self.b)))

    @property
    def C_fro(self):
        """||C||_F over the full symmetric matrix."""
        return float(sp.linalg.norm(self.C))

    @property
    def C_rowsum_max(self):
        """||C||_inf = max_j sum_k |C_jk| over the full symmetric matrix."""
        return float(np.abs(self.C).sum(axis=1).max()) if self.n else 0.0

    @property
    def c_one(self):
        """||c||_1, c = vec(C) (Appendix B)."""
        return float(np.abs(self.C).sum())

    # ---------------------------------------------------------------- the linear maps
    def A_of(self, U, V):
        """q_i = <A_i, U V^T> for i = 1..m (U, V are n x r)."""
        r, c, a = self.A_row, self.A_col, self.A_val
        # <E_rc + E_cr, U V^T> = U_r.V_c + U_c.V_r ;  <E_rr, U V^T> = U_r.V_r
        term = np.einsum("ij,ij->i", U[r], V[c])
        term = term + np.where(self.A_off, np.einsum("ij,ij->i", U[c], V[r]), 0.0)
        q = np.bincount(self.A_con, weights=a * term, minlength=self.m)
        if self.R1 is not None:
            # <s a a^T, U V^T> = s (a^T U) . (a^T V)
            aU = self.R1 @ U
            aV = self.R1 @ V
            q = q + np.bincount(self.r1_con, weights=self.r1_scale * np.einsum("ij,ij->i", aU, aV),
                                minlength=self.m)
        return q

    def At_matrix(self, w):
        """The sparse symmetric matrix sum_i w_i A_i (rank-one terms excluded)."""
        coef = w[self.A_con] * self.A_val
        off = self.A_off
        rows = np.concatenate([self.A_row, self.A_col[off]])
        cols = np.concatenate([self.A_col, self.A_row[off]])
        vals = np.concatenate([coef, coef[off]])
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.n, self.n))

    def At_times(self, w, V):
        """A^T(w) V = (sum_i w_i A_i) V."""
        out = self.At_matrix(w) @ V
        if self.R1 is not None:
            # sum_t w_con(t) s_t a_t (a_t^T V)
            aV = self.R1 @ V
            out = out + self.R1.T @ ((w[self.r1_con] * self.r1_scale)[:, None] * aV)
        return np.asarray(out)

    def C_times(self, V):
        return np.asarray(self.C @ V)

    def C_inner(self, U, V):
        """<C, U V^T>."""
        return float(np.sum(U * (self.C @ V)))

    # ---------------------------------------------------------------- dense forms (tiny n)
    def dense_A(self, i):
        """A_i as a dense n x n matrix."""
        Ai = np.zeros((self.n, self.n))
        sel = self.A_con == i
        for r, c, a in zip(self.A_row[sel], self.A_col[sel], self.A_val[sel]):
            Ai[r, c] += a
            if r != c:
                Ai[c, r] += a
        if self.R1 is not None:
            for t in np.nonzero(self.r1_con == i)[0]:
                a = np.asarray(self.R1[t].todense()).ravel()
                Ai += self.r1_scale[t] * np.outer(a, a)
        return Ai

    def dense_C(self):
        return np.asarray(self.C.todense())

    def dual_slack(self, y):
        """S = C - A^T(y) as a sparse matrix (rank-one terms added densely if present)."""
        S = self.C - self.At_matrix(y)
        if self.R1 is not None:
            S = S.toarray()
            for t in range(self.R1.shape[0]):
                a = np.asarray(self.R1[t].todense()).ravel()
                S -= y[self.r1_con[t]] * self.r1_scale[t] * np.outer(a, a)
            return S
        return S
