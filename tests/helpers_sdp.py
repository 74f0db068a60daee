"""Small random SDP instances for operator tests (general sparse + rank-one constraints)."""
import numpy as np

from paper_2403_09133_gb300.instances import SDPInstance


def random_general_sdp(n, m, nnz_per_con, rng, rank1_terms=0, diag_frac=0.3):
    con, row, col, val = [], [], [], []
    for i in range(m):
        for _ in range(nnz_per_con):
            a, b = sorted(rng.integers(0, n, size=2))
            if rng.random() < diag_frac:
                b = a
            con.append(i); row.append(a); col.append(b); val.append(rng.standard_normal())
    # C: random symmetric sparse
    cr, cc, cv = [], [], []
    for _ in range(3 * n):
        a, b = sorted(rng.integers(0, n, size=2))
        cr.append(a); cc.append(b); cv.append(rng.standard_normal())
    r1 = []
    for t in range(rank1_terms):
        idx = np.unique(rng.integers(0, n, size=3))
        r1.append((int(rng.integers(0, m)), idx, rng.standard_normal(len(idx)), float(rng.uniform(0.5, 2.0))))
    return SDPInstance(n=n, m=m, C_row=cr, C_col=cc, C_val=cv, A_con=con, A_row=row,
                       A_col=col, A_val=val, b=rng.standard_normal(m), rank1=r1)
