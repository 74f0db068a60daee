"""GPU operator parity: each C-ABI operator against the oracle's definition, element by
element, on the same seeded inputs (FP64 to 1e-12 relative, the FP32 operators to 1e-5
relative against the oracle evaluated on the FP32-rounded inputs).

Shapes span one to several 4-column chunks per lane (r from 1 to 64, teams of 1 to 8 lanes)
and ragged row counts; instances cover diagonal constraints (MaxCut), off-diagonal ones
(matrix completion) and signed edge weights."""
import numpy as np
import pytest

from oracle import SDP
import oracle.lorads as OL
from paper_2403_09133_gb300 import instances as I
from paper_2403_09133_gb300 import lorads as L

pytestmark = pytest.mark.gpu

INSTANCES = {
    "er": lambda: I.maxcut_er(777, 7.0, seed=21),
    "torus": lambda: I.maxcut_torus(23, 31, seed=4),
    "mc": lambda: I.matrix_completion(211, 173, 4, 6000, seed=8),
}
RANKS = [1, 3, 9, 15, 24, 33, 64]


def _pad(X, ld):
    out = np.zeros((X.shape[0], ld))
    out[:, : X.shape[1]] = X
    return out


def _abs_sdp(inst):
    """The instance with every value replaced by its absolute value."""
    return SDP.from_instance(I.SDPInstance(
        n=inst.n, m=inst.m, C_row=inst.C_row, C_col=inst.C_col, C_val=np.abs(inst.C_val),
        A_con=inst.A_con, A_row=inst.A_row, A_col=inst.A_col, A_val=np.abs(inst.A_val),
        b=inst.b, rank1=[(c, i, np.abs(a), abs(sc)) for c, i, a, sc in inst.rank1]))


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def problems(cuda):
    out = {}
    for k, f in INSTANCES.items():
        inst = f()
        out[k] = (inst, SDP.from_instance(inst), L.Problem(inst))
    yield out
    for _, _, p in out.values():
        p.close()


def _inputs(n, r, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, r)), rng.standard_normal((n, r))


@pytest.mark.parametrize("name", list(INSTANCES))
@pytest.mark.parametrize("r", RANKS)
@pytest.mark.parametrize("prec", [L.LORADS_PREC_FP64, L.LORADS_PREC_MIXED])
def test_sddmm(problems, cuda, name, r, prec):
    torch = cuda
    inst, sdp, prob = problems[name]
    ld = (r + 3) // 4 * 4
    U, V = _inputs(sdp.n, r, 100 + r)
    dt = torch.float64 if prec == L.LORADS_PREC_FP64 else torch.float32
    if prec == L.LORADS_PREC_MIXED:
        U, V = U.astype(np.float32).astype(np.float64), V.astype(np.float32).astype(np.float64)
    dU = torch.tensor(_pad(U, ld), dtype=dt, device="cuda")
    dV = torch.tensor(_pad(V, ld), dtype=dt, device="cuda")
    q = torch.full((sdp.m,), np.nan, dtype=torch.float64, device="cuda")
    assert L.lorads_op_sddmm(prob.handle, prec, r, ld, dU, dV, q) == 0
    torch.cuda.synchronize()
    want = sdp.A_of(U, V)
    tol = 1e-12 if prec == L.LORADS_PREC_FP64 else 1e-5
    got = q.cpu().numpy()
    scale = np.abs(sdp.A_val[np.argsort(sdp.A_con)]) * (
        np.linalg.norm(U[inst.A_row], axis=1) * np.linalg.norm(V[inst.A_col], axis=1) +
        np.linalg.norm(U[inst.A_col], axis=1) * np.linalg.norm(V[inst.A_row], axis=1))
    assert np.all(np.abs(got - want) <= tol * scale + 1e-300)


@pytest.mark.parametrize("name", list(INSTANCES))
@pytest.mark.parametrize("r", RANKS)
@pytest.mark.parametrize("prec", [L.LORADS_PREC_FP64, L.LORADS_PREC_MIXED])
def test_spmm(problems, cuda, name, r, prec):
    torch = cuda
    inst, sdp, prob = problems[name]
    ld = (r + 3) // 4 * 4
    V, _ = _inputs(sdp.n, r, 200 + r)
    w = np.random.default_rng(r).standard_normal(sdp.m)
    gamma = 0.75
    dt = torch.float64 if prec == L.LORADS_PREC_FP64 else torch.float32
    if prec == L.LORADS_PREC_MIXED:
        V = V.astype(np.float32).astype(np.float64)
    dV = torch.tensor(_pad(V, ld), dtype=dt, device="cuda")
    dw = torch.tensor(w, dtype=torch.float64, device="cuda")
    out = torch.full((sdp.n, ld), np.nan, dtype=dt, device="cuda")
    assert L.lorads_op_spmm(prob.handle, prec, r, ld, dw, gamma, dV, out) == 0
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    want = sdp.At_times(w, V) - sdp.C_times(V) + gamma * V
    assert np.all(got[:, r:] == 0.0)
    # element by element: each row's error against a bound on its terms (the same products on
    # absolute values and row norms, by Cauchy-Schwarz), scaled by the arithmetic's rounding
    sabs = _abs_sdp(inst)
    v = np.linalg.norm(V, axis=1)[:, None]
    bound = (sabs.At_times(np.abs(w), v) + sabs.C_times(v) + gamma * v).ravel()
    tol = 1e-12 if prec == L.LORADS_PREC_FP64 else 1e-5
    err = np.abs(got[:, :r] - want).max(axis=1)
    assert np.all(err <= tol * bound + 1e-300)


@pytest.mark.parametrize("name", list(INSTANCES))
@pytest.mark.parametrize("r", RANKS)
@pytest.mark.parametrize("prec", [L.LORADS_PREC_FP64, L.LORADS_PREC_MIXED])
def test_hessian(problems, cuda, name, r, prec):
    torch = cuda
    inst, sdp, prob = problems[name]
    ld = (r + 3) // 4 * 4
    V, P = _inputs(sdp.n, r, 300 + r)
    rho, gamma = 37.0, 1.25
    dt = torch.float64 if prec == L.LORADS_PREC_FP64 else torch.float32
    if prec == L.LORADS_PREC_MIXED:
        V, P = V.astype(np.float32).astype(np.float64), P.astype(np.float32).astype(np.float64)
    dV = torch.tensor(_pad(V, ld), dtype=dt, device="cuda")
    dP = torch.tensor(_pad(P, ld), dtype=dt, device="cuda")
    out = torch.full((sdp.n, ld), np.nan, dtype=dt, device="cuda")
    assert L.lorads_op_hessian(prob.handle, prec, r, ld, rho, gamma, dV, dP, out) == 0
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    want = OL.hessian_apply(sdp, V, P, rho, gamma)
    assert np.all(got[:, r:] == 0.0)
    tol = 1e-12 if prec == L.LORADS_PREC_FP64 else 1e-5
    assert _rel(got[:, :r], want) <= tol
    # row by row as well (every row, not only in norm)
    rown = np.linalg.norm(want, axis=1) + rho * np.linalg.norm(V, axis=1) ** 2 * np.linalg.norm(P, axis=1)
    assert np.all(np.linalg.norm(got[:, :r] - want, axis=1) <= 10 * tol * (rown + 1e-12))


def test_bad_ld_rejected(problems, cuda):
    torch = cuda
    _, sdp, prob = problems["er"]
    x = torch.zeros((sdp.n, 8), dtype=torch.float64, device="cuda")
    q = torch.zeros(sdp.m, dtype=torch.float64, device="cuda")
    assert L.lorads_op_sddmm(prob.handle, 0, 9, 8, x, x, q) == L.LORADS_ERR_ARG   # ld < r
    assert L.lorads_op_sddmm(prob.handle, 0, 5, 6, x, x, q) == L.LORADS_ERR_ARG   # ld % 4
    assert L.lorads_op_sddmm(prob.handle, 7, 4, 4, x, x, q) == L.LORADS_ERR_ARG   # precision
