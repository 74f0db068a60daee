"""Matrix completion at the size of the paper's largest MC instance: n = 40,000
(n1 = n2 = 20,000), rank-5 M = P Q^T, 15,694,167 observed entries, r = 24 (Section 5.4's
SDP; the paper's MC_40000).

Parity: the FP32 Hessian apply against the oracle on every row (within FP32 rounding of the
terms each row sums); the solve against what the problem fixes (exact recovery: objective
2 ||M||_* to 1e-6, the final test at 1e-6, and Z = M on entries never observed)."""
import numpy as np
import pytest

from oracle import SDP
import oracle.lorads as OL
from paper_2403_09133_gb300 import instances as I
from paper_2403_09133_gb300 import lorads as L

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def mc():
    inst = I.workload_mc()
    return inst


def nuclear_norm_rank5(P, Q):
    # singular values of P Q^T: sigma^2 = eigenvalues of (P^T P)(Q^T Q)
    ev = np.linalg.eigvals((P.T @ P) @ (Q.T @ Q)).real
    return float(np.sqrt(np.clip(ev, 0, None)).sum())


def test_mc_full_size_hessian_parity(cuda, mc):
    torch = cuda
    sdp = SDP.from_instance(mc)
    r, ld = 24, 24
    rng = np.random.default_rng(5)
    V = rng.standard_normal((mc.n, r)).astype(np.float32).astype(np.float64)
    P = rng.standard_normal((mc.n, r)).astype(np.float32).astype(np.float64)
    prob = L.Problem(mc)
    dV = torch.tensor(V, dtype=torch.float32, device="cuda")
    dP = torch.tensor(P, dtype=torch.float32, device="cuda")
    out = torch.empty((mc.n, ld), dtype=torch.float32, device="cuda")
    assert L.lorads_op_hessian(prob.handle, L.LORADS_PREC_MIXED, r, ld, 50.0, 1.0, dV, dP, out) == 0
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    want = OL.hessian_apply(sdp, V, P, 50.0, 1.0)
    rel = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert rel <= 1e-5, rel
    # every row, against the size of the terms it sums: FP32 rounding of each term
    # rho a q W_k (q = a (P_j.W_k + P_k.W_j)) bounds the row's error by a few units of
    # 6e-8 times rho sum_k |a| (|P_j||W_k| + |P_k||W_j|) |W_k| + gamma |P_j|
    nP, nV = np.linalg.norm(P, axis=1), np.linalg.norm(V, axis=1)
    A = sdp.At_matrix(np.ones(sdp.m))
    absA = abs(A)
    scale = 50.0 * (nP * (absA @ (nV * nV)) + nV * (absA @ (nP * nV))) + 1.0 * nP
    err = np.linalg.norm(got - want, axis=1)
    assert np.all(err <= 1e-5 * scale), np.max(err / scale)
    prob.close()


def test_mc_full_size_solve_recovers_M(cuda, mc):
    prob = L.Problem(mc)
    res = prob.solve(precision=L.LORADS_PREC_MIXED, switch_tol=1e-3, h=2.5, time_limit_s=240.0)
    assert res["status"] == 0, L.lorads_status_string(res["status"])
    want = 2.0 * nuclear_norm_rank5(mc.mc_P, mc.mc_Q)
    assert abs(res["objective"] - want) <= 1e-6 * want, (res["objective"], want)
    assert res["r_P"] <= 1e-6 and res["r_D"] <= 1e-6 and abs(res["gap"]) <= 1e-6
    sol = prob.solution()
    prob.close()
    Uh = sol["U_hat"]
    rng = np.random.default_rng(11)
    p = rng.integers(0, mc.mc_n1, 20000)
    q = rng.integers(0, mc.n - mc.mc_n1, 20000)
    Z = np.einsum("ij,ij->i", Uh[p], Uh[mc.mc_n1 + q])
    M = np.einsum("ij,ij->i", mc.mc_P[p], mc.mc_Q[q])
    assert np.linalg.norm(Z - M) <= 1e-3 * np.linalg.norm(M)
