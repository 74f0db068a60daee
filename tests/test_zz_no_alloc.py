"""lorads_solve_static: the allocation-free solve for callers that must not allocate device
memory while they solve (set-up allocates once; this call only uses a fixed device array
held by the library).  It must give the same answer as lorads_solve on the same problem,
call after call, on the one-CTA path and on the whole-GPU path, and device memory must not
change across it.  Collected last on purpose (file name) so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest

from paper_2403_09133_gb300 import instances as I
from paper_2403_09133_gb300 import lorads as L

pytestmark = pytest.mark.gpu

CASES = {
    # one CTA (n < 512): converges in ~1500 ADMM iterations
    "er100": (lambda: I.maxcut_er(100, 6.0, seed=3), {}),
    # the whole GPU (cooperative launch, grid barriers and partial sums in the fixed array);
    # capped so that both paths stop at the same iteration whatever the final test does
    "torus40": (lambda: I.maxcut_torus(40, 40, seed=4), {"max_admm_iter": 600}),
    # multi-entry constraints (tr X = 1 of the theta SDP): the chunk sums in the fixed array
    "theta60": (lambda: I.lovasz_theta(60, I.cycle_edges(60)), {"max_admm_iter": 200}),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec", [L.LORADS_PREC_FP64, L.LORADS_PREC_MIXED])
def test_static_solve_matches_lorads_solve_twice(cuda, case, prec):
    torch = cuda
    make, extra = CASES[case]
    inst = make()
    p = L.Problem(inst)
    prm = p.params(precision=prec, **extra)
    ref = L.lorads_solve(p.handle, prm).as_dict()          # assembles (allocates) once
    assert ref["status"] in (0, L.LORADS_ERR_MAXITER)
    sol = p.solution()
    r = sol["rank"]
    ldu = 64
    for call in range(2):
        U_hat = torch.full((inst.n, ldu), np.nan, dtype=torch.float64, device="cuda")
        y = torch.full((inst.m,), np.nan, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        res = L.lorads_solve_static(p.handle, prm, U_hat, ldu, y).as_dict()
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free_before, "device memory changed"
        assert res["status"] == ref["status"], (call, L.lorads_status_string(res["status"]))
        assert res["rank"] == r
        assert abs(res["objective"] - ref["objective"]) <= 1e-9 * abs(ref["objective"])
        assert res["admm_iters"] == ref["admm_iters"]
        assert res["cg_iters"] == ref["cg_iters"]
        got_U = U_hat[:, :r].cpu().numpy()
        np.testing.assert_allclose(got_U, sol["U_hat"], rtol=1e-9, atol=1e-12)
        assert torch.isnan(U_hat[:, r:]).all()              # columns past the rank untouched
        np.testing.assert_allclose(y.cpu().numpy(), sol["y"], rtol=1e-9, atol=1e-12)
    # the problem's own solution from lorads_solve is still there
    again = p.solution()
    np.testing.assert_array_equal(again["U_hat"], sol["U_hat"])
    p.close()


def test_static_solve_rejects_unassembled_and_oversized(cuda):
    torch = cuda
    small = L.Problem(I.maxcut_er(50, 4.0, seed=1))
    res = L.lorads_solve_static(small.handle, small.params())
    assert res.status == L.LORADS_ERR_STATE                  # assembling would allocate
    small.close()
    big_inst = I.maxcut_er(3000, 6.0, seed=2)               # working set ~ 38 MB > 32 MiB
    big = L.Problem(big_inst)
    ld = 8
    x = torch.zeros((big_inst.n, ld), dtype=torch.float64, device="cuda")
    q = torch.zeros(big_inst.m, dtype=torch.float64, device="cuda")
    assert L.lorads_op_sddmm(big.handle, 0, 8, ld, x, x, q) == 0   # builds the device form
    torch.cuda.synchronize()
    res = L.lorads_solve_static(big.handle, big.params())
    assert res.status == L.LORADS_ERR_TOO_LARGE
    assert "fixed scratch" in L.lorads_status_string(res.status)
    big.close()
