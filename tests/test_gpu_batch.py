"""Batched solves (one persistent launch, one CTA or a group of CTAs per problem, device
queue, largest first) against individual solves of the same problems."""
import numpy as np
import pytest

from oracle import SDP, Params, solve
from paper_2403_09133_gb300 import instances as I
from paper_2403_09133_gb300 import lorads as L

pytestmark = pytest.mark.gpu


def _batch_instances(count=12, seed0=500):
    return I.workload_batch(count=count, seed0=seed0, n_lo=40, n_hi=260)


@pytest.mark.parametrize("prec", [L.LORADS_PREC_FP64, L.LORADS_PREC_MIXED])
def test_batch_equals_individual_at_same_geometry(cuda, prec):
    insts = _batch_instances()
    probs = [L.Problem(x) for x in insts]
    prm = probs[0].params(precision=prec, max_admm_iter=400, threads=256, team_mult=1)
    single = [L.lorads_solve(p.handle, prm).as_dict() for p in probs]
    res, th, mu = L.lorads_solve_batch([p.handle for p in probs], prm)
    assert (th, mu) == (256, 1)
    for a, b in zip(single, res):
        assert a["status"] == b["status"]
        assert a["objective"] == b["objective"]          # same kernel, same order: bit-identical
        assert a["admm_iters"] == b["admm_iters"] and a["cg_iters"] == b["cg_iters"]
    # solutions are readable per problem after the batch
    sol = probs[3].solution()
    assert sol["U_hat"].shape == (insts[3].n, res[3]["rank"])
    for p in probs:
        p.close()


def test_batch_autotuned_matches_oracle(cuda):
    insts = _batch_instances(count=8, seed0=700)
    probs = [L.Problem(x) for x in insts]
    prm = probs[0].params(precision=L.LORADS_PREC_MIXED, max_admm_iter=300)
    prm.threads = 0
    prm.team_mult = 0
    res, th, mu = L.lorads_solve_batch([p.handle for p in probs], prm)
    assert th in (128, 256, 384) and mu in (1, 2, 4)
    for inst, r in zip(insts, res):
        ref = solve(SDP.from_instance(inst), Params(max_admm_iter=300))
        assert abs(r["admm_iters"] - ref["admm_iters"]) <= 2
        assert abs(r["objective"] - ref["objective"]) <= 1e-6 * abs(ref["objective"])
    for p in probs:
        p.close()


def test_batch_rejects_empty(cuda):
    with pytest.raises(L.LoradsError):
        L.lorads_solve_batch([], L.lorads_default_params())


@pytest.mark.parametrize("group", [2, 4])
def test_batch_in_cta_groups(cuda, group):
    """Groups of CTAs share each problem through bounded barriers: every problem passes the
    final test, and the objectives agree with one-CTA solves to what the final test at 1e-6
    fixes (the reduction order differs, so the iterates differ by rounding)."""
    insts = _batch_instances(count=10, seed0=900)
    probs = [L.Problem(x) for x in insts]
    prm = probs[0].params(precision=L.LORADS_PREC_MIXED, threads=256, team_mult=1)
    prm.group = 1
    one, _, _ = L.lorads_solve_batch([p.handle for p in probs], prm)
    prm.group = group
    grp, _, _ = L.lorads_solve_batch([p.handle for p in probs], prm)
    for a, b in zip(one, grp):
        assert a["status"] == 0 and b["status"] == 0
        assert abs(a["objective"] - b["objective"]) <= 1e-5 * abs(a["objective"])
    # a group solve is deterministic
    again, _, _ = L.lorads_solve_batch([p.handle for p in probs], prm)
    assert [r["objective"] for r in again] == [r["objective"] for r in grp]
    for p in probs:
        p.close()
