"""Failure detection without a GPU fault: bounded device waits that run out, the time limit,
and inputs the host rejects.  Every case ends in a status the host reads; the CUDA context
stays usable, which the tests check by solving again afterwards."""
import numpy as np
import pytest

from paper_2403_09133_gb300 import instances as I
from paper_2403_09133_gb300 import lorads as L

pytestmark = pytest.mark.gpu


def _solve(inst, **kw):
    p = L.Problem(inst)
    res = p.solve(**kw)
    return p, res


def test_grid_barrier_wait_runs_out(cuda):
    """A grid barrier allowed one poll gives up as soon as a CTA has to wait for a later one
    (CTAs start and run at different times), sets the error word, and every CTA leaves the
    persistent kernel: LORADS_ERR_DEVICE.  The next solve on the same context is normal."""
    inst = I.maxcut_torus(40, 40, seed=2)            # n = 1,600: the whole-GPU scope
    ref, r0 = _solve(inst)
    ref.close()
    p, res = _solve(inst, barrier_polls=1)
    assert res["status"] == L.LORADS_ERR_DEVICE
    again = p.solve()
    p.close()
    assert r0["status"] == 0 and again["status"] == 0
    assert again["objective"] == r0["objective"] and again["admm_iters"] == r0["admm_iters"]


def test_group_barrier_wait_runs_out(cuda):
    """The same in a batch solved by groups of two CTAs: the batch call returns (the launch
    ran), problems whose group gave up report LORADS_ERR_DEVICE, and a second batch is
    normal."""
    insts = [I.maxcut_er(n, 6.0, seed=300 + n) for n in (600, 900, 1200)]
    hs = [L.Problem(x) for x in insts]
    handles = [h.handle for h in hs]
    prm = hs[0].params(group=2, threads=256, team_mult=1, barrier_polls=1)
    bad, _, _ = L.lorads_solve_batch(handles, prm)
    assert any(r["status"] == L.LORADS_ERR_DEVICE for r in bad)
    assert all(r["status"] in (0, L.LORADS_ERR_DEVICE) for r in bad)
    prm.barrier_polls = 0
    good, _, _ = L.lorads_solve_batch(handles, prm)
    for h in hs:
        h.close()
    assert all(r["status"] == 0 for r in good)


def test_time_limit_and_resume(cuda):
    """A time limit shorter than Phase II ends the solve with LORADS_ERR_TIMEOUT; its state is
    a checkpoint from which the solve then finishes."""
    inst = I.maxcut_torus(40, 40, seed=2)
    p, res = _solve(inst, time_limit_s=2e-3)
    assert res["status"] == L.LORADS_ERR_TIMEOUT
    assert 0 < res["admm_iters"] < 1000
    st = p.get_state()
    p.set_state(st)
    done = p.solve(phase1=0)
    p.close()
    assert done["status"] == 0 and done["admm_iters"] > st["admm_iters"]


def test_rejected_inputs(cuda):
    inst = I.maxcut_er(30, 4.0, seed=1)
    lib = L.load_library()
    p = L.Problem(inst)
    h = p.handle
    nan = np.array([np.nan])
    i0 = np.array([0], dtype=np.int32)
    assert L.lorads_set_C(h, i0, i0, nan) == L.LORADS_ERR_ARG              # NaN value
    assert L.lorads_set_C(h, [1], [0], [1.0]) == L.LORADS_ERR_ARG           # row > col
    assert L.lorads_set_C(h, [0], [30], [1.0]) == L.LORADS_ERR_ARG          # col >= n
    assert L.lorads_add_A_sparse(h, [30], [0], [0], [1.0]) == L.LORADS_ERR_ARG   # con >= m
    assert L.lorads_add_A_sparse(h, [0], [0], [0], [np.inf]) == L.LORADS_ERR_ARG
    b = np.ones(30); b[4] = np.nan
    assert L.lorads_set_b(h, b) == L.LORADS_ERR_ARG
    assert L.lorads_add_A_rank1(h, 0, [0, 40], [1.0, 1.0], 1.0) == L.LORADS_ERR_ARG
    # rejected calls leave the problem as it was: it still solves
    assert p.solve()["status"] == 0
    p.close()
    # solve before b
    q = L.lorads_create(30, 30)
    assert L.lorads_set_C(q, inst.C_row, inst.C_col, inst.C_val) == 0
    assert L.lorads_add_A_sparse(q, inst.A_con, inst.A_row, inst.A_col, inst.A_val) == 0
    prm = L.lorads_default_params()
    assert L.lorads_solve(q, prm).status == L.LORADS_ERR_STATE
    # Phase II start requested without one
    assert L.lorads_set_b(q, inst.b) == 0
    prm.phase1 = 0
    assert L.lorads_solve(q, prm).status == L.LORADS_ERR_STATE
    L.lorads_destroy(q)
    assert lib.lorads_create(0, 5, None) == L.LORADS_ERR_ARG
