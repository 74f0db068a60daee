"""Checkpoint / resume (lorads_get_state, lorads_set_state) and the injected device allocator
on the GPU.

A Phase II checkpoint is (U^k, V^k, lambda^k), the penalty of iteration k+1, k and the
final-test schedule: what Algorithm 1 carries between iterations (the oracle's own resume
repeats its uninterrupted run bit for bit, tests/test_oracle_solve.py).  On the GPU the
continuation recomputes the row-local loop's incrementally kept -(C W) and re-rounds the
FP32 shadows from the FP64 masters.  The uninterrupted loop does the same every 32
iterations, so a checkpoint taken at such k continues bit for bit; at other k the two agree
up to rounding: both pass the final test at 1e-6 and reach the same objective to the
accuracy that test implies, with totals (iterations, counters) that continue the
checkpointed ones.  The allocator tests
check that every device byte of a solve comes from the callbacks and goes back through
them, and that the results do not depend on where the memory came from."""
import numpy as np
import pytest

from paper_2403_09133_gb300 import instances as I
from paper_2403_09133_gb300 import lorads as L

pytestmark = pytest.mark.gpu

CASES = {
    "er500": lambda: I.workload_er500(),                               # one CTA, row-local
    "torus40": lambda: I.maxcut_torus(40, 40, seed=2),                   # grid scope
    "mc1000": lambda: I.matrix_completion(500, 500, 3, 60000, seed=4),   # general, grid
}


def _close(a, b, tol=1e-6):
    return abs(a - b) <= tol * (1.0 + abs(b))


@pytest.mark.parametrize("prec", [L.LORADS_PREC_FP64, L.LORADS_PREC_MIXED])
@pytest.mark.parametrize("case", sorted(CASES))
def test_resume_continues_the_solve(cuda, case, prec):
    inst = CASES[case]()
    p = L.Problem(inst)
    full = p.solve(precision=prec)
    assert full["status"] == 0, L.lorads_status_string(full["status"])
    half = full["admm_iters"] // 2
    k1 = half // 32 * 32 if half >= 32 else half
    part = p.solve(precision=prec, max_admm_iter=k1)
    assert part["status"] == L.LORADS_ERR_MAXITER and part["admm_iters"] == k1
    st = p.get_state()
    p.close()
    assert st["phase"] == 2 and st["admm_iters"] == k1 and st["rank"] == part["rank"]
    assert st["n"] == inst.n and st["m"] == inst.m
    assert st["rho"] == part["rho"] and st["gamma"] == part["gamma"] and st["rho"] > 0
    assert st["cg_iters"] == part["cg_iters"] and st["alm_outer"] == part["alm_outer"]
    assert st["U"].shape == (inst.n, st["rank"]) and st["lam"].shape == (inst.m,)
    # a fresh handle, as another process would have after reading the checkpoint back
    q = L.Problem(inst)
    q.set_state(st)
    res = q.solve(precision=prec, phase1=0)
    q.close()
    assert res["status"] == 0, L.lorads_status_string(res["status"])
    assert res["r_P"] <= 1e-6 and abs(res["gap"]) <= 1e-6 and res["r_D"] <= 1e-6
    assert res["dual_psd"] <= 1e-6
    assert _close(res["objective"], full["objective"])
    if k1 % 32 == 0:
        # the uninterrupted loop itself refreshes -(C W) and the shadows from the masters at
        # such k: the continuation repeats it exactly
        assert res["objective"] == full["objective"]
        assert res["admm_iters"] == full["admm_iters"] and res["cg_iters"] == full["cg_iters"]
    # totals continue the checkpointed counters; Phase I is not repeated
    assert res["admm_iters"] > k1 and abs(res["admm_iters"] - full["admm_iters"]) <= 40
    assert res["cg_iters"] > st["cg_iters"]
    assert res["alm_outer"] == full["alm_outer"] and res["lbfgs_iters"] == full["lbfgs_iters"]
    assert res["gamma"] == full["gamma"] and res["sigma"] == full["sigma"]
    print(f"{case} prec={prec}: full k={full['admm_iters']} obj={full['objective']!r}; "
          f"resumed from {k1}: k={res['admm_iters']} obj={res['objective']!r}; "
          f"identical={res['objective'] == full['objective'] and res['admm_iters'] == full['admm_iters']}")


@pytest.mark.parametrize("k1", [64, 80])
@pytest.mark.parametrize("prec", [L.LORADS_PREC_FP64, L.LORADS_PREC_MIXED])
@pytest.mark.parametrize("case", ["er500", "mc30"])
def test_resume_follows_the_trajectory(cuda, case, prec, k1):
    """Stopped at the same iteration k2, the uninterrupted solve and the one resumed at k1
    hold the same iterate: bit for bit when k1 is a multiple of 32, up to rounding otherwise
    (mc30: the one-CTA general path)."""
    inst = (I.matrix_completion(30, 30, 2, 500, seed=3) if case == "mc30"
            else I.workload_er500())
    kw = dict(precision=prec, h=5.0) if case == "mc30" else dict(precision=prec)
    k2 = 192
    p = L.Problem(inst)
    ref = p.solve(max_admm_iter=k2, tol=1e-12, **kw)
    ref_st = p.get_state()
    p.solve(max_admm_iter=k1, tol=1e-12, **kw)
    st = p.get_state()
    p.close()
    q = L.Problem(inst)
    q.set_state(st)
    res = q.solve(max_admm_iter=k2, tol=1e-12, phase1=0, **kw)
    got = q.get_state()
    q.close()
    assert ref["status"] == res["status"] == L.LORADS_ERR_MAXITER
    assert res["admm_iters"] == ref["admm_iters"] == k2 and got["rho"] == ref_st["rho"]
    # FP64: differences of rounding order only; MIXED: the FP32 shadows of U and V differ by
    # FP32 rounding after the resume (re-rounded from the masters instead of advanced)
    fp64 = prec == L.LORADS_PREC_FP64
    assert _close(res["objective"], ref["objective"], 1e-9 if fp64 else 1e-6)
    assert _close(res["r_P_split"], ref["r_P_split"], 1e-3 if fp64 else 1e-1)
    scale = 1.0 + np.abs(ref_st["lam"]).max()
    assert np.abs(got["lam"] - ref_st["lam"]).max() <= (1e-7 if fp64 else 1e-4) * scale
    if k1 % 32 == 0:
        assert np.array_equal(got["U"], ref_st["U"]) and np.array_equal(got["V"], ref_st["V"])
        assert np.array_equal(got["lam"], ref_st["lam"])
    print(f"{case} prec={prec} k1={k1}: at k={k2} identical "
          f"U={np.array_equal(got['U'], ref_st['U'])} lam={np.array_equal(got['lam'], ref_st['lam'])}")


@pytest.mark.parametrize("prec", [L.LORADS_PREC_FP64, L.LORADS_PREC_MIXED])
def test_resume_with_the_direct_subsolver(cuda, prec):
    """The row-block direct solve keeps delta_U between iterations; a resume recomputes it
    from the checkpoint, and at k a multiple of 32 the continuation is exact."""
    inst = I.maxcut_torus(40, 40, seed=2)
    kw = dict(precision=prec, subsolver=L.LORADS_SUB_ROW_DIRECT)
    p = L.Problem(inst)
    full = p.solve(**kw)
    p.solve(max_admm_iter=256, **kw)
    st = p.get_state()
    p.close()
    q = L.Problem(inst)
    q.set_state(st)
    res = q.solve(phase1=0, **kw)
    q.close()
    assert full["status"] == 0 and res["status"] == 0
    assert res["objective"] == full["objective"] and res["admm_iters"] == full["admm_iters"]


def test_resume_after_phase2_rank_growth(cuda):
    """Without Phase III the 770-vertex batch graph grows its rank 10 -> 15 in Phase II; a
    checkpoint taken after the growth carries rank 15 and the growth count, and the resumed
    solve ends where the uninterrupted one does."""
    inst = [x for x in I.workload_batch() if x.n == 770][0]
    p = L.Problem(inst)
    K = 3000
    full = p.solve(polish=0, max_admm_iter=K)
    assert full["rank"] == 15 and full["rank_growths"] == 1
    k1 = 87 * 32                    # a multiple of 32: the resume repeats the run bit for bit
    part = p.solve(polish=0, max_admm_iter=k1)
    st = p.get_state()
    p.close()
    assert part["status"] == L.LORADS_ERR_MAXITER
    assert st["rank"] == 15 and st["rank_growths"] == 1
    q = L.Problem(inst)
    q.set_state(st)
    res = q.solve(phase1=0, polish=0, max_admm_iter=K)
    q.close()
    assert res["status"] == full["status"] and res["rank"] == 15 and res["rank_growths"] == 1
    assert res["admm_iters"] == full["admm_iters"]
    assert _close(res["objective"], full["objective"])


def test_checkpoint_file_roundtrip_is_deterministic(cuda, tmp_path):
    inst = I.workload_er500()
    p = L.Problem(inst)
    p.solve(max_admm_iter=96)
    path = str(tmp_path / "ckpt.npz")
    p.save_state(path)
    st = p.get_state()
    p.close()
    a = L.Problem(inst)
    a.set_state(st)
    ra = a.solve(phase1=0)
    a.close()
    b = L.Problem(inst)
    b.load_state(path)
    rb = b.solve(phase1=0)
    sb = b.solution()
    b.close()
    assert ra["status"] == 0 and rb["status"] == 0
    assert ra["objective"] == rb["objective"] and ra["admm_iters"] == rb["admm_iters"]
    assert sb["U"].shape[1] == rb["rank"]


def test_batch_checkpoint_and_resume(cuda):
    insts = [I.maxcut_er(n, 6.0, seed=40 + n) for n in (96, 160, 240, 320, 400, 520)]
    prm = L.lorads_default_params()
    prm.threads, prm.team_mult = 256, 1
    hs = [L.Problem(x) for x in insts]
    full, _, _ = L.lorads_solve_batch([h.handle for h in hs], prm)
    prm.max_admm_iter = 64
    part, _, _ = L.lorads_solve_batch([h.handle for h in hs], prm)
    states = [h.get_state() for h in hs]
    for h in hs:
        h.close()
    assert all(r["status"] == L.LORADS_ERR_MAXITER for r in part)
    hs = [L.Problem(x) for x in insts]
    for h, st in zip(hs, states):
        h.set_state(st)
    prm.max_admm_iter = 5000
    prm.phase1 = 0
    res, _, _ = L.lorads_solve_batch([h.handle for h in hs], prm)
    for h in hs:
        h.close()
    for f, r in zip(full, res):
        assert f["status"] == 0 and r["status"] == 0
        assert r["admm_iters"] > 64 and _close(r["objective"], f["objective"])


def test_state_errors(cuda):
    inst = I.maxcut_er(60, 6.0, seed=11)
    p = L.Problem(inst)
    lib = L.load_library()
    st = L.lorads_state()
    # no solve yet
    assert lib.lorads_get_state(p.handle, st, None, None, None) == L.LORADS_ERR_STATE
    p.solve(max_admm_iter=50)
    good = p.get_state()

    def rejected(**change):
        bad = dict(good)
        bad.update(change)
        return L.lorads_set_state(p.handle, bad) == L.LORADS_ERR_ARG

    assert rejected(n=inst.n + 1)
    assert rejected(m=inst.m + 1)
    assert rejected(phase=1)
    assert rejected(rho=0.0)
    assert rejected(gamma=-1.0)
    assert rejected(admm_iters=-1)
    assert rejected(prev_d_infeas=float("inf"))
    U = good["U"].copy()
    U[3, 0] = np.nan
    assert rejected(U=U)
    lam = good["lam"].copy()
    lam[0] = np.inf
    assert rejected(lam=lam)
    assert lib.lorads_set_state(p.handle, None, None, None, None) == L.LORADS_ERR_ARG
    assert L.lorads_set_state(p.handle, good) == L.LORADS_OK
    # an allocation-free solve leaves the problem's own state (the last lorads_solve's) as it was
    prm = p.params(max_admm_iter=50)
    L.lorads_solve_static(p.handle, prm)
    again = p.get_state()
    assert again["admm_iters"] == good["admm_iters"] and again["rho"] == good["rho"]
    assert np.array_equal(again["U"], good["U"]) and np.array_equal(again["lam"], good["lam"])
    p.close()


def test_torch_allocator_holds_every_byte(cuda):
    torch = cuda
    inst = I.maxcut_torus(40, 40, seed=2)
    ref = L.Problem(inst)
    r0 = ref.solve(precision=L.LORADS_PREC_MIXED)
    ref.close()
    torch.cuda.synchronize()
    alloc = L.TorchAllocator()
    before = torch.cuda.memory_allocated()
    p = L.Problem(inst, allocator=alloc)
    r1 = p.solve(precision=L.LORADS_PREC_MIXED)
    assert alloc.allocs >= 2 and alloc.bytes_live > 0
    assert torch.cuda.memory_allocated() - before >= alloc.bytes_live
    # same kernels, same geometry, deterministic reductions: the same result
    assert r1["status"] == 0 and r1["objective"] == r0["objective"]
    assert r1["admm_iters"] == r0["admm_iters"]
    sol = p.solution()
    assert np.isfinite(sol["U_hat"]).all()
    p.close()
    assert alloc.bytes_live == 0
    assert torch.cuda.memory_allocated() == before


def test_torch_allocator_in_batches(cuda):
    insts = [I.maxcut_er(n, 6.0, seed=70 + n) for n in (100, 200, 300)]
    alloc = L.TorchAllocator()
    hs = [L.Problem(x, allocator=alloc) for x in insts]
    prm = hs[0].params(threads=256, team_mult=1)
    res, _, _ = L.lorads_solve_batch([h.handle for h in hs], prm)
    assert all(r["status"] == 0 for r in res)
    live = alloc.bytes_live
    assert live > 0 and alloc.allocs >= 2 * len(hs) + 1   # + the batch's argument block
    for h in hs:
        h.close()
    assert alloc.bytes_live == 0


def test_allocator_failures_are_statuses(cuda):
    """An allocator that fails, or returns memory that is not 256-byte aligned, gives
    LORADS_ERR_NOMEM; a misaligned block goes straight back to its free."""
    torch = cuda
    inst = I.maxcut_er(60, 6.0, seed=11)
    freed = []

    def no_memory(nbytes, stream, ctx):
        return None

    def never(ptr, nbytes, stream, ctx):
        freed.append(ptr)

    p = L.Problem(inst)
    prm = p.params()
    prm.dev_alloc = L.ALLOC_FN(no_memory)
    prm.dev_free = L.FREE_FN(never)
    assert L.lorads_solve(p.handle, prm).status == L.LORADS_ERR_NOMEM
    assert freed == []

    held = {}

    def misaligned(nbytes, stream, ctx):
        base = int(torch.cuda.caching_allocator_alloc(int(nbytes) + 256))
        held[base + 16] = base
        return base + 16

    def give_back(ptr, nbytes, stream, ctx):
        freed.append(ptr)
        torch.cuda.caching_allocator_delete(held.pop(ptr))

    prm.dev_alloc = L.ALLOC_FN(misaligned)
    prm.dev_free = L.FREE_FN(give_back)
    assert L.lorads_solve(p.handle, prm).status == L.LORADS_ERR_NOMEM
    assert len(freed) == 1 and held == {}
    # only one of the two callbacks: an argument error
    prm.dev_free = L.FREE_FN()
    assert L.lorads_solve(p.handle, prm).status == L.LORADS_ERR_ARG
    p.close()
