"""Operator microbenchmark: CUDA-event timing of the CG operators of the library.

Times lorads_op_hessian / lorads_op_spmm / lorads_op_sddmm (the kernels the solver is built
from) on a seeded workload and reports achieved GB/s of algorithmic bytes against the
measured HBM copy peak.  Inputs larger than L2 (129 MB) are used for HBM figures.

  python -m paper_2403_09133_gb300.opbench --family torus --side 2048 --rank 22 --prec mixed

Algorithmic (compulsory) bytes per launch: every input array read once, every output
written once (rows gathered again for neighbours are not counted; they hit L2 when the
factors fit there).  s = element size of the form, ld = 4 ceil(r/4), nnzA / nnzC count both
triangles of the symmetric CSR:
  hessian: P, W read, HP written (3 n ld s) + A rows (4 (n+1) + nnzA (4 + s))
  spmm:    W read, out written (2 n ld s) + C rows (4 (n+1) + nnzC (4 + s)) + A rows
           (4 (n+1) + nnzA (8 + s)) + the weights w (8 m)
  sddmm:   U, V read (2 n ld s) + per constraint row, column, value and q (24 m)
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def make(family, side, n1, samples, seed):
    from paper_2403_09133_gb300 import instances as I
    if family == "torus":
        return I.maxcut_torus(side, side, seed=seed)
    if family == "er":
        return I.maxcut_er(side, 8.0, seed=seed)
    if family == "mc":
        return I.matrix_completion(n1, n1, 5, samples, seed=seed)
    raise ValueError(family)


def main():
    import torch
    from paper_2403_09133_gb300 import lorads as L

    ap = argparse.ArgumentParser()
    ap.add_argument("--family", default="torus", choices=["torus", "er", "mc"])
    ap.add_argument("--side", type=int, default=2048)
    ap.add_argument("--n1", type=int, default=20000)
    ap.add_argument("--samples", type=int, default=15_694_167)
    ap.add_argument("--rank", type=int, default=0)
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--op", default="hessian", choices=["hessian", "spmm", "sddmm", "all", "solve"])
    ap.add_argument("--admm-cap", type=int, default=20, help="--op solve: Phase II iterations")
    ap.add_argument("--subsolver", default="cg", choices=["cg", "row_direct"],
                    help="--op solve: Phase II subproblem solver")
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--seed", type=int, default=2)
    a = ap.parse_args()

    inst = make(a.family, a.side, a.n1, a.samples, a.seed)
    n, m = inst.n, inst.m
    if a.op == "solve":
        # one capped solve (a short launch of the persistent solver kernel, e.g. for ncu)
        prob = L.Problem(inst)
        prec = L.LORADS_PREC_MIXED if a.prec == "mixed" else L.LORADS_PREC_FP64
        out = []
        for it in range(a.warmup + a.iters):
            res = prob.solve(precision=prec, max_admm_iter=a.admm_cap,
                             subsolver=L.LORADS_SUB_ROW_DIRECT if a.subsolver == "row_direct"
                             else L.LORADS_SUB_CG)
            out.append(res)
        prob.close()
        last = out[-1]
        print(json.dumps({"op": "solve", "family": a.family, "n": n, "m": m, "prec": a.prec,
                          "admm_iters": last["admm_iters"], "cg_iters": last["cg_iters"],
                          "status": last["status"], "rank": last["rank"],
                          "alm_outer": last["alm_outer"], "lbfgs_iters": last["lbfgs_iters"],
                          "rank_growths": last["rank_growths"], "sigma": last["sigma"],
                          "rho": last["rho"], "r_P": last["r_P"], "r_stop": last["r_stop"],
                          "ms_phase1": last["time_phase1_s"] * 1e3,
                          "ms_phase2": last["time_phase2_s"] * 1e3,
                          "us_per_admm_iter": last["time_phase2_s"] * 1e6 / max(1, last["admm_iters"])}),
              flush=True)
        return
    r = a.rank or int(np.ceil(np.log2(max(m, 2))))
    ld = (r + 3) // 4 * 4
    prec = L.LORADS_PREC_MIXED if a.prec == "mixed" else L.LORADS_PREC_FP64
    dt = torch.float32 if prec == L.LORADS_PREC_MIXED else torch.float64
    s = 4 if prec == L.LORADS_PREC_MIXED else 8
    prob = L.Problem(inst)
    g = torch.Generator(device="cuda").manual_seed(1)
    V = torch.zeros((n, ld), dtype=dt, device="cuda")
    P = torch.zeros((n, ld), dtype=dt, device="cuda")
    V[:, :r] = torch.randn((n, r), generator=g, device="cuda", dtype=dt)
    P[:, :r] = torch.randn((n, r), generator=g, device="cuda", dtype=dt)
    out = torch.empty((n, ld), dtype=dt, device="cuda")
    w = torch.randn(m, generator=g, device="cuda", dtype=torch.float64)
    q = torch.empty(m, dtype=torch.float64, device="cuda")
    off = int(np.count_nonzero(inst.A_row != inst.A_col))
    nnzA = m + off
    c_off = int(np.count_nonzero(inst.C_row != inst.C_col))
    nnzC = len(inst.C_row) + c_off
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    ops = ["hessian", "spmm", "sddmm"] if a.op == "all" else [a.op]
    report = []
    for op in ops:
        if op == "hessian":
            call = lambda: L.lorads_op_hessian(prob.handle, prec, r, ld, 37.0, 1.5, V, P, out, stream)
            nbytes = 3 * n * ld * s + 4 * (n + 1) + nnzA * (4 + s)
        elif op == "spmm":
            call = lambda: L.lorads_op_spmm(prob.handle, prec, r, ld, w, 1.5, V, out, stream)
            nbytes = 2 * n * ld * s + 8 * (n + 1) + nnzC * (4 + s) + nnzA * (8 + s) + 8 * m
        else:
            call = lambda: L.lorads_op_sddmm(prob.handle, prec, r, ld, V, P, q, stream)
            nbytes = 2 * n * ld * s + 24 * m
        times = []
        for it in range(a.warmup + a.iters):
            flush.fill_(float(it))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc = call()
            e1.record(stream)
            e1.synchronize()
            if rc != 0:
                raise RuntimeError(L.lorads_status_string(rc))
            if it >= a.warmup:
                times.append(e0.elapsed_time(e1) * 1e-3)
        t = statistics.median(times)
        peak = 6766.0
        try:
            peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
        except (OSError, KeyError):
            pass
        report.append({"op": op, "family": a.family, "n": n, "m": m, "r": r, "ld": ld,
                       "prec": a.prec, "us_per_launch": t * 1e6, "alg_bytes": nbytes,
                       "gbs": nbytes / t / 1e9, "frac_of_measured_hbm": nbytes / t / 1e9 / peak})
    prob.close()
    for rep in report:
        print(json.dumps(rep), flush=True)


if __name__ == "__main__":
    main()
