"""Benchmark: LoRADS solves of the 141x141 +-1 toroidal MaxCut SDP on the GPU.

One step = one whole solve (Algorithm 2: Phase I, Phase II with CG, output and residuals)
of the workload with its data already resident on the device, in the chosen (mixed
FP32/FP64) form; the plain FP64 form is timed on the same workload for comparison.  A solve
ends when the output passes the final test at 1e-6: the paper's primal infeasibility, then
the Appendix B gap and dual infeasibility (lambda_min(C - A^T y) by Lanczos on the device), so
the time of a converged step is the time to KKT <= 1e-6 in those measures.

Prints one JSON line; its main keys:
  value       solves per second over all ranks (device-resident inputs, CUDA events)
  e2e         the same metric through the C ABI from host buffers (upload + solve + download)
  roofline    the solver kernel's algorithmic bytes / its CUDA-event time vs measured HBM peak
  cpu_baseline  the FP64 CPU oracle timed on a bounded sample of the same workload

`--impl reference` times the CPU oracle alone (the reference arm for this workload).
Multi-GPU (torchrun): every rank solves its own copy of the headline workload (replicas,
weak scaling) and its share of the batch (no data exchange); rank 0 prints max-over-ranks
timing.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-KKT<=1e-6 & CG-operator HBM GB/s: chosen form vs plain FP64, 1 GB300"
# DRAM read+write bytes of one mixed-form solver launch on this workload, from one ncu capture
# (profiles/solver_traffic_torus141.md); reported only while the solver sources are unchanged.
SOLVER_SOURCES = ["lorads_solver.cuh", "lorads_device.cuh", "lorads_kernels.cuh", "lorads_f32.cu",
                  "lorads_capi.cu"]
SOLVER_TRAFFIC = {"sources_sha256_16": "db5fdb833337b144", "bytes_per_launch": 4144.08e6}


def solver_traffic():
    import hashlib
    h = hashlib.sha256()
    for f in SOLVER_SOURCES:
        with open(os.path.join(ROOT, "paper_2403_09133_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest()[:16] == SOLVER_TRAFFIC["sources_sha256_16"]:
        return SOLVER_TRAFFIC["bytes_per_launch"]
    return None
WORKLOAD = "maxcut_torus_141x141_pm1"
# The FP64 oracle's own full solve of this workload (default parameters, the final test at
# 1e-6; tests/golden/make_torus141.py, 331 s on one x86 host core): 1,960 Phase II iterations,
# then Phase III with 173 trust-region Newton steps and 17,279 Hessian products (rank 15 -> 23).
# The CPU baseline and the reference arm time a bounded sample of each phase and scale it to
# these.
ORACLE_COUNTS = {WORKLOAD: {"admm_iters": 1960, "newton_steps": 173, "newton_cg": 17279}}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lorads", choices=["lorads", "reference"])
    ap.add_argument("--oracle-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-mc", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--batch-count", type=int, default=512)
    return ap.parse_args()


def make_instance(name):
    from paper_2403_09133_gb300 import instances as I
    if name == WORKLOAD:
        return I.workload_torus141()
    if name == "maxcut_er_n500_d8":
        return I.workload_er500()
    raise ValueError(name)


# --------------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4)
                          if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


# --------------------------------------------------------------------------------- CPU oracle
def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


def oracle_sample_here(workload, seconds, counts):
    """The FP64 CPU oracle on a bounded sample of one solve (this process): Phase I in full,
    Phase II iterations for half the budget, then Phase III's Newton-CG iterations (each a
    Hessian-vector product on the product of spheres) at the Phase II point for the other half;
    the per-iteration times are scaled to `counts` (a projection, not a full solve)."""
    from oracle import SDP, Params
    import oracle.lorads as OL
    inst = make_instance(workload)
    sdp = SDP.from_instance(inst)
    p = OL.resolve_auto(sdp, Params())
    t0 = time.perf_counter()
    r = OL.initial_rank(sdp.m, sdp.n, p)
    ph1 = OL.lralm(sdp, OL.initial_factor(sdp, r, p.seed), p)
    t1 = time.perf_counter()
    st = OL.AdmmState(U=ph1["U"].copy(), V=ph1["U"].copy(), lam=ph1["lam"].copy(),
                      rho=min(p.h * ph1["sigma"], p.rho_max), rp=ph1["rp"])
    k = 0
    while time.perf_counter() - t1 < 0.5 * seconds and k < counts["admm_iters"]:
        OL.admm_iteration(sdp, st, p)
        k += 1
    t2 = time.perf_counter()
    rad, con, a = OL.sphere_structure(sdp)
    U = OL.retract(0.5 * (st.U + st.V), rad)
    _, mu, CU = OL.manifold_multiplier(sdp, U, con, a)
    g = 2.0 * (CU - mu[:, None] * U)
    j = 0
    while time.perf_counter() - t2 < 0.5 * seconds and j < counts["newton_cg"]:
        OL.truncated_cg(lambda Z: OL.riemannian_hessian(sdp, U, mu, Z), g, 1e300, 1)
        j += 1
    t3 = time.perf_counter()
    per_admm = (t2 - t1) / max(k, 1)
    per_cg = (t3 - t2) / max(j, 1)
    solve_s = (t1 - t0) + per_admm * counts["admm_iters"] + per_cg * counts["newton_cg"]
    return {"value": 1.0 / solve_s, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "cpu": cpu_model(),
            "sample": f"projection: Phase I in full ({t1 - t0:.2f} s), {k} Phase II iterations "
                      f"({per_admm * 1e3:.2f} ms each) and {j} Phase III CG iterations "
                      f"({per_cg * 1e3:.2f} ms each) timed on one thread, scaled to "
                      f"{counts['admm_iters']} and {counts['newton_cg']} (the oracle's own "
                      f"full solve of this workload)",
            "seconds_per_solve": solve_s}


def oracle_sample(workload, seconds, counts):
    """oracle_sample_here in a child process pinned to one BLAS / OpenMP thread, so that the
    baseline's thread count is known (the oracle is numpy/scipy code)."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
              "BLIS_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[v] = "1"
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_sample_here(%r, %r, %r)))"
            % (ROOT, workload, float(seconds), dict(counts)))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                         timeout=30 * 60)
    if out.returncode != 0:
        raise RuntimeError("oracle sample failed: " + out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


# --------------------------------------------------------------------------------- GPU arm
def algorithmic_bytes(res, n, s):
    """Algorithmic bytes of one solve's Hessian applies, 3 n ld s per apply (read P and the fixed
    factor W, write H P; ld = 4 ceil(r / 4), s the element size): Phase II's applies (CG
    iterations and warm-start residuals, at the initial rank's ld) plus Phase III's Newton-CG
    applies (at the final rank's ld), both in the form's element type."""
    r0 = res.get("rank0", res["rank"])
    ld0 = (r0 + 3) // 4 * 4
    ld1 = (res["rank"] + 3) // 4 * 4
    return res["hessian_applies"] * 3 * n * ld0 * s + res["newton_cg_iters"] * 3 * n * ld1 * s


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2403_09133_gb300 import lorads as L
    from paper_2403_09133_gb300 import shard as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    inst = make_instance(args.workload)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    prob = L.Problem(inst)
    results = {}
    forms = (("mixed", L.LORADS_PREC_MIXED, L.LORADS_SUB_CG),
             ("fp64", L.LORADS_PREC_FP64, L.LORADS_SUB_CG),
             ("mixed_row_direct", L.LORADS_PREC_MIXED, L.LORADS_SUB_ROW_DIRECT),
             ("fp64_row_direct", L.LORADS_PREC_FP64, L.LORADS_SUB_ROW_DIRECT))
    for form, prec, sub in forms:
        prm = prob.params(precision=prec, subsolver=sub)
        times = []
        res = None
        for it in range(args.warmup + args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(it))          # L2 flush outside the timed region
            stream.synchronize()
            if it == args.warmup:
                barrier()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            r = L.lorads_solve(prob.handle, prm, stream)
            ev1.record(stream)
            ev1.synchronize()
            if it >= args.warmup:
                times.append(ev0.elapsed_time(ev1) * 1e-3)
            res = r.as_dict()
        barrier()
        results[form] = dict(res=res, times=times)
    # clocks: one more timed pass of the chosen form under the sampler
    sampler = ClockSampler(local)
    sampler.start()
    prm = prob.params(precision=L.LORADS_PREC_MIXED)
    t_cl = []
    for _ in range(max(1, args.steps)):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        L.lorads_solve(prob.handle, prm, stream)
        ev1.record(stream)
        ev1.synchronize()
        t_cl.append(ev0.elapsed_time(ev1) * 1e-3)
    clocks = sampler.stop()
    # end to end: host buffers through the C ABI, every step
    e2e_times = []
    h2d = (len(inst.C_row) * 16 + len(inst.A_con) * 20 + inst.m * 8)
    for it in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p2 = L.Problem(inst)
        r2 = p2.solve(precision=L.LORADS_PREC_MIXED)
        sol = p2.solution()
        p2.close()
        t1 = time.perf_counter()
        if it >= args.warmup:
            e2e_times.append(t1 - t0)
    d2h = sol["U"].nbytes * 3 + sol["y"].nbytes
    prob.close()

    t_mixed = max(statistics.median(results["mixed"]["times"]), 1e-12)
    t_fp64 = max(statistics.median(results["fp64"]["times"]), 1e-12)
    t_e2e = statistics.median(e2e_times)
    t_mixed_d = max(statistics.median(results["mixed_row_direct"]["times"]), 1e-12)
    t_fp64_d = max(statistics.median(results["fp64_row_direct"]["times"]), 1e-12)
    t_mixed, t_fp64, t_e2e, t_mixed_d, t_fp64_d = S.max_over_ranks(
        [t_mixed, t_fp64, t_e2e, t_mixed_d, t_fp64_d], device=dev)
    # the batch is sharded over the ranks (every rank takes part); the rest is rank 0's
    batch = None if args.no_batch else batch_bench(args, stream, rank, world, dev)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return None
    rm, rf = results["mixed"]["res"], results["fp64"]["res"]
    r0 = int(np.ceil(np.log2(max(inst.m, 2))))
    rm["rank0"] = rf["rank0"] = r0
    bytes_mixed = algorithmic_bytes(rm, inst.n, 4)
    bytes_fp64 = algorithmic_bytes(rf, inst.n, 8)
    tol = 1e-6
    kkt_ok = lambda r: (r["status"] == 0 and r["r_P"] <= tol and r["r_D"] <= tol
                        and abs(r["gap"]) <= tol and r["dual_psd"] <= tol)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    ach = bytes_mixed / t_mixed / 1e9
    line = {
        "metric": METRIC,
        "value": world / t_mixed,
        "unit": "solves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_mixed * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 CG operators / f64 masters",
        "data": "synthetic (seeded generator shaped like the paper's MaxCut workloads)",
        "config": {"workload": args.workload, "n": inst.n, "m": inst.m,
                   "r0": rm["rank"], "form": "mixed", "parallelism": "replicas",
                   "l2": "256 MB buffer written between timed solves"},
        "solve": {k: rm[k] for k in ("status", "objective", "dual_objective", "r_P", "r_P_split",
                                    "r_stop", "r_D", "gap", "p_infeas", "d_infeas", "dual_psd",
                                    "lambda_min", "admm_iters", "cg_iters", "hessian_applies",
                                    "alm_outer", "lbfgs_iters", "rank", "rank_growths", "gamma",
                                    "polished", "newton_steps", "newton_cg_iters",
                                    "time_phase1_s", "time_phase2_s", "time_phase3_s",
                                    "lanczos_steps", "time_lanczos_s")},
        # the final test: max(r_P, r_D) <= 1e-6 with r_D = ||(C - A^T y) U_hat||_F/(1+||C||_F),
        # the Appendix B gap, and lambda_min(C - A^T y) >= -1e-6 (1 + ||C||_inf) (Lanczos)
        "kkt": {"tol": tol, "reached": kkt_ok(rm), "r_P": rm["r_P"], "r_D": rm["r_D"],
                "gap": rm["gap"], "lambda_min": rm["lambda_min"], "dual_psd": rm["dual_psd"],
                "appendix_b_p_infeas": rm["p_infeas"], "appendix_b_d_infeas": rm["d_infeas"]},
        "plain_fp64": {"ms_per_solve": t_fp64 * 1e3, "status": rf["status"],
                       "kkt_reached": kkt_ok(rf),
                       "time_phase1_s": rf["time_phase1_s"], "time_phase2_s": rf["time_phase2_s"],
                       "time_phase3_s": rf["time_phase3_s"],
                       "objective": rf["objective"], "admm_iters": rf["admm_iters"],
                       "cg_iters": rf["cg_iters"], "newton_steps": rf["newton_steps"],
                       "newton_cg_iters": rf["newton_cg_iters"], "rank": rf["rank"],
                       "r_D": rf["r_D"], "dual_psd": rf["dual_psd"], "gap": rf["gap"],
                       "objective_rel_diff_vs_mixed":
                           abs(rf["objective"] - rm["objective"]) / abs(rf["objective"]),
                       "cg_operator_gbs": bytes_fp64 / t_fp64 / 1e9},
        "mixed_speedup_vs_fp64": t_fp64 / t_mixed,
        # the same workload with the exact row-block subproblem solve instead of CG (every
        # constraint one diagonal entry; Section 1 admits direct methods for the subproblems)
        "row_direct": {
            form: {"ms_per_solve": t * 1e3, "status": r["status"], "admm_iters": r["admm_iters"],
                   "cg_iters": r["cg_iters"], "objective": r["objective"],
                   "objective_rel_diff_vs_cg_mixed":
                       abs(r["objective"] - rm["objective"]) / abs(rm["objective"]),
                   "r_P": r["r_P"], "r_D": r["r_D"], "gap": r["gap"], "dual_psd": r["dual_psd"],
                   "kkt_reached": kkt_ok(r), "speedup_vs_cg_mixed": t_mixed / t}
            for form, r, t in (("mixed", results["mixed_row_direct"]["res"], t_mixed_d),
                               ("fp64", results["fp64_row_direct"]["res"], t_fp64_d))},
        "e2e": {"value": world / t_e2e, "unit": "solves/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                     "frac": ach / peak, "traffic": solver_traffic(),
                     "kernel": "lorads::solve_grid_kernel<float, 0>",
                     "unit_bytes": "3 n ld s per Hessian apply (Phase II's eq. linU and Phase "
                                   "III's truncated CG), s the form's element size",
                     "bytes_per_launch": bytes_mixed,
                     "l2_resident": True,
                     "working_set_bytes": 3 * inst.n * ((rm["rank"] + 3) // 4 * 4) * 8,
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one "
                                       "whole solve: nearly all of it the dual tests' kept "
                                       "Lanczos blocks (written once, the failing test's read "
                                       "back once); the iterations' working set stays in L2",
                     "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"},
        "gpu_launches": args.steps,
        "clocks": clocks,
    }
    if batch is not None:
        line["batch"] = batch
    if not args.no_mc:
        line["matrix_completion"] = mc_bench(args, stream)
    if not args.no_learned:
        line["learned_warm_start"] = learned_bench(args)
    if not args.no_cpu_baseline:
        counts = ORACLE_COUNTS.get(args.workload, {"admm_iters": rf["admm_iters"],
                                                     "newton_steps": rf["newton_steps"],
                                                     "newton_cg": rf["newton_cg_iters"]})
        line["cpu_baseline"] = oracle_sample(args.workload, args.oracle_seconds, counts)
    if world > 1:
        dist.destroy_process_group()
    return line


def batch_bench(args, stream, rank=0, world=1, dev=None):
    """512 uneven ER MaxCuts (n ~ U[64, 2048], degree ~ U[3, 12], seeds 1000+i) in one
    persistent launch per GPU (mixed form, autotuned CTA size and lanes per row), against
    plain FP64 one-problem solves on a sample of 16, scaled to the batch.  With several
    ranks each solves its share (longest-processing-time partition, no data exchange); the
    batch time is the maximum over ranks."""
    import torch
    from paper_2403_09133_gb300 import instances as I
    from paper_2403_09133_gb300 import lorads as L
    from paper_2403_09133_gb300 import shard as S
    insts = I.workload_batch(count=args.batch_count)
    works = [S.work_estimate(x.n, len(x.C_row) + len(x.A_con)) for x in insts]
    mine = S.shard(works, rank, world)
    probs = [L.Problem(insts[i]) for i in mine]
    handles = [p.handle for p in probs]
    prm = L.lorads_default_params()
    prm.precision = L.LORADS_PREC_MIXED
    res, th, mu = L.lorads_solve_batch(handles, prm, stream)      # tunes + warms up
    prm.threads, prm.team_mult = th, mu
    times = []
    for _ in range(2):
        torch.cuda.synchronize()
        S.max_over_ranks([0.0], device=dev)                      # start together
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res, _, _ = L.lorads_solve_batch(handles, prm, stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) * 1e-3)
    t_batch = S.max_over_ranks([min(times)], device=dev)[0]
    sample = list(range(0, len(probs), max(1, len(probs) // 16)))[:16]
    p64 = L.lorads_default_params()
    p64.precision = L.LORADS_PREC_FP64
    t_seq = 0.0
    for i in sample:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        L.lorads_solve(handles[i], p64, stream)
        e1.record(stream)
        e1.synchronize()
        t_seq += e0.elapsed_time(e1) * 1e-3
    for p in probs:
        p.close()
    counts = S.sum_over_ranks([
        t_seq * len(probs) / max(1, len(sample)),
        sum(r["status"] == 0 for r in res), sum(r["admm_iters"] for r in res),
        sum(r["rank_growths"] > 0 for r in res)], device=dev)
    t_seq_scaled = counts[0]
    return {"count": len(insts), "ranks": world, "seconds_one_launch": t_batch,
            "solves_per_s": len(insts) / t_batch, "tuned_threads": th, "tuned_team_mult": mu,
            "converged": int(counts[1]), "admm_iters_total": int(counts[2]),
            "rank_grown_in_phase2": int(counts[3]),
            "plain_fp64_sequential_s_est": t_seq_scaled,
            "speedup_vs_sequential_fp64": t_seq_scaled / t_batch,
            "sample": f"{len(sample)} one-problem FP64 solves per rank, scaled to its share"}


def mc_bench(args, stream):
    """Matrix completion at n = 40,000 (n1 = n2 = 20,000), rank-5 M, 15,694,167 observed
    entries (the size of the paper's MC_40000), r0 = 24, library defaults for non-diagonal
    constraints (switch 1e-3, h = 1, gamma = 2 ||C||_inf): one solve per form after a warm-up,
    plus the FP32 Hessian operator at this size."""
    import torch
    from paper_2403_09133_gb300 import instances as I
    from paper_2403_09133_gb300 import lorads as L
    inst = I.workload_mc()
    ev = np.linalg.eigvals((inst.mc_P.T @ inst.mc_P) @ (inst.mc_Q.T @ inst.mc_Q)).real
    nuclear2 = 2.0 * float(np.sqrt(np.clip(ev, 0, None)).sum())
    prob = L.Problem(inst)
    out = {"n": inst.n, "m": inst.m, "two_nuclear_norm": nuclear2}
    for form, prec in (("mixed", L.LORADS_PREC_MIXED), ("fp64", L.LORADS_PREC_FP64)):
        prm = prob.params(precision=prec)    # "auto": switch_tol 1e-3, h 1, gamma 2 ||C||_inf
        L.lorads_solve(prob.handle, prm, stream)          # warm-up (assembly, first touch)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = L.lorads_solve(prob.handle, prm, stream).as_dict()
        e1.record(stream)
        e1.synchronize()
        out[form] = {"seconds": e0.elapsed_time(e1) * 1e-3, "status": r["status"],
                     "objective_rel_err_vs_2nuclear": abs(r["objective"] - nuclear2) / nuclear2,
                     "r_P": r["r_P"], "gap": r["gap"], "d_infeas": r["d_infeas"],
                     "admm_iters": r["admm_iters"], "cg_iters": r["cg_iters"],
                     "time_phase1_s": r["time_phase1_s"], "time_phase2_s": r["time_phase2_s"]}
    # the CG operator at this size (FP32), CUDA events, L2 flushed
    r_, ld = 24, 24
    g = torch.Generator(device="cuda").manual_seed(1)
    V = torch.randn((inst.n, ld), generator=g, device="cuda")
    P = torch.randn((inst.n, ld), generator=g, device="cuda")
    H = torch.empty_like(V)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    times = []
    for it in range(8):
        flush.fill_(float(it))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        L.lorads_op_hessian(prob.handle, L.LORADS_PREC_MIXED, r_, ld, 50.0, 1.0, V, P, H, stream)
        e1.record(stream)
        e1.synchronize()
        if it >= 3:
            times.append(e0.elapsed_time(e1) * 1e-3)
    t = statistics.median(times)
    nnz = 2 * inst.m
    compulsory = 3 * inst.n * ld * 4 + 4 * (inst.n + 1) + nnz * 8
    gathered = nnz * 2 * ld * 4
    out["hessian_fp32"] = {"us_per_apply": t * 1e6, "compulsory_gbs": compulsory / t / 1e9,
                           "gathered_row_gbs": gathered / t / 1e9,
                           "note": "gathered rows (2 per symmetric entry) come from L2"}
    prob.close()
    return out


def learned_bench(args):
    """Learned warm start (small): 32 solver-labelled training graphs (n in [100, 300]),
    15 epochs on the GPU, then 8 held-out graphs solved from the Burer-Monteiro start and from
    the trained network, to the final test at 1e-6."""
    from paper_2403_09133_gb300 import learned as LN
    from paper_2403_09133_gb300 import lorads as L
    t0 = time.perf_counter()
    samples = LN.solve_targets(LN.make_graphs(32, 300_000, 100, 300))
    g = L.lorads_gnn_create(5)
    hist = LN.train(g, samples, epochs=15, lr=2e-3)
    t1 = time.perf_counter()
    rows = LN.evaluate(g, LN.make_graphs(8, 400_000, 100, 300), tol=1e-6)
    L.lorads_gnn_destroy(g)
    return {"train_graphs": 32, "epochs": 15, "loss_first": hist[0], "loss_last": hist[-1],
            "seconds_data_and_training": t1 - t0, "eval_tol": 1e-6,
            "eval": LN.summarize(rows)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    inst = make_instance(args.workload)
    counts = ORACLE_COUNTS.get(args.workload,
                               {"admm_iters": 5000, "newton_steps": 0, "newton_cg": 0})
    vals = []
    last = None
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        last = oracle_sample(args.workload, args.oracle_seconds / max(1, args.steps), counts)
        t1 = time.perf_counter()
        if it >= args.warmup:
            vals.append(last["value"])
    v = statistics.median(vals)
    return {
        "metric": METRIC, "impl": "reference", "value": v, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n": inst.n, "m": inst.m, "form": "oracle"},
        "cpu_baseline": {"value": v, "unit": "solves/s", "cores": last["cores"],
                         "kind": "oracle", "cpu": last["cpu"], "sample": last["sample"]},
        "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    line = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
