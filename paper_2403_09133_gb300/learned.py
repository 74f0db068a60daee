"""Learned warm start: data generation with the solver, training, and held-out evaluation.

Everything numeric runs in the library's kernels through the C ABI (batched solves for the
training targets, the network's forward/backward/Adam on the tensor cores, the solves of
the evaluation); this module only moves arrays between those calls.

Targets are rotation-invariant (U_0 is only defined up to an orthogonal rotation): for every
edge (i, j) the Gram entry U_hat_i . U_hat_j of the solved instance, and the dual y.  The
warm start replaces Phase I: Phase II starts from U = V = U_0, lambda = -y_0, rho_0 = 100
(the paper's initial rho for LRADMM without a warm start, Table 1's note).

  python -m paper_2403_09133_gb300.learned --train 192 --eval 32 --n-lo 500 --n-hi 3000
"""
from __future__ import annotations

import argparse
import json
import math
import time
from dataclasses import dataclass
from typing import List

import numpy as np

from . import instances as I
from . import lorads as L


@dataclass
class Sample:
    inst: object
    ei: np.ndarray
    ej: np.ndarray
    w: np.ndarray
    r: int
    Xs: np.ndarray
    ys: np.ndarray


def graph_arrays(inst):
    off = inst.C_row != inst.C_col
    return (inst.C_row[off].astype(np.int32), inst.C_col[off].astype(np.int32),
            inst.C_val[off].astype(np.float64))


def rank_for(inst) -> int:
    return min(16, max(1, int(math.ceil(math.log2(max(inst.m, 2))))))


def make_graphs(count, seed0, n_lo, n_hi, d_lo=3.0, d_hi=10.0):
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        n = int(rng.integers(n_lo, n_hi + 1))
        d = float(rng.uniform(d_lo, d_hi))
        out.append(I.maxcut_er(n, d, seed=seed0 + i, name=f"learn_{seed0 + i}"))
    return out


def solve_targets(insts, max_admm_iter=1000, stream=None, chunk=128) -> List[Sample]:
    """Solves the instances in batched launches of `chunk` problems (each problem's solver
    state is resident during its batch) and returns their training targets."""
    samples = []
    for c0 in range(0, len(insts), chunk):
        part = insts[c0:c0 + chunk]
        probs = [L.Problem(x) for x in part]
        prm = probs[0].params(precision=L.LORADS_PREC_MIXED, max_admm_iter=max_admm_iter)
        L.lorads_solve_batch([p.handle for p in probs], prm, stream)
        for inst, p in zip(part, probs):
            sol = p.solution()
            Uh = sol["U_hat"]
            ei, ej, w = graph_arrays(inst)
            Xs = np.einsum("ij,ij->i", Uh[ei], Uh[ej])
            samples.append(Sample(inst, ei, ej, w, rank_for(inst), Xs, sol["y"].copy()))
            p.close()
    return samples


def train(g, samples: List[Sample], epochs: int, lr: float, seed: int = 0, stream=None):
    rng = np.random.default_rng(seed)
    history = []
    for ep in range(epochs):
        order = rng.permutation(len(samples))
        tot = 0.0
        for k in order:
            s = samples[k]
            L.lorads_gnn_load_graph(g, s.inst.n, s.ei, s.ej, s.w, feature_seed=s.inst.n)
            loss, _ = L.lorads_gnn_train_step(g, s.r, s.Xs, s.ys, lr, stream=stream)
            tot += loss
        history.append(tot / len(samples))
    return history


def learned_start_solve(g, inst, stream=None, **prm_kw):
    """Forward pass -> (U_0, -y_0, rho_0 = 100) -> Phase II only."""
    ei, ej, w = graph_arrays(inst)
    r = rank_for(inst)
    t0 = time.perf_counter()
    L.lorads_gnn_load_graph(g, inst.n, ei, ej, w, feature_seed=inst.n)
    U0, y0 = L.lorads_gnn_forward(g, inst.n, r, stream)
    t1 = time.perf_counter()
    p = L.Problem(inst)
    L.lorads_set_start(p.handle, U0, -y0, 100.0)
    res = p.solve(phase1=0, precision=L.LORADS_PREC_MIXED, stream=stream, **prm_kw)
    p.close()
    res["time_network_s"] = t1 - t0
    return res


def bm_solve(inst, stream=None, **prm_kw):
    p = L.Problem(inst)
    res = p.solve(precision=L.LORADS_PREC_MIXED, stream=stream, **prm_kw)
    p.close()
    return res


def evaluate(g, insts, **prm_kw):
    rows = []
    for inst in insts:
        a = bm_solve(inst, **prm_kw)
        b = learned_start_solve(g, inst, **prm_kw)
        rows.append(dict(n=inst.n, bm_status=a["status"], bm_iters=a["admm_iters"],
                         bm_time=a["time_phase1_s"] + a["time_phase2_s"] + a["time_phase3_s"],
                         bm_obj=a["objective"],
                         ln_status=b["status"], ln_iters=b["admm_iters"],
                         ln_time=(b["time_phase2_s"] + b["time_phase3_s"] +
                                  b["time_network_s"]),
                         ln_obj=b["objective"]))
    return rows


def summarize(rows):
    both = [r for r in rows if r["bm_status"] == 0 and r["ln_status"] == 0]
    out = dict(count=len(rows), both_converged=len(both),
               bm_converged=sum(r["bm_status"] == 0 for r in rows),
               learned_converged=sum(r["ln_status"] == 0 for r in rows))
    if both:
        out.update(
            bm_mean_iters=float(np.mean([r["bm_iters"] for r in both])),
            learned_mean_iters=float(np.mean([r["ln_iters"] for r in both])),
            bm_mean_time_s=float(np.mean([r["bm_time"] for r in both])),
            learned_mean_time_s=float(np.mean([r["ln_time"] for r in both])),
            max_rel_objective_diff=float(max(abs(r["ln_obj"] - r["bm_obj"]) / abs(r["bm_obj"])
                                             for r in both)))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=192)
    ap.add_argument("--eval", type=int, default=32)
    ap.add_argument("--n-lo", type=int, default=500)
    ap.add_argument("--n-hi", type=int, default=3000)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--eval-tol", type=float, default=1e-6)
    a = ap.parse_args()
    t0 = time.perf_counter()
    train_graphs = make_graphs(a.train, 100_000, a.n_lo, a.n_hi)
    samples = solve_targets(train_graphs)
    t1 = time.perf_counter()
    g = L.lorads_gnn_create(a.seed)
    hist = train(g, samples, a.epochs, a.lr)
    t2 = time.perf_counter()
    rows = evaluate(g, make_graphs(a.eval, 200_000, a.n_lo, a.n_hi), tol=a.eval_tol)
    L.lorads_gnn_destroy(g)
    print(json.dumps({"train_graphs": a.train, "eval_graphs": a.eval, "n_range": [a.n_lo, a.n_hi],
                      "epochs": a.epochs, "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1],
                      "seconds_targets": t1 - t0, "seconds_training": t2 - t1,
                      "eval_tol": a.eval_tol,
                      "eval": summarize(rows)}))


if __name__ == "__main__":
    main()
