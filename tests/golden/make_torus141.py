"""Writes tests/golden/torus141_pm1.npz: the FP64 oracle's full solve of the 141 x 141 toroidal
MaxCut SDP with weights uniform in {-1, +1} (seed 2; n = m = 19,881, C = -L/4, X_jj = 1; the
bench workload).  Calls only the oracle and the seeded instance generator.

Stored: the objective <C, X>, the dual y (19,881 values), lambda_min(C - A^T y) from the
oracle's eigensolver, the oracle's residual report (r_P, r_D, gap) and its iteration counts.
The optimum's objective and y are what the CUDA library is compared with; the iteration counts
are the oracle's trajectory (Phase II, then Phase III) and are stored for reference only.

Usage: python tests/golden/make_torus141.py    (about 3 minutes on one x86 core)
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import SDP, Params, solve  # noqa: E402
from paper_2403_09133_gb300 import instances as I  # noqa: E402


def main():
    inst = I.workload_torus141()
    t0 = time.perf_counter()
    res = solve(SDP.from_instance(inst), Params())
    seconds = time.perf_counter() - t0
    if not res["converged"]:
        raise SystemExit("the oracle did not pass its final test")
    np.savez_compressed(
        os.path.join(HERE, "torus141_pm1.npz"),
        objective=res["objective"], y=res["y"], lambda_min=res["lambda_min"],
        r_P=res["r_P"], r_D=res["r_D"], gap=res["gap"], rank=res["rank"],
        admm_iters=res["admm_iters"], newton_steps=res["newton_steps"],
        newton_cg=res["newton_cg"], oracle_seconds=seconds)
    print(f"objective {res['objective']:.12f}  r_D {res['r_D']:.2e}  lambda_min "
          f"{res['lambda_min']:.2e}  ADMM {res['admm_iters']}  Newton {res['newton_steps']}  "
          f"({seconds:.0f} s)")


if __name__ == "__main__":
    main()
