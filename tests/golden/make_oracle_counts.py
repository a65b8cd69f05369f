"""Write tests/golden/medium_box_oracle.json with the CPU oracle alone.

The file records how many iterations the oracle's Algorithm 1 takes on the
256 x 256 x 128 benchmark problem (tol 1e-8 on the updated residual) and the
residuals it ends with.  bench.py uses the count to express the oracle's
per-pass time in solves/s.  Run: python tests/golden/make_oracle_counts.py
(about 20 minutes of one CPU core).
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402
from oracle import FluxOperator, LinePreconditioner, assemble_csr, pcg_interleaved  # noqa: E402


def main():
    p = W.medium_box()
    b = W.medium_box_rhs(p)
    t0 = time.time()
    res = pcg_interleaved(FluxOperator(p), LinePreconditioner(assemble_csr(p), p), b, eps=1e-8, maxiter=100000)
    out = {
        "workload": "box256x256x128, depth 0.004, grading 1.05, lambda2 1e-2, beta exp(-z/0.005), "
                    "rhs uniform(seed 0) + sin(2 pi x) cos(2 pi y) zeta",
        "tol": 1e-8,
        "iterations": res.iterations,
        "converged": bool(res.converged),
        "relres_recursive": res.residual_history[-1] / float(np.linalg.norm(b)),
        "relres_true": res.final_true_relres,
        "oracle_seconds": time.time() - t0,
    }
    with open(os.path.join(HERE, "medium_box_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)


if __name__ == "__main__":
    main()
