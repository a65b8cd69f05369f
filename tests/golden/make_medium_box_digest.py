"""Write digests of the CPU oracle's solutions of the 256 x 256 x 128 box.

The benchmark problem (box 256 x 256 x 128, depth 0.004, grading 1.05,
lambda^2 = 1e-2, beta = exp(-z/0.005), b = uniform(seed 0) + the smooth mode
sin(2 pi x) cos(2 pi y) zeta) is solved by the oracle's Algorithm 1
(Section 4.3) with the line preconditioner (Section 4.2) twice:

  fixed   exactly ITERS iterations (eps = 0), the count the oracle needs for
          tol 1e-8 (tests/golden/medium_box_oracle.json);
  tight   to tol 1e-12 on the updated residual.

A full x (8.4 M values) is too large to commit, so each file keeps a digest
that a GPU solve of the same problem can be compared with at full size:
||x||_2, the sum of x over every level (n_z values), and x itself at
SAMPLES cells drawn from a fixed seed (flat indices into [n_z][n_y][n_x]).

Only oracle/ and the seeded inputs of workloads/ are used.  Each part takes
tens of minutes of one CPU core; the two can run side by side:
    python tests/golden/make_medium_box_digest.py fixed
    python tests/golden/make_medium_box_digest.py tight
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

ITERS = 641          # the oracle's count at tol 1e-8 (medium_box_oracle.json)
SAMPLES = 4096
SAMPLE_SEED = 20130228


def sample_cells(n_cells):
    """Flat indices of the sampled cells (sorted, distinct)."""
    rng = np.random.default_rng(SAMPLE_SEED)
    return np.sort(rng.choice(n_cells, size=SAMPLES, replace=False))


def digest(x, cells):
    return {
        "norm2": float(np.linalg.norm(x.ravel())),
        "level_sums": [float(v) for v in x.reshape(x.shape[0], -1).sum(axis=1)],
        "cells": [int(c) for c in cells],
        "x": [float(v) for v in x.ravel()[cells]],
    }


def main(part):
    p = W.medium_box()
    b = W.medium_box_rhs(p)
    A = FluxOperator(p)
    M = LinePreconditioner(assemble_csr(p), p)
    t0 = time.time()
    if part == "fixed":
        res = pcg_interleaved(A, M, b, eps=0.0, maxiter=ITERS)
        tol = 0.0
    elif part == "tight":
        res = pcg_interleaved(A, M, b, eps=1e-12, maxiter=20000)
        tol = 1e-12
    else:
        raise SystemExit("part must be 'fixed' or 'tight'")
    bn = float(np.linalg.norm(b))
    out = {
        "workload": "box256x256x128, depth 0.004, grading 1.05, lambda2 1e-2, beta exp(-z/0.005), "
                    "rhs uniform(seed 0) + sin(2 pi x) cos(2 pi y) zeta",
        "solver": "oracle pcg_interleaved (Algorithm 1), line preconditioner, x0 = 0",
        "tol": tol,
        "maxiter": ITERS if part == "fixed" else 20000,
        "iterations": res.iterations,
        "converged": bool(res.converged),
        "relres_recursive": res.residual_history[-1] / bn,
        "relres_true": res.final_true_relres,
        "oracle_seconds": time.time() - t0,
        "sample_seed": SAMPLE_SEED,
    }
    out.update(digest(res.x, sample_cells(p.n_cells)))
    name = "medium_box_fixed%d.json" % ITERS if part == "fixed" else "medium_box_tol1e-12.json"
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(out, f, indent=0)
    print({k: v for k, v in out.items() if k not in ("cells", "x", "level_sums")})


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "fixed")
