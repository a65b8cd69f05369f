"""The two large configurations at full size, in the launch configuration
bench.py times, checked where the oracle cannot run whole:

* sampled outputs, each computed by the oracle on its own: operator rows
  (``apply_rows``) and column solves of the preconditioner
  (``solve_columns``, ``apply_columns`` for the backward error);
* properties that hold at any size: the mixed-precision solve and the FP64
  solve of the same system agree, and both reach the stopping test or the
  rounding floor.

Box: 1024 x 1024 x 128 with alpha = 1 + 0.5 sin(2 pi x) sin(2 pi y).
Band: 1440 x 640 x 64 latitude-longitude band of the shell r in [1, 1.002],
two right-hand sides solved together.

The 256 x 256 x 128 benchmark box is small enough for the oracle to solve
whole (tests/golden/make_medium_box_digest.py, about half an hour of one
core): its solutions after exactly the oracle's 641 iterations and at tol
1e-12 are stored as digests (2-norm, per-level sums, x at 4096 seeded cells),
and the GPU solves of the same problem are compared with them at full size.
"""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import apply_columns, apply_rows, solve_columns

pytestmark = pytest.mark.gpu

EPS64 = np.finfo(np.float64).eps
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU test needs cuda:0"
    return torch


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a).ravel().copy()).cuda()


def _sampled_checks(torch, s, p, seed):
    """Operator rows and column solves at sampled places of a full-size grid."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, p.shape)
    cells = np.stack([rng.integers(0, n, 3000) for n in p.shape])
    y = torch.empty(p.n_cells, dtype=torch.float64, device="cuda")
    s.apply_A(_dev(torch, x), y)
    yg = y.cpu().numpy().reshape(p.shape)[tuple(cells)]
    yo = apply_rows(p, x, cells)
    assert np.allclose(yg, yo, rtol=1e-12, atol=1e-12 * np.abs(yo).max())
    # preconditioner: 48 sampled columns
    r = rng.uniform(-1, 1, p.shape)
    z = torch.empty(p.n_cells, dtype=torch.float64, device="cuda")
    s.precond(_dev(torch, r), z)
    zg = z.cpu().numpy().reshape(p.shape)
    cols = np.stack([rng.integers(0, p.n_y, 48), rng.integers(0, p.n_x, 48)])
    r_cols = np.stack([r[:, j, i] for j, i in cols.T])
    z_cols = np.stack([zg[:, j, i] for j, i in cols.T])
    mz, scale = apply_columns(p, z_cols, cols)
    assert (np.abs(mz - r_cols) <= 16 * p.n_z * EPS64 * scale).all()        # backward error
    zo = solve_columns(p, r_cols, cols)
    assert np.linalg.norm(z_cols - zo) / np.linalg.norm(zo) < 1e-10          # forward, vs oracle


def _reached(st, tol):
    return st.status == 0 and (st.relres_true < tol or st.relres_true <= 2.0 * st.relres_floor)


def test_large_box_full_size(torch_cuda):
    import paper_1302_7193_gb300 as pkg
    torch = torch_cuda
    p = W.large_box()
    b = W.rhs_for(p, seed=0)
    with pkg.Solver(p) as s:
        _sampled_checks(torch, s, p, seed=21)
        xf = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
        stf = s.solve(_dev(torch, b), xf, tol=1e-8, maxit=100000)
    with pkg.Solver(p, precision="mixed") as s:
        xm = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
        stm = s.solve(_dev(torch, b), xm, tol=1e-8, maxit=100000)
    # FP64 stops on the updated residual (Algorithm 1); its true residual sits
    # a little above it at this grading
    assert stf.status == 0 and stf.relres_recursive < 1e-8 and stf.relres_true < 1e-7, stf
    assert _reached(stm, 1e-8), stm
    rel = (torch.linalg.norm(xm - xf) / torch.linalg.norm(xf)).item()
    assert rel < 1e-7, rel


def test_shell_band_full_size(torch_cuda):
    import paper_1302_7193_gb300 as pkg
    torch = torch_cuda
    p = W.latlon_problem(1440, 640, 64)
    bs = W.batched_rhs(p, [0, 1])
    with pkg.Solver(p) as s:
        _sampled_checks(torch, s, p, seed=22)
    with pkg.Solver(p, nrhs=2, precision="mixed") as s:
        xm = torch.zeros(bs.size, dtype=torch.float64, device="cuda")
        s.solve(_dev(torch, bs), xm, tol=1e-8, maxit=100000)
        stm = [s.pcg_rhs_stats(r) for r in range(2)]
    with pkg.Solver(p, nrhs=2) as s:
        xf = torch.zeros(bs.size, dtype=torch.float64, device="cuda")
        s.solve(_dev(torch, bs), xf, tol=1e-8, maxit=100000)
        stf = [s.pcg_rhs_stats(r) for r in range(2)]
    n = p.n_cells
    for r in range(2):
        assert _reached(stm[r], 1e-8), stm[r]
        # after ~4600 FP64 iterations the updated residual has drifted from the
        # true one (CG's attainable accuracy on this band: true ~7e-7 measured)
        assert stf[r].status == 0 and stf[r].relres_recursive < 1e-8 and stf[r].relres_true < 1e-5, stf[r]
        d = (torch.linalg.norm(xm[r * n:(r + 1) * n] - xf[r * n:(r + 1) * n]) /
             torch.linalg.norm(xf[r * n:(r + 1) * n])).item()
        assert d < 1e-7, (r, d)


def _digest(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _against_digest(x, d, n_z):
    """Relative distance of a full solution x from an oracle digest: on the
    sampled cells, in the 2-norm and in the per-level sums."""
    x = np.asarray(x, dtype=np.float64).ravel()
    xo = np.array(d["x"])
    e_cells = np.linalg.norm(x[np.array(d["cells"])] - xo) / np.linalg.norm(xo)
    e_norm = abs(np.linalg.norm(x) - d["norm2"]) / d["norm2"]
    lo = np.array(d["level_sums"])
    e_levels = np.abs(x.reshape(n_z, -1).sum(axis=1) - lo).max() / np.abs(lo).max()
    return e_cells, e_norm, e_levels


def test_medium_box_fixed_count_matches_oracle(torch_cuda):
    """Algorithm 1 (Section 4.3) on the 256 x 256 x 128 box with both sides
    taking exactly the oracle's 641 iterations (tol = 0): the FP64 solution
    equals the oracle's to 1e-10 relative."""
    import paper_1302_7193_gb300 as pkg
    torch = torch_cuda
    p = W.medium_box()
    d = _digest("medium_box_fixed641.json")
    assert d["iterations"] == 641 and d["tol"] == 0.0
    with pkg.Solver(p) as s:
        x = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
        st = s.solve(_dev(torch, W.medium_box_rhs(p)), x, tol=0.0, maxit=641)
    assert st.iterations == 641, st
    errs = _against_digest(x.cpu().numpy(), d, p.n_z)
    assert max(errs) < 1e-10, errs


def test_medium_box_tight_solves_match_oracle(torch_cuda):
    """Both sides solve the 256 x 256 x 128 box to tol 1e-12: the FP64 solution
    equals the oracle's to 1e-10; the mixed-precision solution (FP64
    refinement to the same tolerance, or to the FP64 rounding floor) equals it
    to 1e-8.  The iteration counts agree only loosely: the updated residual
    passes 1e-12 about 100 iterations after the true residual has stopped
    falling (at 2e-6, CG's attainable accuracy here), and in that stretch it
    follows the rounding of each implementation (oracle 779, GPU 740)."""
    import paper_1302_7193_gb300 as pkg
    torch = torch_cuda
    p = W.medium_box()
    d = _digest("medium_box_tol1e-12.json")
    assert d["converged"] and d["tol"] == 1e-12
    b = _dev(torch, W.medium_box_rhs(p))
    with pkg.Solver(p) as s:
        x = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
        st = s.solve(b, x, tol=1e-12, maxit=20000)
    assert st.status == 0 and st.relres_recursive < 1e-12, st
    assert abs(st.iterations - d["iterations"]) <= 0.1 * d["iterations"], (st, d["iterations"])
    errs = _against_digest(x.cpu().numpy(), d, p.n_z)
    assert max(errs) < 1e-10, errs
    with pkg.Solver(p, precision="mixed") as s:
        x.zero_()
        st = s.solve(b, x, tol=1e-12, maxit=20000)
    assert st.status == 0 and (st.relres_true < 1e-12 or st.relres_true <= 2.0 * st.relres_floor), st
    errs = _against_digest(x.cpu().numpy(), d, p.n_z)
    assert max(errs) < 1e-8, errs
