"""Parity of the single-reduction PCG (PCG_ALG_SINGLE_REDUCTION, the
Chronopoulos-Gear form cited in Section 4.3) with the oracle's
``pcg_single_reduction``.

* Fixed iteration counts: the GPU iterates equal the oracle's to relative
  1e-10 in x, on grids whose tiles' rings wrap around periodic axes, stop at
  Neumann latitude edges, are narrower than a tile (1 x 2 columns) or ragged
  (37 x 13), with per-column factors (panel) and deep columns (128 levels).
* Converged solves (tol 1e-10) equal the oracle's, in about its number of
  iterations, and the reported true residual is the oracle's evaluation.
* A batch of right-hand sides equals its single solves bitwise; b = 0,
  warm starts and maxit = 0 behave as in Algorithm 1's path.
* The mixed form with the single-reduction inner solve (FP32 sweep, excess-
  form Thomas, compensated sums) reaches the FP64 oracle's solution to 1e-8,
  and its batch equals its single solves bitwise.
"""
import numpy as np
import pytest

import workloads as W
from oracle import FluxOperator, LinePreconditioner, assemble_csr, pcg_interleaved, pcg_single_reduction

pytestmark = pytest.mark.gpu

CASES = [
    ("box32x32x16", W.small_box()),
    ("ragged37x13x9", W.box_problem(37, 13, 9, 0.02)),
    ("sinalpha48x40x12", W.box_problem(48, 40, 12, 0.01, alpha="sin")),
    ("latlon72x32x16", W.latlon_problem(72, 32, 16)),
    ("box64x64x128_d0.004", W.medium_box(scale=4)),
    ("tiny1x2x3", W.box_problem(1, 2, 3, 0.01)),
    ("panel40x36x24", W.panel_problem(40, 36, 24)),
]
IDS = [c[0] for c in CASES]


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need cuda:0"
    return torch


def _solver(p, **kw):
    import paper_1302_7193_gb300 as pkg
    return pkg.Solver(p, algorithm="single-reduction", **kw)


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel().copy()).cuda()


def _oracle(p, b, **kw):
    return pcg_single_reduction(FluxOperator(p), LinePreconditioner(assemble_csr(p), p), b, **kw)


@pytest.mark.parametrize("name,p", CASES, ids=IDS)
def test_fixed_iterations(torch_cuda, name, p):
    torch = torch_cuda
    b = W.rhs_for(p, seed=0, smooth=(p.kind == W.GEOM_BOX))
    with _solver(p) as s:
        for k in (1, 4, 25):
            ref = _oracle(p, b, eps=0.0, maxiter=k)
            x = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
            st = s.solve(_dev(torch, b), x, tol=0.0, maxit=k)
            assert st.iterations == k == ref.iterations
            err = np.linalg.norm(x.cpu().numpy().reshape(p.shape) - ref.x) / np.linalg.norm(ref.x)
            assert err < 1e-10, (k, err)


@pytest.mark.parametrize("name,p", CASES, ids=IDS)
def test_converged(torch_cuda, name, p):
    torch = torch_cuda
    b = W.rhs_for(p, seed=0, smooth=(p.kind == W.GEOM_BOX))
    ref = _oracle(p, b, eps=1e-10, maxiter=20000)
    with _solver(p) as s:
        x = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
        st = s.solve(_dev(torch, b), x, tol=1e-10, maxit=20000)
    assert st.status == 0 and st.relres_recursive < 1e-10
    assert abs(st.iterations - ref.iterations) <= 2, (st.iterations, ref.iterations)
    xg = x.cpu().numpy().reshape(p.shape)
    assert np.linalg.norm(xg - ref.x) / np.linalg.norm(ref.x) < 1e-10
    rt = np.linalg.norm(b.ravel() - FluxOperator(p) @ xg) / np.linalg.norm(b)
    assert abs(rt - st.relres_true) <= 1e-3 * rt + 1e-15


def test_batch_equals_single_bitwise(torch_cuda):
    torch = torch_cuda
    p = W.box_problem(40, 24, 12, 0.01)
    bs = W.batched_rhs(p, [0, 5, 9])
    bs[1] *= 1e-3
    with _solver(p, nrhs=3) as s:
        xb = torch.zeros(bs.size, dtype=torch.float64, device="cuda")
        s.solve(_dev(torch, bs), xb, tol=1e-9, maxit=5000)
        stats = [s.pcg_rhs_stats(r) for r in range(3)]
    xb = xb.cpu().numpy().reshape(bs.shape)
    with _solver(p) as s1:
        for r in range(3):
            x1 = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
            st = s1.solve(_dev(torch, bs[r]), x1, tol=1e-9, maxit=5000)
            assert st.iterations == stats[r].iterations
            assert np.array_equal(x1.cpu().numpy().reshape(p.shape), xb[r])


def test_zero_rhs_and_warm_start_and_maxit0(torch_cuda):
    torch = torch_cuda
    p = W.small_box()
    b = W.rhs_for(p, seed=3)
    with _solver(p) as s:
        x = torch.full((p.n_cells,), 7.0, dtype=torch.float64, device="cuda")
        st = s.solve(torch.zeros(p.n_cells, dtype=torch.float64, device="cuda"), x, tol=1e-8, maxit=100)
        assert st.status == 0 and st.iterations == 0 and not x.any()
        x = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
        st = s.solve(_dev(torch, b), x, tol=1e-10, maxit=5000)
        st2 = s.solve(_dev(torch, b), x, tol=1e-8, maxit=5000)   # warm start at the solution
        assert st2.iterations <= 1
        x0 = torch.full((p.n_cells,), 0.25, dtype=torch.float64, device="cuda")
        st3 = s.solve(_dev(torch, b), x0, tol=1e-8, maxit=0)
        assert st3.status == 4 and st3.iterations == 0
        assert bool((x0 == 0.25).all())


@pytest.mark.parametrize("name,p", CASES, ids=IDS)
def test_mixed_matches_fp64_oracle(torch_cuda, name, p):
    torch = torch_cuda
    b = W.rhs_for(p, seed=0, smooth=(p.kind == W.GEOM_BOX))
    ref = pcg_interleaved(FluxOperator(p), LinePreconditioner(assemble_csr(p), p), b, eps=1e-12, maxiter=20000)
    with _solver(p, precision="mixed") as s:
        x = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
        st = s.solve(_dev(torch, b), x, tol=1e-10, maxit=20000)
    assert st.status == 0, st
    err = np.linalg.norm(x.cpu().numpy().reshape(p.shape) - ref.x) / np.linalg.norm(ref.x)
    assert err < 1e-8, (err, st)


def test_mixed_batch_equals_single_bitwise(torch_cuda):
    torch = torch_cuda
    p = W.box_problem(40, 24, 12, 0.01)
    bs = W.batched_rhs(p, [0, 5, 9])
    bs[1] *= 1e-3
    with _solver(p, nrhs=3, precision="mixed") as s:
        xb = torch.zeros(bs.size, dtype=torch.float64, device="cuda")
        s.solve(_dev(torch, bs), xb, tol=1e-9, maxit=5000)
        stats = [s.pcg_rhs_stats(r) for r in range(3)]
    xb = xb.cpu().numpy().reshape(bs.shape)
    with _solver(p, precision="mixed") as s1:
        for r in range(3):
            x1 = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
            st = s1.solve(_dev(torch, bs[r]), x1, tol=1e-9, maxit=5000)
            assert st.iterations == stats[r].iterations and st.outer_sweeps == stats[r].outer_sweeps
            assert np.array_equal(x1.cpu().numpy().reshape(p.shape), xb[r])
