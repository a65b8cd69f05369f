"""Parity of the multigrid preconditioner (PCG_PREC_MULTIGRID) with the oracle.

* One V-cycle on the GPU (pcg_precond of a multigrid handle) equals the
  oracle's V-cycle, on grids that coarsen down to one column (periodic box)
  and on grids whose coarsest level keeps many columns (odd sizes: smoothing
  sweeps there), including the latitude-longitude band and the panel.
* Algorithm 1 with the V-cycle as preconditioner reproduces the oracle's
  iterates at a fixed iteration count, and the converged solution equals the
  oracle's solution of the same system in a number of iterations close to
  the oracle's.
* The FP32 V-cycle (PCG_PREC_MULTIGRID_F32) agrees with the oracle's FP64
  V-cycle to FP32 accuracy, and the FP64 CG around it still reaches the
  oracle's solution.
"""
import numpy as np
import pytest

import workloads as W
from oracle import FluxOperator, assemble_csr, pcg_interleaved
from oracle.linesolve import LinePreconditioner
from oracle.multigrid import MultigridPreconditioner

pytestmark = pytest.mark.gpu

CASES = [
    ("box32x32x16", W.small_box()),
    ("sinalpha48x40x12", W.box_problem(48, 40, 12, 0.01, alpha="sin")),
    ("latlon72x32x16", W.latlon_problem(72, 32, 16)),
    ("panel40x36x24", W.panel_problem(40, 36, 24)),
    ("box64x64x128", W.medium_box(scale=4)),
]
IDS = [c[0] for c in CASES]


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU test needs cuda:0"
    return torch


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel().copy()).cuda()


@pytest.mark.parametrize("name,p", CASES, ids=IDS)
def test_vcycle_matches_oracle(torch_cuda, name, p):
    import paper_1302_7193_gb300 as pkg
    torch = torch_cuda
    r = np.random.default_rng(5).uniform(-1, 1, p.shape)
    with pkg.Solver(p, preconditioner="multigrid") as s:
        z = torch.empty(p.n_cells, dtype=torch.float64, device="cuda")
        s.precond(_dev(torch, r), z)
        zg = z.cpu().numpy().reshape(p.shape)
        # twice in a row: the V-cycle leaves nothing behind that changes the next one
        s.precond(_dev(torch, r), z)
        assert np.array_equal(z.cpu().numpy().reshape(p.shape), zg)
    zo = MultigridPreconditioner(p)(r)
    err = np.linalg.norm(zg - zo) / np.linalg.norm(zo)
    assert err < 1e-10, err


@pytest.mark.parametrize("name,p", CASES, ids=IDS)
def test_mg_pcg_fixed_iterations(torch_cuda, name, p):
    import paper_1302_7193_gb300 as pkg
    torch = torch_cuda
    b = W.rhs_for(p, seed=0)
    mg = MultigridPreconditioner(p)
    with pkg.Solver(p, preconditioner="multigrid") as s:
        for k in (1, 3, 8):
            ref = pcg_interleaved(FluxOperator(p), mg, b, eps=0.0, maxiter=k)
            x = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
            st = s.solve(_dev(torch, b), x, tol=0.0, maxit=k)
            assert st.iterations == k == ref.iterations
            err = np.linalg.norm(x.cpu().numpy().reshape(p.shape) - ref.x) / np.linalg.norm(ref.x)
            assert err < 1e-10, (k, err)


@pytest.mark.parametrize("name,p", CASES, ids=IDS)
def test_mg_pcg_converged(torch_cuda, name, p):
    import paper_1302_7193_gb300 as pkg
    torch = torch_cuda
    b = W.rhs_for(p, seed=1)
    a = FluxOperator(p)
    ref_mg = pcg_interleaved(a, MultigridPreconditioner(p), b, eps=1e-10, maxiter=2000)
    ref = pcg_interleaved(a, LinePreconditioner(assemble_csr(p), p), b, eps=1e-12, maxiter=20000)
    with pkg.Solver(p, preconditioner="multigrid") as s:
        x = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
        st = s.solve(_dev(torch, b), x, tol=1e-10, maxit=2000)
    assert st.status == 0 and st.relres_recursive < 1e-10, st
    assert abs(st.iterations - ref_mg.iterations) <= 2, (st.iterations, ref_mg.iterations)
    xg = x.cpu().numpy().reshape(p.shape)
    assert np.linalg.norm(xg - ref.x) / np.linalg.norm(ref.x) < 1e-8


def test_mg_batch_equals_single_bitwise(torch_cuda):
    import paper_1302_7193_gb300 as pkg
    torch = torch_cuda
    p = W.box_problem(32, 16, 12, 0.01)
    bs = W.batched_rhs(p, [0, 5, 9])
    bs[1] *= 1e-3
    with pkg.Solver(p, nrhs=3, preconditioner="multigrid") as s:
        xb = torch.zeros(bs.size, dtype=torch.float64, device="cuda")
        s.solve(_dev(torch, bs), xb, tol=1e-9, maxit=500)
        stats = [s.pcg_rhs_stats(r) for r in range(3)]
    xb = xb.cpu().numpy().reshape(bs.shape)
    with pkg.Solver(p, preconditioner="multigrid") as s1:
        for r in range(3):
            x1 = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
            st = s1.solve(_dev(torch, bs[r]), x1, tol=1e-9, maxit=500)
            assert st.iterations == stats[r].iterations
            assert np.array_equal(x1.cpu().numpy().reshape(p.shape), xb[r])


@pytest.mark.parametrize("name,p", CASES, ids=IDS)
def test_fp32_vcycle_inside_fp64_cg(torch_cuda, name, p):
    """PCG_PREC_MULTIGRID_F32: the V-cycle in FP32 (r rounded on the way in,
    z widened on the way out) inside the FP64 CG.  The cycle agrees with the
    oracle's FP64 V-cycle to FP32 accuracy; the FP64 CG still reaches the
    oracle's solution, in about the oracle's number of multigrid iterations."""
    import paper_1302_7193_gb300 as pkg
    torch = torch_cuda
    r = np.random.default_rng(6).uniform(-1, 1, p.shape)
    mg = MultigridPreconditioner(p)
    b = W.rhs_for(p, seed=1)
    a = FluxOperator(p)
    ref_mg = pcg_interleaved(a, mg, b, eps=1e-10, maxiter=2000)
    ref = pcg_interleaved(a, LinePreconditioner(assemble_csr(p), p), b, eps=1e-12, maxiter=20000)
    with pkg.Solver(p, preconditioner="multigrid-f32") as s:
        z = torch.empty(p.n_cells, dtype=torch.float64, device="cuda")
        s.precond(_dev(torch, r), z)
        zo = mg(r)
        err = np.linalg.norm(z.cpu().numpy().reshape(p.shape) - zo) / np.linalg.norm(zo)
        assert err < 1e-4, err
        x = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
        st = s.solve(_dev(torch, b), x, tol=1e-10, maxit=2000)
    assert st.status == 0 and st.relres_recursive < 1e-10, st
    # The FP32 cycle is symmetric only to FP32 rounding, so CG loses some of its
    # short-recurrence orthogonality as the residual falls towards 1e-10: about
    # 20 % more iterations than the FP64 cycle there (none to 4 at 1e-8).
    assert st.iterations <= 1.3 * ref_mg.iterations + 3, (st.iterations, ref_mg.iterations)
    xg = x.cpu().numpy().reshape(p.shape)
    assert np.linalg.norm(xg - ref.x) / np.linalg.norm(ref.x) < 1e-8


def test_mg_f32_batch_equals_single_bitwise(torch_cuda):
    import paper_1302_7193_gb300 as pkg
    torch = torch_cuda
    p = W.box_problem(32, 16, 12, 0.01)
    bs = W.batched_rhs(p, [0, 5, 9])
    bs[1] *= 1e-3
    with pkg.Solver(p, nrhs=3, preconditioner="multigrid-f32") as s:
        xb = torch.zeros(bs.size, dtype=torch.float64, device="cuda")
        s.solve(_dev(torch, bs), xb, tol=1e-9, maxit=500)
        stats = [s.pcg_rhs_stats(r) for r in range(3)]
    xb = xb.cpu().numpy().reshape(bs.shape)
    with pkg.Solver(p, preconditioner="multigrid-f32") as s1:
        for r in range(3):
            x1 = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
            st = s1.solve(_dev(torch, bs[r]), x1, tol=1e-9, maxit=500)
            assert st.iterations == stats[r].iterations
            assert np.array_equal(x1.cpu().numpy().reshape(p.shape), xb[r])


FUSED = {"PCG_MG_TAIL": "4096", "PCG_MG_QUAD": "1"}      # the fused kernels on every level that allows them
SEPARATE = {"PCG_MG_TAIL": "0", "PCG_MG_QUAD": "0"}      # one launch per step, scalar residuals


@pytest.mark.parametrize("prec", ["multigrid", "multigrid-f32"])
@pytest.mark.parametrize("name,p", CASES, ids=IDS)
def test_fused_vcycle_matches_separate_launches_bitwise(torch_cuda, monkeypatch, name, p, prec):
    """The smallest levels in one launch (k_mg_tail) and the FP32 residuals on
    float4 quads of row pairs (k_mg_resid4, here on every level whose shape
    allows it) against one launch per step with the scalar kernels
    (PCG_MG_TAIL=0, PCG_MG_QUAD=0).  Both plans do the same arithmetic in the
    same order, so the V-cycles and the CG iterates built on them agree bit
    for bit, and the fused plan makes fewer launches."""
    import paper_1302_7193_gb300 as pkg
    torch = torch_cuda
    r = np.random.default_rng(7).uniform(-1, 1, p.shape)
    b = W.rhs_for(p, seed=2)
    out = []
    for plan in (FUSED, SEPARATE):
        for k, v in plan.items():
            monkeypatch.setenv(k, v)
        with pkg.Solver(p, preconditioner=prec) as s:
            z = torch.empty(p.n_cells, dtype=torch.float64, device="cuda")
            s.precond(_dev(torch, r), z)
            x = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
            st = s.solve(_dev(torch, b), x, tol=0.0, maxit=6)
            out.append((z.cpu().numpy(), x.cpu().numpy(), st.iterations, s.kernel_launches))
    (z1, x1, it1, n1), (z0, x0, it0, n0) = out
    assert np.array_equal(z1, z0)
    assert it1 == it0 == 6 and np.array_equal(x1, x0)
    assert n1 < n0, (n1, n0)


def test_fused_vcycle_batched(torch_cuda, monkeypatch):
    """Three right-hand sides, one of them stopped early: the batched FP32
    cycle inside CG equals the separate launches bit for bit."""
    import paper_1302_7193_gb300 as pkg
    torch = torch_cuda
    p = W.box_problem(32, 16, 12, 0.01)
    bs = W.batched_rhs(p, [0, 5, 9])
    bs[1] *= 1e-3
    xs = []
    for plan in (FUSED, SEPARATE):
        for k, v in plan.items():
            monkeypatch.setenv(k, v)
        with pkg.Solver(p, nrhs=3, preconditioner="multigrid-f32") as s:
            xb = torch.zeros(bs.size, dtype=torch.float64, device="cuda")
            s.solve(_dev(torch, bs), xb, tol=1e-9, maxit=500)
            xs.append((xb.cpu().numpy(), [s.pcg_rhs_stats(k).iterations for k in range(3)]))
    assert xs[0][1] == xs[1][1]
    assert np.array_equal(xs[0][0], xs[1][0])
