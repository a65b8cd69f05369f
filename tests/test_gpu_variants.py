"""Parity of every sweep variant against the oracle.

The solver picks one kernel per sweep at creation (one thread per column,
chunked columns, TMA-staged tiles, persistent TMA pipelines); the PCG_* environment
variables force the others.  Each variant must reproduce the oracle's
Algorithm 1 iterates (FP64, fixed iteration count, 1e-10) and the oracle's
converged solution through the mixed-precision refinement (1e-8), on grids
whose tiles are ragged in x, y and z, on the latitude-longitude band and on
the cubed-sphere panel.
"""
import numpy as np
import pytest

import workloads as W
from oracle.discretisation import FluxOperator, assemble_csr
from oracle.linesolve import LinePreconditioner
from oracle.pcg import pcg_interleaved

pytestmark = pytest.mark.gpu

CASES = [
    ("sinalpha48x40x12", W.box_problem(48, 40, 12, 0.01, alpha="sin")),
    ("latlon72x32x16", W.latlon_problem(72, 32, 16)),
    ("panel40x36x24", W.panel_problem(40, 36, 24)),
    ("box64x64x40", W.box_problem(64, 64, 40, 0.004)),
    ("box44x30x20", W.box_problem(44, 30, 20, 0.01)),      # ragged tiles in x, y and z
    ("box4x6x5", W.box_problem(4, 6, 5, 0.01)),            # one tile wrapping onto itself
]

FP64_VARIANTS = {
    "column-by4": {"PCG_COL_BY": "4"},
    "column-by1": {"PCG_COL_BY": "1"},
    "chunked": {"PCG_KERNELS": "chunked"},
    "spmv-split": {"PCG_SPMV_KSPLIT": "2"},
    "spmv-plain-loop": {"PCG_SPMV_PIPE": "0"},
}

FP32_VARIANTS = {
    "default": {},
    "spmv-column": {"PCG_SPMV": "column"},
    "spmv-chunked": {"PCG_SPMV": "chunked"},
    "spmv-tma-single-stage": {"PCG_SPMV": "tma"},
    "spmv-tma-single-stage-8rows": {"PCG_SPMV": "tma", "PCG_TMA_BY": "8"},
    "prec-chunked": {"PCG_PREC": "chunked"},
    "prec-tma-chunked": {"PCG_PREC": "tma"},
    "all-column": {"PCG_KERNELS": "column"},
}


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU test needs cuda:0"
    return torch


def _oracle(p, b, **kw):
    return pcg_interleaved(FluxOperator(p), LinePreconditioner(assemble_csr(p), p), b, **kw)


def _set(monkeypatch, env):
    for k in ("PCG_COL_BY", "PCG_KERNELS", "PCG_SPMV", "PCG_PREC", "PCG_SPMV_KSPLIT", "PCG_TMA_BY", "PCG_SPMV_PIPE"):
        monkeypatch.delenv(k, raising=False)
    for k, v in env.items():
        monkeypatch.setenv(k, v)


@pytest.mark.parametrize("variant", list(FP64_VARIANTS))
@pytest.mark.parametrize("name,p", CASES, ids=[c[0] for c in CASES])
def test_fp64_variant_iterates(torch_cuda, monkeypatch, variant, name, p):
    import paper_1302_7193_gb300 as pkg
    torch = torch_cuda
    _set(monkeypatch, FP64_VARIANTS[variant])
    b = W.rhs_for(p, seed=3)
    ref = _oracle(p, b, eps=0.0, maxiter=12)
    with pkg.Solver(p) as s:
        x = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
        st = s.solve(torch.from_numpy(b.ravel().copy()).cuda(), x, tol=0.0, maxit=12)
    assert st.iterations == 12
    err = np.linalg.norm(x.cpu().numpy().reshape(p.shape) - ref.x) / np.linalg.norm(ref.x)
    assert err < 1e-10, err


@pytest.mark.parametrize("variant", list(FP32_VARIANTS))
@pytest.mark.parametrize("name,p", CASES, ids=[c[0] for c in CASES])
def test_mixed_variant_solution(torch_cuda, monkeypatch, variant, name, p):
    import paper_1302_7193_gb300 as pkg
    torch = torch_cuda
    _set(monkeypatch, FP32_VARIANTS[variant])
    b = W.rhs_for(p, seed=4)
    ref = _oracle(p, b, eps=1e-12, maxiter=20000)
    with pkg.Solver(p, precision="mixed") as s:
        x = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
        st = s.solve(torch.from_numpy(b.ravel().copy()).cuda(), x, tol=1e-10, maxit=20000)
    assert st.status == 0, st
    err = np.linalg.norm(x.cpu().numpy().reshape(p.shape) - ref.x) / np.linalg.norm(ref.x)
    assert err < 1e-8, (err, st)


def test_multi_rhs_tma_sweeps_match_single(torch_cuda):
    """The TMA tensor maps fold the right-hand side into the level index:
    three right-hand sides solved together give each one's single solve
    bitwise (the halo copies at rhs boundaries must not leak)."""
    import paper_1302_7193_gb300 as pkg
    torch = torch_cuda
    p = W.box_problem(64, 40, 24, 0.004)
    bs = [W.rhs_for(p, seed=10 + i) for i in range(3)]
    with pkg.Solver(p, nrhs=3, precision="mixed") as s:
        xb = torch.zeros(3 * p.n_cells, dtype=torch.float64, device="cuda")
        s.solve(torch.from_numpy(np.concatenate([b.ravel() for b in bs])).cuda(), xb, tol=1e-9, maxit=20000)
    xb = xb.cpu().numpy().reshape(3, -1)
    with pkg.Solver(p, precision="mixed") as s1:
        for i, b in enumerate(bs):
            x1 = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
            s1.solve(torch.from_numpy(b.ravel().copy()).cuda(), x1, tol=1e-9, maxit=20000)
            assert np.array_equal(x1.cpu().numpy(), xb[i]), i


@pytest.mark.parametrize("p", [W.box_problem(96, 32, 128, 0.004), W.box_problem(64, 64, 40, 0.004),
                               W.box_problem(64, 32, 32, 0.01), W.box_problem(32, 24, 16, 0.01)],
                         ids=["nz128-R1", "nz40-R2-ragged", "nz32-R4", "nz16-R8"])
def test_prec_tables_match_generic_sweep_bitwise(torch_cuda, monkeypatch, p):
    """With one factor set for all columns (uniform box), the FP32
    preconditioner sweep reads the chunk-carry weights from per-level tables
    instead of recomputing them per column; the tables are built with the same
    FP32 operations, so the mixed solve must equal the generic sweep's bitwise
    (items of 1, 2, 4 and 8 rows; a ragged last chunk)."""
    import paper_1302_7193_gb300 as pkg
    torch = torch_cuda
    b = torch.from_numpy(W.rhs_for(p, seed=6).ravel().copy()).cuda()
    xs = []
    for env in ({}, {"PCG_PREC": "tma-generic"}):
        _set(monkeypatch, env)
        with pkg.Solver(p, precision="mixed") as s:
            x = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
            st = s.solve(b, x, tol=1e-10, maxit=20000)
            assert st.status == 0, st
        xs.append(x.cpu().numpy())
    assert np.array_equal(xs[0], xs[1])
