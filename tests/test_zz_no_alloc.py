"""pcg_precond_noalloc: the line preconditioner for callers that cannot
allocate device memory when they call (a CUDA graph being captured, a
real-time loop, device memory owned by another allocator).

It must give what pcg_precond gives on the same grid and input.  Its tables
live in one fixed device array shared by every call, so the test makes calls
on two different grids back to back and then repeats the first: stale tables
from the previous call would show up as a mismatch.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _structs(pkg, p, nrhs=1):
    keep = []
    z, zp = pkg._dbl(p.z_iface)
    be, bp = pkg._dbl(p.beta_iface)
    ae, aep = pkg._dbl(p.alpha_e)
    an, anp = pkg._dbl(p.alpha_n)
    keep += [z, be, ae, an]
    g = pkg.pcg_grid_t(p.kind, p.n_x, p.n_y, p.n_z, nrhs, zp, p.lx, p.ly, p.lat0, p.lat1)
    c = pkg.pcg_coeffs_t(aep, anp, bp, p.lambda2)
    return g, c, keep


def test_noalloc_precond_matches_handle_precond():
    import torch
    assert torch.cuda.is_available(), "GPU test needs cuda:0"
    import paper_1302_7193_gb300 as pkg
    from paper_1302_7193_gb300 import build as B
    B.build()
    lib = pkg.load_library()
    problems = [W.small_box(), W.latlon_problem(96, 40, 24), W.box_problem(40, 24, 12, 0.01, alpha="sin")]
    order = [0, 1, 0, 2]                       # two calls in a row on different grids, then a repeat
    stream = torch.cuda.current_stream().cuda_stream
    for call, idx in enumerate(order):
        p = problems[idx]
        rng = np.random.default_rng(100 + call)
        r = torch.from_numpy(rng.uniform(-1, 1, p.n_cells)).cuda()
        z_ref = torch.empty_like(r)
        with pkg.Solver(p) as s:
            s.precond(r, z_ref)
            torch.cuda.synchronize()
        z = torch.full_like(r, float("nan"))
        g, c, keep = _structs(pkg, p)
        rc = lib.pcg_precond_noalloc(ctypes.byref(g), ctypes.byref(c), ctypes.c_void_p(r.data_ptr()),
                                     ctypes.c_void_p(z.data_ptr()), ctypes.c_void_p(stream))
        assert rc == pkg.PCG_OK, lib.pcg_last_error(None).decode()
        torch.cuda.synchronize()
        zn, zr = z.cpu().numpy(), z_ref.cpu().numpy()
        assert np.isfinite(zn).all()
        assert np.linalg.norm(zn - zr) / np.linalg.norm(zr) < 1e-10, (call, p.name)


def test_noalloc_precond_rejects_grids_beyond_its_scratch():
    import torch
    assert torch.cuda.is_available(), "GPU test needs cuda:0"
    import paper_1302_7193_gb300 as pkg
    lib = pkg.load_library()
    p = W.large_box(scale=4)                   # 256 x 256 x 128 with a varying alpha: per-column factors
    g, c, keep = _structs(pkg, p)
    r = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
    z = torch.zeros_like(r)
    rc = lib.pcg_precond_noalloc(ctypes.byref(g), ctypes.byref(c), ctypes.c_void_p(r.data_ptr()),
                                 ctypes.c_void_p(z.data_ptr()), None)
    assert rc == pkg.PCG_ERR_INVALID_ARG
    assert "scratch" in lib.pcg_last_error(None).decode()
