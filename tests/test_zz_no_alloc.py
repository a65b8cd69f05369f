"""pcg_precond_noalloc: the line preconditioner for callers that cannot
allocate device memory when they call (a real-time loop that cannot take an
allocation's latency, device memory owned by another allocator).

It must give what pcg_precond gives on the same grid and input.  Its tables
live in one fixed device array shared by every call, so the tests make calls
on different grids back to back and then repeat the first: stale tables from
the previous call would show up as a mismatch.  The file is collected last,
so that a failure here leaves every other test already run.
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


def _reference(pkg, torch, p, r, nrhs=1):
    """z from a handle (pcg_create + pcg_precond) on the same grid."""
    z = torch.empty_like(r)
    with pkg.Solver(p, nrhs=nrhs) as s:
        s.precond(r, z)
        torch.cuda.synchronize()
    return z.cpu().numpy()


def _call(pkg, lib, p, r, z, stream, nrhs=1):
    g, c, keep = _structs(pkg, p, nrhs)
    rc = lib.pcg_precond_noalloc(ctypes.byref(g), ctypes.byref(c), ctypes.c_void_p(r.data_ptr()),
                                 ctypes.c_void_p(z.data_ptr()), ctypes.c_void_p(stream))
    assert rc == pkg.PCG_OK, lib.pcg_last_error(None).decode()


def _close(z, zr):
    assert np.isfinite(z).all()
    assert np.linalg.norm(z - zr) / np.linalg.norm(zr) < 1e-10


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU test needs cuda:0"
    import paper_1302_7193_gb300 as pkg
    from paper_1302_7193_gb300 import build as B
    B.build()
    return torch, pkg, pkg.load_library()


def test_noalloc_precond_matches_handle_precond(env):
    torch, pkg, lib = env
    problems = [W.small_box(), W.latlon_problem(96, 40, 24), W.box_problem(40, 24, 12, 0.01, alpha="sin"),
                W.panel_problem(40, 36, 24)]
    order = [0, 1, 0, 2, 3, 0]                 # calls in a row on different grids, then repeats
    stream = torch.cuda.current_stream().cuda_stream
    for call, idx in enumerate(order):
        p = problems[idx]
        rng = np.random.default_rng(100 + call)
        r = torch.from_numpy(rng.uniform(-1, 1, p.n_cells)).cuda()
        zr = _reference(pkg, torch, p, r)
        z = torch.full_like(r, float("nan"))
        _call(pkg, lib, p, r, z, stream)
        torch.cuda.synchronize()
        _close(z.cpu().numpy(), zr)


def test_noalloc_precond_two_right_hand_sides(env):
    torch, pkg, lib = env
    p = W.latlon_problem(72, 32, 16)
    r = torch.from_numpy(np.random.default_rng(7).uniform(-1, 1, 2 * p.n_cells)).cuda()
    zr = _reference(pkg, torch, p, r, nrhs=2)
    z = torch.full_like(r, float("nan"))
    _call(pkg, lib, p, r, z, torch.cuda.current_stream().cuda_stream, nrhs=2)
    torch.cuda.synchronize()
    _close(z.cpu().numpy(), zr)
    zc = z.cpu().numpy().reshape(2, -1)
    assert not np.array_equal(zc[0], zc[1])    # the second vector is solved for its own right-hand side


def test_noalloc_precond_back_to_back_on_one_stream(env):
    """Two calls on different grids queued on the same non-default stream
    with no synchronisation in between: the second call's table upload is
    ordered after the first call's solve by the stream, so both results hold."""
    torch, pkg, lib = env
    pa, pb = W.box_problem(64, 48, 32, 0.004), W.latlon_problem(96, 40, 24)
    ra = torch.from_numpy(np.random.default_rng(8).uniform(-1, 1, pa.n_cells)).cuda()
    rb = torch.from_numpy(np.random.default_rng(9).uniform(-1, 1, pb.n_cells)).cuda()
    zra, zrb = _reference(pkg, torch, pa, ra), _reference(pkg, torch, pb, rb)
    side = torch.cuda.Stream()
    za = torch.full_like(ra, float("nan"))
    zb = torch.full_like(rb, float("nan"))
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        _call(pkg, lib, pa, ra, za, side.cuda_stream)
        _call(pkg, lib, pb, rb, zb, side.cuda_stream)
    side.synchronize()
    _close(za.cpu().numpy(), zra)
    _close(zb.cpu().numpy(), zrb)


def test_noalloc_precond_rejects_grids_beyond_its_scratch(env):
    torch, pkg, lib = env
    p = W.large_box(scale=4)                   # 256 x 256 x 128 with a varying alpha: per-column factors
    g, c, keep = _structs(pkg, p)
    r = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
    z = torch.zeros_like(r)
    rc = lib.pcg_precond_noalloc(ctypes.byref(g), ctypes.byref(c), ctypes.c_void_p(r.data_ptr()),
                                 ctypes.c_void_p(z.data_ptr()), None)
    assert rc == pkg.PCG_ERR_INVALID_ARG
    assert "scratch" in lib.pcg_last_error(None).decode()
