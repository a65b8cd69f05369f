"""The C-ABI library loads and exports every entry point of include/pcg.h, and
its host-side argument checks reject bad input before touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1302_7193_gb300 as pkg
import workloads as W
from paper_1302_7193_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return pkg.load_library()


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "pcg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pcg_[A-Za-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("pcg_create", "pcg_solve", "pcg_apply_A", "pcg_precond", "pcg_destroy", "pcg_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert names
    for name in names:
        assert hasattr(lib, name), name
    assert set(pkg.EXPORTED) == set(names)


def _create(p, **over):
    z, zp = pkg._dbl(p.z_iface)
    be, bp = pkg._dbl(p.beta_iface)
    g = pkg.pcg_grid_t(p.kind, p.n_x, p.n_y, p.n_z, 1, zp, 1.0, 1.0, p.lat0, p.lat1)
    c = pkg.pcg_coeffs_t(None, None, bp, p.lambda2)
    o = pkg.pcg_opts_t(0, 0.0, 0, 0, 0, None)
    for k, v in over.items():
        setattr(g if hasattr(g, k) else (o if hasattr(o, k) else c), k, v)
    h = ctypes.c_void_p()
    lib = pkg.load_library()
    rc = lib.pcg_create(ctypes.byref(g), ctypes.byref(c), ctypes.byref(o), ctypes.byref(h))
    return rc, h, lib.pcg_last_error(None).decode(), (z, be)


@pytest.mark.parametrize("field,value", [("n_x", 0), ("n_z", 0), ("nrhs", 0), ("lambda2", -1.0),
                                         ("geometry", 7), ("lambda2", float("nan"))])
def test_create_rejects_bad_arguments(lib, field, value):
    rc, h, msg, _ = _create(W.small_box(), **{field: value})
    assert rc == pkg.PCG_ERR_INVALID_ARG and not h.value, (rc, msg)
    assert msg


@pytest.mark.parametrize("over", [{"preconditioner": 5}, {"preconditioner": 1, "precision": 1}, {"precision": 3},
                                  {"algorithm": 2}, {"algorithm": 1, "preconditioner": 1},
                                  {"algorithm": 1, "preconditioner": 2}])
def test_create_rejects_bad_options(lib, over):
    # unknown preconditioner; multigrid is FP64 only; unknown precision; unknown
    # algorithm; the single-reduction sweep has the line preconditioner only
    rc, h, msg, _ = _create(W.small_box(), **over)
    assert rc == pkg.PCG_ERR_INVALID_ARG and not h.value, (rc, msg)
    assert msg


def test_single_reduction_rejects_deep_columns(lib):
    # its sweep keeps n_z x 108 doubles of u in shared memory
    rc, h, msg, _ = _create(W.box_problem(4, 4, 300, 0.01), algorithm=pkg.PCG_ALG_SINGLE_REDUCTION)
    assert rc == pkg.PCG_ERR_INVALID_ARG and "n_z <= 256" in msg


def test_create_rejects_non_monotone_levels(lib):
    p = W.small_box()
    p.z_iface = p.z_iface.copy()
    p.z_iface[3] = p.z_iface[2]
    rc, h, msg, _ = _create(p)
    assert rc == pkg.PCG_ERR_INVALID_ARG and "increasing" in msg


def test_create_rejects_bad_latitude_band(lib):
    p = W.latlon_problem(8, 4, 4)
    p.lat1 = 2.0
    rc, h, msg, _ = _create(p)
    assert rc == pkg.PCG_ERR_INVALID_ARG and "latitude" in msg


def test_null_handle_calls_fail_cleanly(lib):
    st = pkg.pcg_stats_t()
    assert lib.pcg_solve(None, None, None, 1e-8, 10, ctypes.byref(st)) == pkg.PCG_ERR_INVALID_ARG
    assert lib.pcg_apply_A(None, None, None) == pkg.PCG_ERR_INVALID_ARG
    assert lib.pcg_precond(None, None, None) == pkg.PCG_ERR_INVALID_ARG
    assert lib.pcg_device_bytes(None) == 0
    lib.pcg_destroy(None)


def test_binding_refuses_missing_library(tmp_path):
    saved = pkg._lib
    pkg._lib = None
    try:
        with pytest.raises(ImportError):
            pkg.load_library(str(tmp_path / "libpcg.so"))
    finally:
        pkg._lib = saved


def test_structs_match_header_layout(tmp_path):
    # size and field offsets of every ctypes mirror equal the C structs of
    # include/pcg.h as the C compiler lays them out
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"pcg_grid_t": pkg.pcg_grid_t, "pcg_coeffs_t": pkg.pcg_coeffs_t, "pcg_opts_t": pkg.pcg_opts_t,
               "pcg_stats_t": pkg.pcg_stats_t}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pcg.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        name, field, val = line.split()
        got[(name, field)] = int(val)
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)


def _noalloc_structs(p, alpha=None):
    keep = []
    z, zp = pkg._dbl(p.z_iface)
    be, bp = pkg._dbl(p.beta_iface)
    keep += [z, be]
    ap = None
    if alpha is not None:
        a, ap = pkg._dbl(alpha)
        keep.append(a)
    g = pkg.pcg_grid_t(p.kind, p.n_x, p.n_y, p.n_z, 1, zp, p.lx, p.ly, p.lat0, p.lat1)
    c = pkg.pcg_coeffs_t(ap, None, bp, p.lambda2)
    return g, c, keep


def test_noalloc_precond_rejects_bad_arguments_before_the_device(lib):
    """pcg_precond_noalloc checks its arguments and the size of its fixed
    scratch on the host, before any CUDA call: each bad case returns
    PCG_ERR_INVALID_ARG with its reason.  The vector pointers are never
    dereferenced on these paths (skipped where a GPU is present, so that no
    kernel could ever be handed them)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("host-only argument checks; the GPU path is covered by test_zz_no_alloc.py")
    r = z = ctypes.c_void_p(256)

    def call(g, c, rr=r, zz=z):
        rc = lib.pcg_precond_noalloc(ctypes.byref(g) if g is not None else None,
                                     ctypes.byref(c) if c is not None else None, rr, zz, None)
        return rc, lib.pcg_last_error(None).decode()

    p = W.small_box()
    g, c, keep = _noalloc_structs(p)
    for args in ((None, c), (g, None)):
        rc, msg = call(*args)
        assert rc == pkg.PCG_ERR_INVALID_ARG and "required" in msg
    rc, msg = call(g, c, rr=None)
    assert rc == pkg.PCG_ERR_INVALID_ARG and "required" in msg
    g.geometry = 7
    rc, msg = call(g, c)
    assert rc == pkg.PCG_ERR_INVALID_ARG and "geometry" in msg
    g, c, keep = _noalloc_structs(p)
    c.lambda2 = float("nan")
    rc, msg = call(g, c)
    assert rc == pkg.PCG_ERR_INVALID_ARG and "lambda2" in msg
    g, c, keep = _noalloc_structs(p)
    g.n_z = 0
    rc, msg = call(g, c)
    assert rc == pkg.PCG_ERR_INVALID_ARG and ">= 1" in msg
    # per-column factors of a 256 x 256 x 128 grid need 3 * 128 * 65536 doubles
    big = W.box_problem(256, 256, 128, 0.004)
    g, c, keep = _noalloc_structs(big, alpha=np.ones(big.n_x * big.n_y))
    rc, msg = call(g, c)
    assert rc == pkg.PCG_ERR_INVALID_ARG and "scratch" in msg, msg
    assert str(3 * 128 * 65536 + 3 * 128 + 256 + 2 * 65536) in msg
