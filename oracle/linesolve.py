"""Vertical-line preconditioner z = M^{-1} r with M = block-diag(A).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 4.2 of the paper builds the preconditioner by dropping the couplings
between different vertical columns, so that M is block diagonal with one
symmetric tridiagonal block A_T per column; each block is solved on its own.
This oracle forms one tridiagonal system of size n in the column-contiguous
order (blocks separated by zero couplings), factors it once with LAPACK's
partial-pivoting tridiagonal LU (dgttrf) and applies it with dgttrs: the
GTTRF/GTTRS routines the paper's CPU code used (Section 6.2).  It is a
different algorithm from the pivot-free Thomas recurrence of the GPU path.

At strong anisotropy a row's diagonal is the sum of two large vertical
couplings and a much smaller remainder s (the zero-order term plus the
horizontal couplings); stored in FP64 the diagonal keeps s only to a
relative accuracy of about eps * W / s, and the LU inherits that error.  The
solve therefore refines the LU solution with the residual r - M z evaluated
in flux form,
    (M z)_k = s_k z_k + W_k (z_k - z_{k+1}) + W_{k-1} (z_k - z_{k-1}),
which is exact to rounding, until the correction falls below rounding (at
most ``refine_steps`` steps): one step suffices while a column has
horizontal couplings; a column block without them (the coarsest level of the
multigrid hierarchy, condition number ~1e9) needs several.  The returned z is
M^{-1} r to FP64 accuracy.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg.lapack as lapack

from workloads import Problem
from .discretisation import _row_entries, column_blocks, operator_terms


class LinePreconditioner:
    def __init__(self, a, p: Problem, refine_steps: int = 20):
        self.p = p
        self.refine_steps = refine_steps
        lower, main, upper = column_blocks(a, p)
        self.lower, self.main, self.upper = lower, main, upper
        # flux form of the column blocks: remainder s and vertical couplings W
        t = operator_terms(p)
        kk, jj, ii = np.meshgrid(np.arange(p.n_z), np.arange(p.n_y), np.arange(p.n_x), indexing="ij")
        cols, vals = _row_entries(p, t, kk.ravel(), jj.ravel(), ii.ravel())
        own_col = cols[0] % (p.n_x * p.n_y)
        rem = t.area[jj.ravel(), ii.ravel()] * t.mass[kk.ravel()]
        for f in range(1, 5):                       # horizontal neighbours in other columns
            other = (cols[f] % (p.n_x * p.n_y)) != own_col
            rem = rem + np.where(other, -vals[f], 0.0)
        self.s_col = self._to_columns(rem).reshape(-1, p.n_z)
        self.w_col = self._to_columns(-vals[5]).reshape(-1, p.n_z)     # coupling k -> k+1 (0 at the top)
        # column-contiguous flattening: position c * n_z + k
        dl = lower[:, 1:]          # couplings k -> k-1 for k >= 1
        du = upper[:, :-1]         # couplings k -> k+1 for k <= n_z-2
        ncol, nz = main.shape
        dl_full = np.zeros((ncol, nz))
        du_full = np.zeros((ncol, nz))
        dl_full[:, :nz - 1] = dl   # sub-diagonal entry (c*nz+k+1, c*nz+k); last one per block is 0
        du_full[:, :nz - 1] = du   # super-diagonal entry (c*nz+k, c*nz+k+1)
        n = ncol * nz
        dlf = np.ascontiguousarray(dl_full.ravel()[: n - 1])
        duf = np.ascontiguousarray(du_full.ravel()[: n - 1])
        df = np.ascontiguousarray(main.ravel())
        if n == 1:
            dlf = np.zeros(0)
            duf = np.zeros(0)
        out = lapack.dgttrf(dlf, df, duf)
        info = out[-1]
        if info != 0:
            raise np.linalg.LinAlgError(f"dgttrf failed, info={info}")
        self._lu = out[:-1]

    def _to_columns(self, v):
        nz = self.p.n_z
        return np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(nz, -1).T).ravel()

    def _from_columns(self, v):
        nz = self.p.n_z
        return np.ascontiguousarray(v.reshape(-1, nz).T).reshape(self.p.shape)

    def _lu_solve(self, rc):
        dl, d, du, du2, ipiv = self._lu
        x, info = lapack.dgttrs(dl, d, du, du2, ipiv, rc)
        if info != 0:
            raise np.linalg.LinAlgError(f"dgttrs failed, info={info}")
        return x

    def apply_flux(self, zc: np.ndarray) -> np.ndarray:
        """M z in flux form for a column-contiguous vector."""
        z = zc.reshape(-1, self.p.n_z)
        w = self.w_col
        f = w[:, :-1] * (z[:, :-1] - z[:, 1:])          # flux from level k to k+1
        y = self.s_col * z
        y[:, :-1] += f
        y[:, 1:] -= f
        return y.ravel()

    def solve(self, r: np.ndarray) -> np.ndarray:
        """z = M^{-1} r for a canonical-layout vector (any shape with n entries)."""
        shape = np.shape(r)
        rc = self._to_columns(r)
        x = self._lu_solve(rc)
        eps = np.finfo(np.float64).eps
        for _ in range(self.refine_steps):
            d = self._lu_solve(rc - self.apply_flux(x))
            x = x + d
            if np.linalg.norm(d) <= 4 * eps * np.linalg.norm(x):
                break
        return self._from_columns(x).reshape(shape)

    def __call__(self, r):
        return self.solve(r)


def _column_flux(p: Problem, t, j: int, i: int):
    """Flux form of column (j, i)'s block of A: s_k (zero-order term plus the
    couplings to other columns) and W_k (coupling of level k to k+1, 0 at
    the top), from the operator's rows restricted to the column."""
    nx, ny, nz = p.n_x, p.n_y, p.n_z
    k = np.arange(nz)
    cl, vals = _row_entries(p, t, k, np.full(nz, j), np.full(nz, i))
    own = j * nx + i
    s = t.area[j, i] * t.mass
    for f in range(1, 5):                           # horizontal neighbours in other columns
        s = s + np.where((cl[f] % (nx * ny)) != own, -vals[f], 0.0)
    return s, -vals[5]


def _flux_apply(s, w, z):
    f = w[:-1] * (z[:-1] - z[1:])
    y = s * z
    y[:-1] += f
    y[1:] -= f
    return y


def solve_columns(p: Problem, r_cols: np.ndarray, cols) -> np.ndarray:
    """z = M^{-1} r on selected columns only (Section 4.2: each column's
    tridiagonal block A_T solved on its own), for sampled checks of very
    large grids.

    ``cols`` is a (2, m) array of (j, i); ``r_cols`` (m, n_z) holds r on
    those columns.  Each block is taken in flux form (``_column_flux``),
    factored with LAPACK's GTTRF and applied with GTTRS, then refined with the
    flux-form residual until the correction falls below rounding, exactly as
    ``LinePreconditioner`` does for the whole grid.
    """
    t = operator_terms(p)
    nz = p.n_z
    jj, ii = (np.asarray(c, dtype=np.int64) for c in cols)
    r_cols = np.asarray(r_cols, dtype=np.float64).reshape(len(jj), nz)
    out = np.empty_like(r_cols)
    for c in range(len(jj)):
        s, w = _column_flux(p, t, int(jj[c]), int(ii[c]))
        wd = np.concatenate([[0.0], w[:-1]])        # coupling k -> k-1
        main = s + w + wd
        rc = r_cols[c]
        if nz == 1:
            out[c] = rc / main
            continue
        off = -w[:-1]
        dl, d, du, du2, ipiv, info = lapack.dgttrf(off.copy(), main.copy(), off.copy())
        if info != 0:
            raise np.linalg.LinAlgError(f"dgttrf failed, info={info}")

        def lu_solve(b):
            x, inf = lapack.dgttrs(dl, d, du, du2, ipiv, b)
            if inf != 0:
                raise np.linalg.LinAlgError(f"dgttrs failed, info={inf}")
            return x

        x = lu_solve(rc)
        eps = np.finfo(np.float64).eps
        for _ in range(20):
            dx = lu_solve(rc - _flux_apply(s, w, x))
            x = x + dx
            if np.linalg.norm(dx) <= 4 * eps * np.linalg.norm(x):
                break
        out[c] = x
    return out


def apply_columns(p: Problem, z_cols: np.ndarray, cols):
    """M z on selected columns, in flux form, and |M| |z| of every row (the
    scale of a backward-error bound of a tridiagonal solve): two (m, n_z)
    arrays."""
    t = operator_terms(p)
    nz = p.n_z
    jj, ii = (np.asarray(c, dtype=np.int64) for c in cols)
    z_cols = np.asarray(z_cols, dtype=np.float64).reshape(len(jj), nz)
    mz = np.empty_like(z_cols)
    scale = np.empty_like(z_cols)
    for c in range(len(jj)):
        s, w = _column_flux(p, t, int(jj[c]), int(ii[c]))
        z = z_cols[c]
        mz[c] = _flux_apply(s, w, z)
        wd = np.concatenate([[0.0], w[:-1]])
        sc = np.abs(s + w + wd) * np.abs(z)
        sc[:-1] += np.abs(w[:-1] * z[1:])
        sc[1:] += np.abs(w[:-1] * z[:-1])
        scale[c] = sc
    return mz, scale
