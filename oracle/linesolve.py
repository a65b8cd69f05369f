"""Vertical-line preconditioner z = M^{-1} r with M = block-diag(A).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 4.1 of the paper builds the preconditioner by dropping the couplings
between different vertical columns, so that M is block diagonal with one
symmetric tridiagonal block A_T per column; each block is solved on its own.
This oracle forms one tridiagonal system of size n in the column-contiguous
order (blocks separated by zero couplings), factors it once with LAPACK's
partial-pivoting tridiagonal LU (dgttrf) and applies it with dgttrs: the
GTTRF/GTTRS routines the paper's CPU code used (Section 6.2).  It is a
different algorithm from the pivot-free Thomas recurrence of the GPU path.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg.lapack as lapack

from workloads import Problem
from .discretisation import column_blocks


class LinePreconditioner:
    def __init__(self, a, p: Problem):
        self.p = p
        lower, main, upper = column_blocks(a, p)
        self.lower, self.main, self.upper = lower, main, upper
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

    def solve(self, r: np.ndarray) -> np.ndarray:
        """z = M^{-1} r for a canonical-layout vector (any shape with n entries)."""
        shape = np.shape(r)
        rc = self._to_columns(r)
        dl, d, du, du2, ipiv = self._lu
        x, info = lapack.dgttrs(dl, d, du, du2, ipiv, rc)
        if info != 0:
            raise np.linalg.LinAlgError(f"dgttrs failed, info={info}")
        return self._from_columns(x).reshape(shape)

    def __call__(self, r):
        return self.solve(r)
