"""Geometric multigrid with vertical line smoothing, as a preconditioner for CG.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper closes (Section 8) with multigrid as the next solver for these
equations, its line preconditioner as the smoother and restriction and
prolongation as the missing pieces; Section 2 points to the tensor-product
multigrid of Boerm and Hiptmair for this anisotropy.  The vertical-line
smoother removes the strong vertical coupling, so what is left is an
isotropic horizontal problem, which a hierarchy of horizontally coarsened
grids solves in a number of iterations that does not grow with the grid.
This module states that V-cycle plainly:

* Hierarchy: n_x and n_y halved per level while both are even, the
  vertical grid kept; each level's operator is the same discretisation on
  the coarser grid (``coarse_problem``), so every level has the structure of
  the fine one (flux-form operator, tridiagonal column blocks).
* Transfer: restriction R sums the four fine cells of a coarse cell (the
  finite-volume rows are cell integrals, so the coarse right-hand side is
  the sum of the fine residuals); prolongation P = R^T copies a coarse value
  to its four fine cells.
* Smoother: damped block Jacobi with the column blocks,
  z <- z + omega M^{-1} (r - A z), nu sweeps before and nu after the coarse
  correction, the first from z = 0.
* Coarsest level: M^{-1} itself when the level is a single column (its
  block is all of A there; ``LinePreconditioner`` refines it to rounding),
  otherwise ``coarsest_sweeps`` smoother sweeps.

With R = P^T and the same number of Jacobi sweeps on both sides, the V-cycle
applied to r from a zero guess is a symmetric positive definite operator B,
so CG preconditioned by B converges (Section 4.1's PCG with M replaced by B).
"""
from __future__ import annotations

import dataclasses
from typing import List

import numpy as np

from workloads import Problem
from .discretisation import FluxOperator, assemble_csr
from .linesolve import LinePreconditioner


def coarse_problem(p: Problem) -> Problem:
    """The same problem on the grid with n_x and n_y halved (both even).

    Vertical grid and profiles are unchanged.  Where alpha is given as face
    values, a coarse face takes the mean of the two fine faces it is made of:
    the east face of coarse cell (I, J) is made of the east faces of fine
    cells (2I+1, 2J) and (2I+1, 2J+1), its north face of the north faces of
    (2I, 2J+1) and (2I+1, 2J+1).
    """
    if p.n_x % 2 or p.n_y % 2:
        raise ValueError("coarsening needs even n_x and n_y")
    ae = an = None
    if p.alpha_e is not None:
        a = np.asarray(p.alpha_e, dtype=np.float64)
        ae = np.ascontiguousarray(0.5 * (a[0::2, 1::2] + a[1::2, 1::2]))
    if p.alpha_n is not None:
        a = np.asarray(p.alpha_n, dtype=np.float64)
        an = np.ascontiguousarray(0.5 * (a[1::2, 0::2] + a[1::2, 1::2]))
    return dataclasses.replace(p, n_x=p.n_x // 2, n_y=p.n_y // 2, alpha_e=ae, alpha_n=an,
                               name=(p.name or "p") + "/2")


def restrict(r: np.ndarray) -> np.ndarray:
    """Sum of the four fine cells of every coarse cell, per level: (n_z, n_y, n_x) -> (n_z, n_y/2, n_x/2)."""
    return r[:, 0::2, 0::2] + r[:, 0::2, 1::2] + r[:, 1::2, 0::2] + r[:, 1::2, 1::2]


def prolong(e: np.ndarray) -> np.ndarray:
    """Copy of every coarse value to its four fine cells (the transpose of ``restrict``)."""
    return np.repeat(np.repeat(e, 2, axis=1), 2, axis=2)


class MultigridPreconditioner:
    """z = B r, one V-cycle from a zero guess."""

    def __init__(self, p: Problem, nu: int = 1, omega: float = 0.8, coarsest_sweeps: int = 8,
                 max_levels: int = 32):
        self.nu, self.omega, self.coarsest_sweeps = nu, omega, coarsest_sweeps
        self.problems: List[Problem] = [p]
        while len(self.problems) < max_levels:
            q = self.problems[-1]
            if q.n_x % 2 or q.n_y % 2 or q.n_x * q.n_y == 1:
                break
            self.problems.append(coarse_problem(q))
        self.ops = [FluxOperator(q) for q in self.problems]
        self.lines = [LinePreconditioner(assemble_csr(q), q) for q in self.problems]

    @property
    def levels(self) -> int:
        return len(self.problems)

    def _smooth(self, l: int, r: np.ndarray, z: np.ndarray, sweeps: int) -> np.ndarray:
        a, m, w = self.ops[l], self.lines[l], self.omega
        for _ in range(sweeps):
            z = z + w * m(r - (a @ z).reshape(r.shape))
        return z

    def vcycle(self, l: int, r: np.ndarray) -> np.ndarray:
        q = self.problems[l]
        m = self.lines[l]
        if l == self.levels - 1:
            if q.n_x * q.n_y == 1:
                return m(r)                                  # the single column's block is all of A
            return self._smooth(l, r, np.zeros_like(r), self.coarsest_sweeps)
        z = self._smooth(l, r, np.zeros_like(r), self.nu)
        rc = restrict(r - (self.ops[l] @ z).reshape(r.shape))
        z = z + prolong(self.vcycle(l + 1, rc))
        return self._smooth(l, r, z, self.nu)

    def __call__(self, r: np.ndarray) -> np.ndarray:
        shape = np.shape(r)
        return self.vcycle(0, np.asarray(r, dtype=np.float64).reshape(self.problems[0].shape)).reshape(shape)
