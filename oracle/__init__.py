"""CPU oracle for the matrix-free line-preconditioned CG solver.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 restatement
of what the solver computes, written from the paper (Mueller, Guo, Scheichl,
Shi: "Matrix-free GPU implementation of a preconditioned conjugate gradient
solver for anisotropic elliptic PDEs").  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline and
``--impl reference`` legs) may import it.  The product path never calls it
and shares no code with it; the two meet only in the seeded inputs of the
``workloads`` package.

Contents
--------
discretisation  explicit CSR matrix of the finite-volume operator
                (Section 3.1, Eqs. (ModelEqnCubedSphere), (DiagonalMatrix),
                (TridiagonalMatrix); Section 4.2 stencil), assembled from the
                problem data with scipy.sparse, and the same operator applied
                in flux form (FluxOperator), which the solvers use.
linesolve       vertical-line preconditioner M = block-diag(A) (Section 4.2),
                solved with LAPACK's tridiagonal LU (GTTRF/GTTRS), the routines
                of the paper's CPU code (Section 6.2); on the whole grid, or on
                selected columns for sampled checks of very large grids.
pcg             textbook left-preconditioned CG (Section 4.1) and the
                interleaved loop of Algorithm 1 (Section 4.3).

Every function here is pinned by ``tests/test_oracle_*.py`` against facts the
paper and the mathematics fix (symmetry, definiteness, closed-form row sums,
dense direct solves, manufactured-solution convergence).
"""
from .discretisation import (OperatorTerms, operator_terms, assemble_csr, apply_rows,
                             column_blocks, cell_volumes, FluxOperator)
from .linesolve import LinePreconditioner, apply_columns, solve_columns
from .pcg import pcg_textbook, pcg_interleaved, pcg_single_reduction, PCGResult, rounding_floor

__all__ = [
    "OperatorTerms", "operator_terms", "assemble_csr", "apply_rows", "column_blocks", "cell_volumes",
    "FluxOperator",
    "LinePreconditioner", "solve_columns", "apply_columns", "pcg_textbook", "pcg_interleaved", "pcg_single_reduction", "PCGResult", "rounding_floor",
]
