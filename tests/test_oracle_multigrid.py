"""Pins of the oracle's multigrid preconditioner (the V-cycle with vertical
line smoothing and horizontal coarsening that the paper names as the next
solver, Section 8).

* Transfer operators: prolongation is the transpose of restriction, exactly.
* Coarse grids: the coarse operator is the same discretisation on a coarser
  grid, so its row sums (lambda^2 times the coarse cell volumes) are the
  sums of the fine row sums of its four children: the cells tile the same
  domain.  A dropped or doubled area, a wrong panel or latitude metric on the
  coarse grid fails this.
* The V-cycle is a symmetric positive definite operator (what CG needs):
  <B r1, r2> = <r1, B r2> and <B r, r> > 0.  A restriction not matched to
  its prolongation, or unequal smoothing before and after, breaks symmetry.
* A single column is solved exactly by its block (the coarsest level of a
  periodic box), and the V-cycle of a one-column problem is A^{-1}.
* MG-preconditioned CG reaches the dense direct solution, and its iteration
  count does not grow when the horizontal grid is refined (the property
  multigrid is for; a wrong coarse-grid scaling makes it grow).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import FluxOperator, assemble_csr, pcg_interleaved, pcg_textbook
from oracle.discretisation import cell_volumes
from oracle.linesolve import LinePreconditioner
from oracle.multigrid import MultigridPreconditioner, coarse_problem, prolong, restrict


def _problems():
    return [
        W.box_problem(8, 8, 6, 0.01, name="box"),
        W.box_problem(8, 4, 5, 0.02, alpha="sin", name="box-sin"),
        W.latlon_problem(12, 8, 5, thickness=0.01, name="latlon"),
        W.panel_problem(8, 8, 5, thickness=0.05, name="panel"),
    ]


def test_prolongation_is_transpose_of_restriction():
    rng = np.random.default_rng(1)
    r = rng.uniform(-1, 1, (5, 8, 6))
    e = rng.uniform(-1, 1, (5, 4, 3))
    assert abs(np.sum(restrict(r) * e) - np.sum(r * prolong(e))) <= 1e-13 * np.sum(np.abs(r)) * np.abs(e).max()


@pytest.mark.parametrize("p", _problems(), ids=lambda p: p.name)
def test_coarse_row_sums_are_sums_of_fine_row_sums(p):
    pc = coarse_problem(p)
    ones_f = np.ones(p.shape)
    ones_c = np.ones(pc.shape)
    af = (FluxOperator(p) @ ones_f).reshape(p.shape)
    ac = (FluxOperator(pc) @ ones_c).reshape(pc.shape)
    assert np.allclose(restrict(af), ac, rtol=1e-12, atol=0)
    assert np.allclose(restrict(cell_volumes(p)), cell_volumes(pc), rtol=1e-12, atol=0)


@pytest.mark.parametrize("p", _problems(), ids=lambda p: p.name)
def test_vcycle_is_symmetric_positive_definite(p):
    mg = MultigridPreconditioner(p)
    rng = np.random.default_rng(2)
    r1 = rng.uniform(-1, 1, p.shape)
    r2 = rng.uniform(-1, 1, p.shape)
    b1, b2 = mg(r1), mg(r2)
    lhs, rhs = np.sum(b1 * r2), np.sum(r1 * b2)
    scale = np.sqrt(np.sum(b1 * r1) * np.sum(b2 * r2))
    assert abs(lhs - rhs) <= 1e-10 * scale, (lhs, rhs)
    for r in (r1, r2, np.ones(p.shape)):
        assert np.sum(mg(r) * r) > 0


def test_single_column_vcycle_is_the_inverse():
    p = W.box_problem(1, 1, 7, 0.01)
    mg = MultigridPreconditioner(p)
    assert mg.levels == 1
    b = W.rhs_for(p, seed=3)
    x = mg(b)
    a = assemble_csr(p).toarray()
    xd = np.linalg.solve(a, b.ravel())
    # both solves are backward stable: forward difference <= c n cond(A) eps
    bound = 10 * p.n_z * np.linalg.cond(a) * np.finfo(float).eps
    assert np.linalg.norm(x.ravel() - xd) <= bound * np.linalg.norm(xd)


@pytest.mark.parametrize("p", _problems(), ids=lambda p: p.name)
def test_mg_pcg_reaches_the_direct_solution(p):
    b = W.rhs_for(p, seed=4)
    a = assemble_csr(p)
    xd = spla.spsolve(a.tocsc(), b.ravel())
    res = pcg_textbook(FluxOperator(p), MultigridPreconditioner(p), b, tol=1e-13, maxit=500)
    assert res.converged
    assert np.linalg.norm(res.x.ravel() - xd) <= 1e-9 * np.linalg.norm(xd)
    # Algorithm 1 with the V-cycle in place of M produces the same iterates
    ri = pcg_interleaved(FluxOperator(p), MultigridPreconditioner(p), b, eps=0.0, maxiter=6)
    rt = pcg_textbook(FluxOperator(p), MultigridPreconditioner(p), b, tol=0.0, maxit=6)
    assert np.linalg.norm(ri.x - rt.x) <= 1e-11 * np.linalg.norm(rt.x)


def test_iterations_do_not_grow_with_the_grid():
    its_mg, its_line = [], []
    for n in (16, 32, 64):
        p = W.box_problem(n, n, 16, 0.004)
        b = W.rhs_for(p, seed=0)
        a = FluxOperator(p)
        its_mg.append(pcg_textbook(a, MultigridPreconditioner(p), b, tol=1e-8, maxit=500).iterations)
        its_line.append(pcg_textbook(a, LinePreconditioner(assemble_csr(p), p), b, tol=1e-8, maxit=5000).iterations)
    assert its_mg[-1] <= its_mg[0] + 3, its_mg
    assert its_line[-1] >= 2 * its_line[0], its_line          # the plain line preconditioner does grow
    assert max(its_mg) < min(its_line), (its_mg, its_line)
