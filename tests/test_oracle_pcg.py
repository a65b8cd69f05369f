"""Pins of the oracle's line preconditioner and PCG loops.

* M = block-diag(A) (Section 4.2): the LAPACK tridiagonal solve of every
  column equals a dense LU solve of the block cut out of the assembled A;
  the column-by-column solve used for sampled checks of large grids equals
  it too.
* With a single column (no horizontal coupling survives) M = A, so one
  preconditioner application is the exact solution and PCG stops after one
  iteration.
* PCG converges to the dense direct solution; the A-norm of the error never
  increases (a theorem of CG in exact arithmetic, observable here to rounding).
* Algorithm 1 produces the textbook iterates (Section 4.3: the loop is only
  a reordering of the same operations), and so does the single-reduction
  form (Chronopoulos-Gear, cited in Section 4.3), whose alpha comes from
  gamma and delta by a recurrence instead of <p, A p>: a wrong recurrence
  (a dropped beta term, the old gamma in place of the new) changes the
  iterates from the second step on.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from oracle import (FluxOperator, LinePreconditioner, assemble_csr, column_blocks, pcg_interleaved,
                    pcg_single_reduction, pcg_textbook, rounding_floor, solve_columns, apply_columns)


def _problems():
    return [
        W.box_problem(5, 4, 6, 0.01, name="box"),
        W.box_problem(4, 6, 7, 0.02, alpha="sin", name="box-sin"),
        W.latlon_problem(8, 5, 6, thickness=0.01, name="latlon"),
    ]


@pytest.mark.parametrize("p", _problems(), ids=lambda p: p.name)
def test_line_solve_equals_dense_block_lu(p):
    a = assemble_csr(p)
    m = LinePreconditioner(a, p)
    rng = np.random.default_rng(7)
    r = rng.uniform(-1, 1, p.shape)
    z = m(r)
    dense = a.toarray()
    plane = p.n_x * p.n_y
    for col in range(plane):
        idx = col + plane * np.arange(p.n_z)
        block = dense[np.ix_(idx, idx)]
        lu = sla.lu_factor(block)
        zc = sla.lu_solve(lu, r.ravel()[idx])
        # both solves are backward stable: forward difference <= c n cond(block) eps
        bound = 10 * p.n_z * np.linalg.cond(block) * np.finfo(float).eps
        err = np.linalg.norm(z.ravel()[idx] - zc) / np.linalg.norm(zc)
        assert err <= max(bound, 1e-14), (col, err, bound)


@pytest.mark.parametrize("p", _problems() + [W.panel_problem(6, 5, 7, thickness=0.05, name="panel"),
                                             W.box_problem(1, 3, 4, 0.01, name="box-1x3")],
                         ids=lambda p: p.name)
def test_column_solve_equals_dense_block_lu(p):
    a = assemble_csr(p)
    dense = a.toarray()
    plane = p.n_x * p.n_y
    rng = np.random.default_rng(11)
    r = rng.uniform(-1, 1, p.shape)
    cols = np.array([[c // p.n_x for c in range(plane)], [c % p.n_x for c in range(plane)]])
    r_cols = np.stack([r[:, j, i] for j, i in cols.T])
    z = solve_columns(p, r_cols, cols)
    for c, (j, i) in enumerate(cols.T):
        idx = (j * p.n_x + i) + plane * np.arange(p.n_z)
        block = dense[np.ix_(idx, idx)]
        zc = sla.lu_solve(sla.lu_factor(block), r_cols[c])
        bound = 10 * p.n_z * np.linalg.cond(block) * np.finfo(float).eps
        err = np.linalg.norm(z[c] - zc) / np.linalg.norm(zc)
        assert err <= max(bound, 1e-14), (c, err, bound)
        # the flux-form product of the column block is the block times z, to
        # the rounding of the assembled product (the flux form is the exact one)
        mz, scale = apply_columns(p, z[c:c + 1], cols[:, c:c + 1])
        tol = 64 * np.finfo(float).eps * (np.abs(block) @ np.abs(z[c]) + scale[0])
        assert (np.abs(mz[0] - block @ z[c]) <= tol).all()


@pytest.mark.parametrize("p", _problems(), ids=lambda p: p.name)
def test_blocks_are_exact_entries_of_a(p):
    a = assemble_csr(p).toarray()
    lower, main, upper = column_blocks(assemble_csr(p), p)
    plane = p.n_x * p.n_y
    for col in (0, plane // 2, plane - 1):
        idx = col + plane * np.arange(p.n_z)
        blk = a[np.ix_(idx, idx)]
        assert (np.diag(blk) == main[col]).all()
        assert (np.diag(blk, 1) == upper[col, :-1]).all()
        assert (np.diag(blk, -1) == lower[col, 1:]).all()


def test_single_column_preconditioner_is_exact():
    p = W.box_problem(1, 1, 9, 0.5, lambda2=1.0, beta_scale=0.5)   # 1x1 periodic: horizontal couplings cancel
    a = assemble_csr(p)
    m = LinePreconditioner(a, p)
    b = W.rhs_for(p, seed=4)
    ad = a.toarray()
    xd = np.linalg.solve(ad, b.ravel())
    bound = 10 * p.n_z * np.linalg.cond(ad) * np.finfo(float).eps
    assert np.linalg.norm(m(b).ravel() - xd) / np.linalg.norm(xd) <= bound
    res = pcg_textbook(FluxOperator(p), m, b, tol=1e-12, maxit=5)
    assert res.iterations == 1 and res.converged


@pytest.mark.parametrize("p", [W.box_problem(8, 8, 8, 0.5, lambda2=1.0, beta_scale=0.5),
                               W.box_problem(6, 7, 8, 0.3, lambda2=2.0, beta_scale=0.5, alpha="sin"),
                               W.latlon_problem(8, 6, 8, thickness=0.2, lambda2=1.0, beta_scale=0.5)],
                         ids=["box", "box-sin", "latlon"])
def test_pcg_equals_dense_solve(p):
    a = assemble_csr(p)
    m = LinePreconditioner(a, p)
    b = W.rhs_for(p, seed=11)
    xd = np.linalg.solve(a.toarray(), b.ravel())
    op = FluxOperator(p)
    for fn in (pcg_textbook, pcg_interleaved, pcg_single_reduction):
        kw = dict(tol=1e-14) if fn is pcg_textbook else dict(eps=1e-14)
        res = fn(op, m, b, maxit=500, **kw) if fn is pcg_textbook else fn(op, m, b, maxiter=500, **kw)
        err = np.linalg.norm(res.x.ravel() - xd) / np.linalg.norm(xd)
        assert err < 1e-12, (fn.__name__, err)


def test_error_a_norm_decreases():
    p = W.box_problem(8, 8, 6, 0.05, lambda2=0.5, beta_scale=0.5)
    a = assemble_csr(p)
    m = LinePreconditioner(a, p)
    b = W.rhs_for(p, seed=2)
    ad = a.toarray()
    xd = np.linalg.solve(ad, b.ravel())
    prev = np.inf
    floor = None
    op = FluxOperator(p)
    for k in range(0, 25):
        x = pcg_textbook(op, m, b, tol=0.0, maxit=k).x.ravel()
        e = x - xd
        en = float(np.sqrt(e @ (ad @ e)))
        floor = floor or 1e-9 * en          # below this the dense reference's own rounding shows
        assert en <= prev * (1 + 1e-10) or en < floor, (k, en, prev)
        prev = en
    assert prev < floor


@pytest.mark.parametrize("p", _problems() + [W.small_box()], ids=lambda p: p.name or "small")
def test_interleaved_equals_textbook(p):
    a = FluxOperator(p)
    m = LinePreconditioner(assemble_csr(p), p)
    b = W.rhs_for(p, seed=0)
    for k in (0, 1, 2, 5, 13):
        xt = pcg_textbook(a, m, b, tol=0.0, maxit=k)
        xi = pcg_interleaved(a, m, b, eps=0.0, maxiter=k)
        assert xt.iterations == xi.iterations == k
        scale = max(np.linalg.norm(xt.x), 1e-300)
        assert np.linalg.norm(xt.x - xi.x) / scale < 1e-12
        r0 = xt.residual_history[0]
        np.testing.assert_allclose(xi.residual_history, xt.residual_history, rtol=1e-10, atol=1e-12 * r0)
    rt = pcg_textbook(a, m, b, tol=1e-8, maxit=5000)
    ri = pcg_interleaved(a, m, b, eps=1e-8, maxiter=5000)
    assert rt.converged and ri.converged
    assert abs(rt.iterations - ri.iterations) <= 1
    assert ri.final_true_relres < 2e-8


@pytest.mark.parametrize("p", _problems() + [W.small_box()], ids=lambda p: p.name or "small")
def test_single_reduction_equals_textbook(p):
    a = FluxOperator(p)
    m = LinePreconditioner(assemble_csr(p), p)
    b = W.rhs_for(p, seed=0)
    for k in (0, 1, 2, 5, 13):
        xt = pcg_textbook(a, m, b, tol=0.0, maxit=k)
        xs = pcg_single_reduction(a, m, b, eps=0.0, maxiter=k)
        assert xt.iterations == xs.iterations == k
        scale = max(np.linalg.norm(xt.x), 1e-300)
        assert np.linalg.norm(xt.x - xs.x) / scale < 1e-11, k
        r0 = xt.residual_history[0]
        np.testing.assert_allclose(xs.residual_history, xt.residual_history, rtol=1e-9, atol=1e-12 * r0)
    rt = pcg_textbook(a, m, b, tol=1e-8, maxit=5000)
    rs = pcg_single_reduction(a, m, b, eps=1e-8, maxiter=5000)
    assert rt.converged and rs.converged
    assert abs(rt.iterations - rs.iterations) <= 1
    assert rs.final_true_relres < 2e-8


def test_zero_rhs_returns_zero():
    p = W.small_box(scale=4)
    a = FluxOperator(p)
    m = LinePreconditioner(assemble_csr(p), p)
    b = np.zeros(p.shape)
    for res in (pcg_textbook(a, m, b), pcg_interleaved(a, m, b)):
        assert res.iterations == 0 and not res.x.any()


# ---------------------------------------------------------------------------
# Accuracy against a compensated-arithmetic reference.  Error-free
# transformations (Dekker's exact product via Veltkamp splitting, Knuth's
# TwoSum) evaluate the flux-form residual to about twice the working
# precision; refining with it gives the solution to FP64 rounding, so the
# oracle's own solution error can be measured rather than assumed.
# ---------------------------------------------------------------------------

def _two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def _split(a):
    c = 134217729.0 * a
    h = c - (c - a)
    return h, a - h


def _two_prod(a, b):
    p = a * b
    ah, al = _split(a)
    bh, bl = _split(b)
    return p, al * bl - (((p - ah * bh) - al * bh) - ah * bl)


def _accurate_residual(op, b, x):
    """b - A x with A in flux form, evaluated with compensated arithmetic."""
    xf = x.ravel()
    rows, cols, c = op._rows, op.C.indices, op.C.data
    s, e = _two_prod(op.mass, xf)
    s, e = -s, -e
    s, e2 = _two_sum(b.ravel(), s)
    e = e + e2
    d, de = _two_sum(xf[rows], -xf[cols])
    pp, pe = _two_prod(c, d)
    pe = pe + c * de
    # per-row compensated sums of the fluxes (rows are sorted in CSR order)
    order_pos = np.arange(rows.size) - op.C.indptr[rows]
    for t in range(order_pos.max() + 1 if rows.size else 0):
        sel = order_pos == t
        r_ = rows[sel]
        s_new, err = _two_sum(s[r_], -pp[sel])
        s[r_] = s_new
        e[r_] += err - pe[sel]
    return s + e


@pytest.mark.parametrize("p", [W.small_box(), W.medium_box(scale=8, n_z=64)], ids=["box32x32x16", "box32x32x64"])
def test_oracle_solution_matches_refined_reference(p):
    op = FluxOperator(p)
    m = LinePreconditioner(assemble_csr(p), p)
    b = W.rhs_for(p, seed=0, smooth=True)
    x = np.zeros(p.n_cells)
    for _ in range(4):
        r = _accurate_residual(op, b, x)
        x = x + pcg_textbook(op, m, r.reshape(p.shape), tol=1e-13, maxit=5000).x.ravel()
    res = pcg_interleaved(op, m, b, eps=1e-10, maxiter=5000)
    err = np.linalg.norm(res.x.ravel() - x) / np.linalg.norm(x)
    assert res.converged and err < 1e-11, err


@pytest.mark.parametrize("p", [W.small_box(), W.medium_box(scale=8, n_z=64)], ids=["box32x32x16", "box32x32x64"])
def test_rounding_floor_predicts_residual_of_rounded_solution(p):
    """The floor model equals the measured true residual of the (refined)
    solution rounded to FP64, evaluated with compensated arithmetic."""
    op = FluxOperator(p)
    a = assemble_csr(p)
    m = LinePreconditioner(a, p)
    b = W.rhs_for(p, seed=0, smooth=True)
    x = np.zeros(p.n_cells)
    for _ in range(4):
        r = _accurate_residual(op, b, x)
        x = x + pcg_textbook(op, m, r.reshape(p.shape), tol=1e-13, maxit=5000).x.ravel()
    measured = np.linalg.norm(_accurate_residual(op, b, x)) / np.linalg.norm(b)
    model = rounding_floor(a, x, b)
    assert 0.8 < measured / model < 1.25, (measured, model)
