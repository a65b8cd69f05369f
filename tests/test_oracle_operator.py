"""Pins of the oracle's operator against facts fixed by the paper and the mathematics.

* Symmetry and definiteness: the paper's operator is symmetric positive
  definite (Section 3, Eq. (ModelEquation); the column blocks are "symmetric
  tridiagonal", Eq. (TridiagonalMatrix)).
* Row sums: every difference term vanishes on a constant vector, so
  A 1 = lambda^2 x (cell volume), and A 1 = 0 when lambda^2 = 0.
* Discrete Fourier eigenvalues of the periodic horizontal operator (a closed
  form independent of the assembly code).
* Total area of the latitude band and total shell volume (closed forms).
* Second-order convergence to a manufactured solution of the continuous PDE
  (the finite-volume scheme of Section 3.1), which fails for a dropped term,
  a wrong sign, a wrong metric factor or a misplaced face coefficient.
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import FluxOperator, apply_rows, assemble_csr, cell_volumes, operator_terms


def _problems():
    return [
        W.box_problem(5, 4, 6, 0.01, name="box"),
        W.box_problem(4, 6, 5, 0.02, alpha="sin", name="box-sin"),
        W.box_problem(3, 3, 4, 0.01, lambda2=0.5, name="box-3"),
        W.latlon_problem(8, 5, 4, thickness=0.01, name="latlon"),
        W.box_problem(1, 2, 3, 0.01, name="box-1x2"),
        W.panel_problem(6, 6, 5, thickness=0.05, name="panel"),
    ]


@pytest.mark.parametrize("p", _problems(), ids=lambda p: p.name)
def test_symmetric_bitwise(p):
    a = assemble_csr(p)
    diff = a - a.T
    diff.eliminate_zeros()
    assert diff.nnz == 0


@pytest.mark.parametrize("p", _problems(), ids=lambda p: p.name)
def test_positive_definite(p):
    a = assemble_csr(p).toarray()
    np.linalg.cholesky(a)            # raises if not SPD
    assert np.linalg.eigvalsh(a).min() > 0


@pytest.mark.parametrize("p", _problems(), ids=lambda p: p.name)
def test_row_sums_are_mass_terms(p):
    # flux form: every flux vanishes on a constant vector, so A 1 is the mass
    # term exactly; the assembled matrix agrees to the rounding of its diagonal.
    vol = cell_volumes(p).ravel()
    op = FluxOperator(p)
    rs = op @ np.ones(p.n_cells)
    np.testing.assert_allclose(rs, p.lambda2 * vol, rtol=1e-13, atol=0)
    assert (rs == op.mass).all()
    a = assemble_csr(p)
    ra = a @ np.ones(p.n_cells)
    assert np.abs(ra - rs).max() <= 8 * np.finfo(float).eps * np.abs(a.diagonal()).max()


def test_row_sums_vanish_without_mass():
    for p in (W.box_problem(6, 5, 7, 0.01, lambda2=0.0, alpha="sin"),
              W.latlon_problem(8, 6, 5, thickness=0.01, lambda2=0.0)):
        assert not (FluxOperator(p) @ np.ones(p.n_cells)).any()
        a = assemble_csr(p)
        rs = a @ np.ones(p.n_cells)
        assert np.abs(rs).max() <= 1e-14 * np.abs(a.diagonal()).max()


@pytest.mark.parametrize("p", _problems(), ids=lambda p: p.name)
def test_flux_form_is_the_assembled_operator(p):
    a = assemble_csr(p)
    op = FluxOperator(p)
    rng = np.random.default_rng(5)
    for _ in range(3):
        x = rng.standard_normal(p.n_cells)
        ya, yf = a @ x, op @ x
        bound = 16 * np.finfo(float).eps * (abs(a) @ abs(x))      # componentwise SpMV error bound
        assert (np.abs(yf - ya) <= bound).all()
    if min(p.n_x, p.n_y) > 1:      # on a one-cell periodic axis a cell couples to itself
        np.testing.assert_allclose(op.diagonal(), a.diagonal(), rtol=8 * np.finfo(float).eps)
    diff = op.C - op.C.T
    diff.eliminate_zeros()
    assert diff.nnz == 0 and (op.C.data > 0).all()


def test_stencil_has_seven_points_and_neumann_ends():
    p = W.box_problem(6, 5, 4, 0.01)
    a = assemble_csr(p)
    nnz_per_row = np.diff(a.indptr).reshape(p.shape)
    assert (nnz_per_row[1:-1] == 7).all()          # interior levels: 7-point stencil
    assert (nnz_per_row[0] == 6).all() and (nnz_per_row[-1] == 6).all()
    p = W.latlon_problem(8, 5, 4, thickness=0.01)
    nnz = np.diff(assemble_csr(p).indptr).reshape(p.shape)
    assert (nnz[1:-1, 1:-1] == 7).all()
    assert (nnz[1:-1, 0] == 6).all() and (nnz[1:-1, -1] == 6).all()   # latitude edges: Neumann


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_horizontal_fourier_eigenvalues(mode):
    # u_ijk = cos(2 pi m (i + 1/2)/n_x) for every j, k: vertical and y terms vanish,
    # and the periodic second difference has eigenvalue 2 - 2 cos(2 pi m / n_x).
    n_x, n_y, n_z = 12, 5, 4
    p = W.box_problem(n_x, n_y, n_z, 0.01, lambda2=0.3)
    a = assemble_csr(p)
    hx, hy = 1.0 / n_x, 1.0 / n_y
    dz = np.diff(p.z_iface)
    i = np.arange(n_x)
    u = np.broadcast_to(np.cos(2 * np.pi * mode * (i + 0.5) / n_x), p.shape)
    lam = p.lambda2 * hx * hy + (hy / hx) * (2 - 2 * np.cos(2 * np.pi * mode / n_x))
    expect = lam * dz[:, None, None] * u
    np.testing.assert_allclose((a @ u.ravel()).reshape(p.shape), expect, rtol=1e-11, atol=1e-17)
    # the same in y
    j = np.arange(n_y)
    u = np.broadcast_to(np.cos(2 * np.pi * mode * (j[:, None] + 0.5) / n_y), p.shape)
    lam = p.lambda2 * hx * hy + (hx / hy) * (2 - 2 * np.cos(2 * np.pi * mode / n_y))
    np.testing.assert_allclose((a @ u.ravel()).reshape(p.shape), lam * dz[:, None, None] * u,
                               rtol=1e-11, atol=1e-17)


def test_latlon_band_area_and_volume():
    p = W.latlon_problem(36, 20, 6, thickness=0.05, lat_deg=70.0)
    t = operator_terms(p)
    band = 2 * np.pi * (math.sin(p.lat1) - math.sin(p.lat0))
    assert abs(t.area.sum() - band) < 1e-13 * band
    r0, r1 = p.z_iface[0], p.z_iface[-1]
    shell = band * (r1 ** 3 - r0 ** 3) / 3
    assert abs(cell_volumes(p).sum() - shell) < 1e-12 * shell


@pytest.mark.parametrize("p", _problems(), ids=lambda p: p.name)
def test_apply_rows_matches_matrix(p):
    rng = np.random.default_rng(3)
    x = rng.standard_normal(p.shape)
    a = assemble_csr(p)
    y = (a @ x.ravel()).reshape(p.shape)
    cells = np.stack(np.meshgrid(np.arange(p.n_z), np.arange(p.n_y), np.arange(p.n_x), indexing="ij")).reshape(3, -1)
    yr = apply_rows(p, x, cells)
    np.testing.assert_allclose(yr, y.ravel(), rtol=1e-13, atol=1e-13 * np.abs(y).max())


# ---------------------------------------------------------------------------
# Manufactured solutions: second-order convergence of the discrete solution to
# the continuous one under uniform refinement of every spacing.
# ---------------------------------------------------------------------------

def _mms_box(n, depth=1.0, bscale=0.5, lam2=1.0):
    sym = pytest.importorskip("sympy")
    x, y, z = sym.symbols("x y z", real=True)
    u = sym.cos(2 * sym.pi * x) * sym.cos(2 * sym.pi * y) * sym.cos(sym.pi * z / depth)
    alpha = 1 + sym.Rational(1, 2) * sym.sin(2 * sym.pi * x) * sym.sin(2 * sym.pi * y)
    beta = sym.exp(-z / bscale)
    f = (-sym.diff(alpha * sym.diff(u, x), x) - sym.diff(alpha * sym.diff(u, y), y)
         - sym.diff(beta * sym.diff(u, z), z) + lam2 * u)
    fn = sym.lambdify((x, y, z), f, "numpy")
    un = sym.lambdify((x, y, z), u, "numpy")
    zi = W.smooth_graded_interfaces(n, depth)
    ae, an = W.sinusoidal_alpha(n, n)
    p = W.Problem(kind=W.GEOM_BOX, n_x=n, n_y=n, n_z=n, z_iface=zi,
                  beta_iface=W.exp_profile(zi, bscale), lambda2=lam2, alpha_e=ae, alpha_n=an)
    xc = (np.arange(n) + 0.5) / n
    zc = 0.5 * (zi[1:] + zi[:-1])
    Z, Y, X = np.meshgrid(zc, xc, xc, indexing="ij")
    b = fn(X, Y, Z) * cell_volumes(p)
    ue = un(X, Y, Z)
    uh = spla.spsolve(assemble_csr(p).tocsc(), b.ravel()).reshape(p.shape)
    return np.sqrt(np.mean((uh - ue) ** 2))


def _mms_latlon(n, H=0.5, bscale=0.5, lam2=1.0, lat_deg=60.0):
    sym = pytest.importorskip("sympy")
    lon, lat, r = sym.symbols("lon lat r", real=True)
    L0 = -sym.pi * lat_deg / 180
    L1 = sym.pi * lat_deg / 180
    u = sym.cos(lon) * sym.cos(sym.pi * (lat - L0) / (L1 - L0)) * sym.cos(sym.pi * (r - 1) / H)
    beta = sym.exp(-(r - 1) / bscale)
    lap_sphere = (sym.diff(sym.cos(lat) * sym.diff(u, lat), lat) / sym.cos(lat)
                  + sym.diff(u, lon, 2) / sym.cos(lat) ** 2)
    f = -lap_sphere / r ** 2 - sym.diff(r ** 2 * beta * sym.diff(u, r), r) / r ** 2 + lam2 * u
    fn = sym.lambdify((lon, lat, r), f, "numpy")
    un = sym.lambdify((lon, lat, r), u, "numpy")
    ri = 1.0 + W.smooth_graded_interfaces(n, H)
    p = W.Problem(kind=W.GEOM_LATLON, n_x=2 * n, n_y=n, n_z=n, z_iface=ri,
                  beta_iface=W.exp_profile(ri, bscale, origin=1.0), lambda2=lam2,
                  lat0=-math.radians(lat_deg), lat1=math.radians(lat_deg))
    lonc = (np.arange(2 * n) + 0.5) * 2 * np.pi / (2 * n)
    dlat = (p.lat1 - p.lat0) / n
    latc = p.lat0 + (np.arange(n) + 0.5) * dlat
    rc = 0.5 * (ri[1:] + ri[:-1])
    R, LAT, LON = np.meshgrid(rc, latc, lonc, indexing="ij")
    b = fn(LON, LAT, R) * cell_volumes(p)
    ue = un(LON, LAT, R)
    uh = spla.spsolve(assemble_csr(p).tocsc(), b.ravel()).reshape(p.shape)
    return np.sqrt(np.mean((uh - ue) ** 2))


def test_manufactured_solution_box_second_order():
    e = [_mms_box(n) for n in (8, 16, 32)]
    ratios = [e[0] / e[1], e[1] / e[2]]
    assert all(3.3 < q < 4.8 for q in ratios), (e, ratios)


def test_manufactured_solution_latlon_second_order():
    e = [_mms_latlon(n) for n in (8, 16, 32)]
    ratios = [e[0] / e[1], e[1] / e[2]]
    assert all(3.3 < q < 4.8 for q in ratios), (e, ratios)


# ---------------------------------------------------------------------------
# Cubed-sphere panel (the paper's geometry, Section 3.2)
# ---------------------------------------------------------------------------

def test_panel_covers_a_sixth_of_the_sphere():
    for n in (4, 17, 64):
        t = operator_terms(W.panel_problem(n, n, 3))
        assert abs(t.area.sum() - 4 * np.pi / 6) < 1e-12


def test_panel_operator_commutes_with_the_panel_symmetries():
    # the gnomonic panel is invariant under x <-> y and under x -> -x, y -> -y;
    # the operator must commute with the induced permutations of the columns
    p = W.panel_problem(7, 7, 4, thickness=0.05)
    op = FluxOperator(p)
    x = np.random.default_rng(9).standard_normal(p.shape)
    ax = (op @ x).reshape(p.shape)
    for perm in (lambda v: np.swapaxes(v, 1, 2), lambda v: v[:, :, ::-1], lambda v: v[:, ::-1, :]):
        lhs = (op @ np.ascontiguousarray(perm(x))).reshape(p.shape)
        np.testing.assert_allclose(lhs, perm(ax), rtol=1e-12, atol=1e-12 * np.abs(ax).max())


def test_panel_edges_are_neumann():
    p = W.panel_problem(5, 4, 3)
    t = operator_terms(p)
    assert (t.mu_e[:, -1] == 0).all() and (t.mu_n[-1, :] == 0).all()
    assert (t.mu_e[:, :-1] > 0).all() and (t.mu_n[:-1, :] > 0).all()


# The face weights of the panel, pinned independently of the oracle's
# formulas.  Section 3.1 defines the horizontal coupling of two cells as the
# length of their common edge divided by the distance between their
# midpoints.  The checks below recompute both from normalised 3-D points
# (great-circle arcs as atan2(|a x b|, a.b)), compare each cell's area with a
# quadrature of the gnomonic area element, and compare the two-point flux with
# the exact flux of a smooth function through faces where the grid is
# orthogonal (the panel's two central lines), where it must converge at second
# order.  On skewed faces a two-point flux is not consistent (its error stays
# O(1) near the panel corners), so the panel has no manufactured-solution
# convergence test like the box and the band.

def _panel_unit(x, y):
    v = np.stack(np.broadcast_arrays(np.ones_like(x), x, y), axis=-1)
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _great_arc(a, b):
    return np.arctan2(np.linalg.norm(np.cross(a, b), axis=-1), np.sum(a * b, axis=-1))


@pytest.mark.parametrize("n_x,n_y", [(6, 6), (17, 9), (64, 64)])
def test_panel_face_weights_are_edge_over_centre_distance(n_x, n_y):
    p = W.panel_problem(n_x, n_y, 2)
    t = operator_terms(p)
    xf = np.linspace(-1.0, 1.0, n_x + 1)
    yf = np.linspace(-1.0, 1.0, n_y + 1)
    xc = 0.5 * (xf[1:] + xf[:-1])
    yc = 0.5 * (yf[1:] + yf[:-1])
    alpha = np.asarray(p.alpha_e)
    mu_e = np.zeros((n_y, n_x))
    mu_n = np.zeros((n_y, n_x))
    for j in range(n_y):
        for i in range(n_x):
            centre = _panel_unit(xc[i], yc[j])
            if i + 1 < n_x:     # east edge: x = xf[i+1], y from yf[j] to yf[j+1]
                edge = _great_arc(_panel_unit(xf[i + 1], yf[j]), _panel_unit(xf[i + 1], yf[j + 1]))
                mu_e[j, i] = edge / _great_arc(centre, _panel_unit(xc[i + 1], yc[j]))
            if j + 1 < n_y:     # north edge: y = yf[j+1], x from xf[i] to xf[i+1]
                edge = _great_arc(_panel_unit(xf[i], yf[j + 1]), _panel_unit(xf[i + 1], yf[j + 1]))
                mu_n[j, i] = edge / _great_arc(centre, _panel_unit(xc[i], yc[j + 1]))
    np.testing.assert_allclose(t.mu_e, alpha * mu_e, rtol=1e-12, atol=0)
    np.testing.assert_allclose(t.mu_n, np.asarray(p.alpha_n) * mu_n, rtol=1e-12, atol=0)


def test_panel_cell_areas_match_quadrature_of_the_area_element():
    # the gnomonic map (x, y) -> (1, x, y)/|(1, x, y)| has area element
    # (1 + x^2 + y^2)^(-3/2) dx dy; 8-point Gauss-Legendre per cell and axis
    n_x, n_y = 12, 7
    t = operator_terms(W.panel_problem(n_x, n_y, 2))
    g, wg = np.polynomial.legendre.leggauss(8)
    xf = np.linspace(-1.0, 1.0, n_x + 1)
    yf = np.linspace(-1.0, 1.0, n_y + 1)
    for j in range(n_y):
        for i in range(n_x):
            hx, hy = xf[i + 1] - xf[i], yf[j + 1] - yf[j]
            x = xf[i] + 0.5 * hx * (g + 1.0)
            y = yf[j] + 0.5 * hy * (g + 1.0)
            X, Y = np.meshgrid(x, y)
            q = 0.25 * hx * hy * np.einsum("a,b,ab->", wg, wg, (1.0 + X * X + Y * Y) ** -1.5)
            assert abs(t.area[j, i] - q) <= 1e-13 * q, (j, i, t.area[j, i], q)


def _smooth_on_sphere(v):
    """A smooth function of the 3-D point and its 3-D gradient."""
    X, Y, Z = v[..., 0], v[..., 1], v[..., 2]
    u = np.sin(2 * Y + 0.5) * np.cos(1.5 * Z) + Y * Z + 0.3 * X * X
    grad = np.stack([0.6 * X,
                     2 * np.cos(2 * Y + 0.5) * np.cos(1.5 * Z) + Z,
                     -1.5 * np.sin(2 * Y + 0.5) * np.sin(1.5 * Z) + Y], axis=-1)
    return u, grad


def _exact_face_flux(a, b, towards):
    """Integral over the great-circle edge from a to b of grad u . N, N the
    unit normal of the edge within the sphere, oriented towards ``towards``.
    N = a x b / |a x b| is the same at every point of the edge and tangent to
    the sphere there, so the 3-D gradient of any extension gives grad u . N."""
    nrm = np.cross(a, b)
    nrm /= np.linalg.norm(nrm)
    if nrm @ towards < 0:
        nrm = -nrm
    theta = _great_arc(a, b)
    tang = b - (a @ b) * a
    tang /= np.linalg.norm(tang)
    g, wg = np.polynomial.legendre.leggauss(12)
    s = 0.5 * theta * (g + 1.0)
    pts = np.cos(s)[:, None] * a + np.sin(s)[:, None] * tang
    _, grad = _smooth_on_sphere(pts)
    return 0.5 * theta * float(wg @ (grad @ nrm))


def _central_line_flux_error(n):
    p = W.panel_problem(n, n, 2)
    t = operator_terms(p)
    mu_e = t.mu_e / np.asarray(p.alpha_e)
    mu_n = t.mu_n / np.asarray(p.alpha_n)
    f = np.linspace(-1.0, 1.0, n + 1)
    c = 0.5 * (f[1:] + f[:-1])
    m = n // 2 - 1                       # faces on x = 0 (east of column m) and on y = 0 (north of row m)
    errs, scale = [], []
    for k in range(n):
        uP, _ = _smooth_on_sphere(_panel_unit(c[m], c[k]))
        uE, _ = _smooth_on_sphere(_panel_unit(c[m + 1], c[k]))
        exact = _exact_face_flux(_panel_unit(0.0, f[k]), _panel_unit(0.0, f[k + 1]), np.array([0.0, 1.0, 0.0]))
        errs.append(mu_e[k, m] * (uE - uP) - exact)
        scale.append(abs(exact))
        uP, _ = _smooth_on_sphere(_panel_unit(c[k], c[m]))
        uN, _ = _smooth_on_sphere(_panel_unit(c[k], c[m + 1]))
        exact = _exact_face_flux(_panel_unit(f[k], 0.0), _panel_unit(f[k + 1], 0.0), np.array([0.0, 0.0, 1.0]))
        errs.append(mu_n[m, k] * (uN - uP) - exact)
        scale.append(abs(exact))
    return np.abs(errs).max() / max(scale)


def test_panel_two_point_flux_is_second_order_on_the_orthogonal_central_lines():
    e = [_central_line_flux_error(n) for n in (8, 16, 32, 64)]
    ratios = [e[i] / e[i + 1] for i in range(3)]
    assert all(3.5 < q < 4.5 for q in ratios), (e, ratios)
    assert e[-1] < 1e-3
