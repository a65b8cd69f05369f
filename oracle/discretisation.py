"""Finite-volume operator of the model equation as an explicit CSR matrix.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper writes the discrete operator column by column (Section 3.1,
Eq. (ModelEqnCubedSphere)):

    (A u)^(T) = A_T u^(T) + sum_{T' in N(T)} A_{T,T'} u^(T'),

with diagonal horizontal couplings A_{T,T'} = alpha_{T,T'} diag(d)
(Eq. (DiagonalMatrix)) and a symmetric tridiagonal column block
A_T = |T| diag(a) - alpha_T diag(d) + |T| tridiag(-(b+c), b, c)
(Eq. (TridiagonalMatrix)).  The paper's alpha_{T,T'}, b and c are negative
for this SPD operator (it absorbs the -omega^2 of Eq. (ModelEquation)); here
the positive face weights mu_f = -alpha_{T,T'} and vertical weights
w_{k+1/2} = -b_k = -c_{k+1} are used instead, so that every row reads

    (A u)_{ijk} = |T_ij| [ a_k u_ijk + w_{k+1/2} (u_ijk - u_ij,k+1)
                                     + w_{k-1/2} (u_ijk - u_ij,k-1) ]
                + d_k sum_f mu_f (u_ijk - u_f,k)

which is the cell integral of -div_h(alpha grad_h u) - (1/S) d_z(S beta d_z u)
+ lambda^2 u over cell (i, j, k) with two-point fluxes (the paper's
Section 4.2 stencil is this row after dividing by d_k).  Vertical fluxes are
dropped at the bottom and top (Neumann); horizontal faces wrap periodically,
except the latitude edges of the latlon band, which are Neumann.

Geometry
--------
box     periodic lx x ly rectangle, hx = lx/n_x, hy = ly/n_y:
        |T| = hx hy, d_k = dz_k, a_k = lambda^2 dz_k,
        w_{k+1/2} = beta(z_{k+1}) / (zc_{k+1} - zc_k),
        mu_E = alpha_e hy/hx, mu_N = alpha_n hx/hy.
latlon  longitude periodic over 2 pi (dlon = 2 pi/n_x), latitude
        [lat0, lat1] (dlat = (lat1-lat0)/n_y), radius interfaces r_k:
        |T_j| = dlon (sin lat_{j+1/2} - sin lat_{j-1/2}) = 2 dlon cos lat_j sin(dlat/2),
        d_k = r_{k+1} - r_k, a_k = lambda^2 (r_{k+1}^3 - r_k^3)/3
            = lambda^2 (r_{k+1} - r_k)(r_{k+1}^2 + r_{k+1} r_k + r_k^2)/3,
        w_{k+1/2} = beta(r_{k+1}) r_{k+1}^2 / (rc_{k+1} - rc_k),
        mu_E(j) = alpha_e dlat / (cos lat_j dlon),
        mu_N(j) = alpha_n cos lat_{j+1/2} dlon / dlat (0 on the northern edge).
        The alpha_{T,T'} of the paper is the ratio of edge length to centre
        distance (Section 3.1); |T| is the cell area on the unit sphere.
panel   one panel of an equidistant gnomonic cubed sphere (Section 3.2): cell
        (i, j) covers [x_i, x_{i+1}] x [y_j, y_{j+1}] of the tangent plane
        [-1, 1]^2, mapped to the unit sphere by P(x, y) = (1, x, y)/|(1, x, y)|;
        |T_ij| = its solid angle, mu_E = alpha (arc of the east edge)/(arc
        between the two cell centres), likewise north; radial factors as for
        latlon; the four panel edges are Neumann (zero face weight).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

from workloads import GEOM_BOX, GEOM_LATLON, GEOM_PANEL, Problem


@dataclasses.dataclass
class OperatorTerms:
    """Per-level and per-column factors of the tensor-product operator."""

    area: np.ndarray      # (n_y, n_x)   |T| of every column
    d: np.ndarray         # (n_z,)       horizontal-coupling weight per level
    mass: np.ndarray      # (n_z,)       a_k (zero-order term per unit area)
    w_up: np.ndarray      # (n_z,)       w_{k+1/2} per unit area (0 at the top level)
    mu_e: np.ndarray      # (n_y, n_x)   east-face weight
    mu_n: np.ndarray      # (n_y, n_x)   north-face weight (0 on a Neumann edge)
    periodic_y: bool


def operator_terms(p: Problem) -> OperatorTerms:
    z = np.asarray(p.z_iface, dtype=np.float64)
    nz = p.n_z
    dz = z[1:] - z[:-1]
    zc = 0.5 * (z[:-1] + z[1:])
    gap = zc[1:] - zc[:-1]                        # centre distances, n_z-1 values
    beta = np.asarray(p.beta_iface, dtype=np.float64)
    ae = np.ones((p.n_y, p.n_x)) if p.alpha_e is None else np.asarray(p.alpha_e, dtype=np.float64)
    an = np.ones((p.n_y, p.n_x)) if p.alpha_n is None else np.asarray(p.alpha_n, dtype=np.float64)
    w_up = np.zeros(nz)
    if p.kind == GEOM_BOX:
        hx = p.lx / p.n_x
        hy = p.ly / p.n_y
        area = np.full((p.n_y, p.n_x), hx * hy)
        d = dz.copy()
        mass = p.lambda2 * dz
        w_up[:-1] = beta[1:-1] / gap
        mu_e = ae * (hy / hx)
        mu_n = an * (hx / hy)
        periodic_y = True
    elif p.kind == GEOM_LATLON:
        dlon = 2.0 * np.pi / p.n_x
        dlat = (p.lat1 - p.lat0) / p.n_y
        lat_f = p.lat0 + dlat * np.arange(p.n_y + 1)          # faces lat_{j-1/2}, j = 0..n_y
        lat_c = p.lat0 + dlat * (np.arange(p.n_y) + 0.5)       # centres
        # sin(a) - sin(b) = 2 cos((a+b)/2) sin((a-b)/2) and
        # r1^3 - r0^3 = (r1 - r0)(r1^2 + r1 r0 + r0^2): the same quantities
        # without the cancellation of two nearly equal numbers
        area = np.broadcast_to((dlon * 2.0 * np.cos(lat_c) * np.sin(0.5 * dlat))[:, None], (p.n_y, p.n_x)).copy()
        d = dz.copy()
        mass = p.lambda2 * dz * (z[1:] * z[1:] + z[1:] * z[:-1] + z[:-1] * z[:-1]) / 3.0
        w_up[:-1] = beta[1:-1] * z[1:-1] ** 2 / gap
        mu_e = ae * (dlat / (np.cos(lat_c) * dlon))[:, None]
        mu_n = an * (np.cos(lat_f[1:]) * dlon / dlat)[:, None]
        mu_n = mu_n.copy()
        mu_n[-1, :] = 0.0                                       # northern edge: Neumann
        periodic_y = False
    elif p.kind == GEOM_PANEL:
        xf = -1.0 + 2.0 * np.arange(p.n_x + 1) / p.n_x
        yf = -1.0 + 2.0 * np.arange(p.n_y + 1) / p.n_y
        xc = 0.5 * (xf[1:] + xf[:-1])
        yc = 0.5 * (yf[1:] + yf[:-1])

        # all from unnormalised points (1, x, y) and exact coordinate
        # differences, so that nothing small is taken as a difference of
        # nearly equal quantities
        def nrm(x, y):
            return np.sqrt(1.0 + x * x + y * y)

        def arc_same_y(x1, x2, y):          # points (1, x1, y), (1, x2, y)
            return np.arctan2(np.abs(x2 - x1) * np.sqrt(1.0 + y * y), 1.0 + x1 * x2 + y * y)

        def arc_same_x(x, y1, y2):          # points (1, x, y1), (1, x, y2)
            return np.arctan2(np.abs(y2 - y1) * np.sqrt(1.0 + x * x), 1.0 + x * x + y1 * y2)

        def tri(xa, ya, xb, yb, xc_, yc_):
            # solid angle of a spherical triangle from unnormalised vertices
            # (Van Oosterom and Strackee, 1983)
            det = np.abs((xb - xa) * (yc_ - ya) - (xc_ - xa) * (yb - ya))
            na, nb, nc = nrm(xa, ya), nrm(xb, yb), nrm(xc_, yc_)
            ab = 1.0 + xa * xb + ya * yb
            bc = 1.0 + xb * xc_ + yb * yc_
            ca = 1.0 + xc_ * xa + yc_ * ya
            return 2.0 * np.arctan2(det, na * nb * nc + ab * nc + bc * na + ca * nb)

        X0, Y0 = np.meshgrid(xf[:-1], yf[:-1])
        X1, Y1 = np.meshgrid(xf[1:], yf[1:])
        area = tri(X0, Y0, X1, Y0, X1, Y1) + tri(X0, Y0, X1, Y1, X0, Y1)
        XC, YC = np.meshgrid(xc, yc)
        mu_e = np.zeros((p.n_y, p.n_x))
        mu_e[:, :-1] = (arc_same_x(X1, Y0, Y1)[:, :-1]
                        / arc_same_y(XC[:, :-1], XC[:, 1:], YC[:, :-1]))
        mu_n = np.zeros((p.n_y, p.n_x))
        mu_n[:-1, :] = (arc_same_y(X0, X1, Y1)[:-1, :]
                        / arc_same_x(XC[:-1, :], YC[:-1, :], YC[1:, :]))
        mu_e = ae * mu_e
        mu_n = an * mu_n
        d = dz.copy()
        mass = p.lambda2 * dz * (z[1:] * z[1:] + z[1:] * z[:-1] + z[:-1] * z[:-1]) / 3.0
        w_up[:-1] = beta[1:-1] * z[1:-1] ** 2 / gap
        periodic_y = True       # the wrapped faces carry weight 0: Neumann edges
    else:
        raise ValueError(f"unknown geometry kind {p.kind}")
    return OperatorTerms(area=area, d=d, mass=mass, w_up=w_up, mu_e=mu_e, mu_n=mu_n,
                         periodic_y=periodic_y)


def cell_volumes(p: Problem) -> np.ndarray:
    """Cell volumes (n_z, n_y, n_x): |T| dz_k (box) or |T_j| (r_{k+1}^3 - r_k^3)/3."""
    z = np.asarray(p.z_iface, dtype=np.float64)
    t = operator_terms(p)
    if p.kind == GEOM_BOX:
        vz = z[1:] - z[:-1]
    else:
        vz = (z[1:] - z[:-1]) * (z[1:] * z[1:] + z[1:] * z[:-1] + z[:-1] * z[:-1]) / 3.0
    return np.broadcast_to(vz[:, None, None] * t.area[None, :, :], p.shape).copy()


def _row_entries(p: Problem, t: OperatorTerms, k, j, i):
    """Column indices and values of the rows of cells (k, j, i) (index arrays).

    Returns (cols, vals), each of shape (7, n): diagonal, east, west, north,
    south, up, down.  Entries of absent (Neumann) couplings have value 0.
    """
    nx, ny, nz = p.n_x, p.n_y, p.n_z
    k = np.asarray(k, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    i = np.asarray(i, dtype=np.int64)
    area = t.area[j, i]
    dk = t.d[k]
    ie = (i + 1) % nx
    iw = (i - 1) % nx
    jn = (j + 1) % ny
    js = (j - 1) % ny
    c_e = dk * t.mu_e[j, i]
    c_w = dk * t.mu_e[j, iw]
    c_n = dk * t.mu_n[j, i]
    if t.periodic_y:
        c_s = dk * t.mu_n[js, i]
    else:
        c_s = np.where(j > 0, dk * t.mu_n[js, i], 0.0)
    c_u = area * t.w_up[k]                                   # zero at the top level
    c_d = np.where(k > 0, area * t.w_up[np.maximum(k - 1, 0)], 0.0)
    diag = area * t.mass[k] + (c_e + c_w + c_n + c_s) + (c_u + c_d)

    def lin(kk, jj, ii):
        return (kk * ny + jj) * nx + ii

    ku = np.minimum(k + 1, nz - 1)
    kd = np.maximum(k - 1, 0)
    cols = np.stack([lin(k, j, i), lin(k, j, ie), lin(k, j, iw), lin(k, jn, i), lin(k, js, i),
                     lin(ku, j, i), lin(kd, j, i)])
    vals = np.stack([diag, -c_e, -c_w, -c_n, -c_s, -c_u, -c_d])
    return cols, vals


def assemble_csr(p: Problem) -> sp.csr_matrix:
    """The full n x n operator in CSR form, rows and columns in the canonical
    order l = (k n_y + j) n_x + i."""
    t = operator_terms(p)
    n = p.n_cells
    kk, jj, ii = np.meshgrid(np.arange(p.n_z), np.arange(p.n_y), np.arange(p.n_x), indexing="ij")
    cols, vals = _row_entries(p, t, kk.ravel(), jj.ravel(), ii.ravel())
    rows = np.broadcast_to(np.arange(n, dtype=np.int64), cols.shape)
    keep = vals != 0.0
    keep[0, :] = True
    a = sp.coo_matrix((vals[keep], (rows[keep], cols[keep])), shape=(n, n))
    a = a.tocsr()
    a.sum_duplicates()
    a.sort_indices()
    return a


class FluxOperator:
    """The operator applied in flux form: (A x)_l = m_l x_l + sum_j c_lj (x_l - x_j).

    ``C`` holds the positive couplings c_lj = -A_lj (l != j) as an explicit
    CSR matrix and ``mass`` the zero-order terms m_l = |T| a_k.  This is the
    row of Eq. (TridiagonalMatrix) with its diagonal written as the sum of its
    parts (the paper's alpha_T is the sum of the horizontal couplings), and it
    is the form in which the finite-volume fluxes are defined.  It is also the
    form that keeps the operator exact on near-constant vectors: the stored
    FP64 diagonal of the assembled matrix cannot resolve m_l when m_l is below
    the rounding of the much larger couplings, so A 1 computed from assembled
    entries is wrong in the low bits that carry the zero-order term, whereas
    here A 1 = m exactly.
    """

    def __init__(self, p: Problem):
        self.p = p
        t = operator_terms(p)
        self.terms = t
        n = p.n_cells
        kk, jj, ii = np.meshgrid(np.arange(p.n_z), np.arange(p.n_y), np.arange(p.n_x), indexing="ij")
        k, j = kk.ravel(), jj.ravel()
        cols, vals = _row_entries(p, t, k, j, ii.ravel())
        self.mass = t.area[j, ii.ravel()] * t.mass[k]
        rows = np.broadcast_to(np.arange(n, dtype=np.int64), cols[1:].shape)
        c = -vals[1:]
        keep = c != 0.0
        cm = sp.coo_matrix((c[keep], (rows[keep], cols[1:][keep])), shape=(n, n)).tocsr()
        cm.sum_duplicates()
        cm.sort_indices()
        self.C = cm
        self._rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(cm.indptr))
        self.shape = (n, n)

    def matvec(self, x: np.ndarray) -> np.ndarray:
        xf = np.asarray(x, dtype=np.float64).reshape(-1)
        flux = self.C.data * (xf[self._rows] - xf[self.C.indices])
        y = self.mass * xf
        y += np.bincount(self._rows, weights=flux, minlength=xf.size)
        return y

    def __matmul__(self, x):
        return self.matvec(x)

    def diagonal(self) -> np.ndarray:
        return self.mass + np.asarray(self.C.sum(axis=1)).ravel()


def apply_rows(p: Problem, x: np.ndarray, cells) -> np.ndarray:
    """(A x) at the given cells only, in flux form; ``cells`` is a (3, m)
    array of (k, j, i).

    Evaluates the rows of ``FluxOperator`` without forming the matrix, so
    that sampled outputs of very large problems can be checked one by one.
    """
    t = operator_terms(p)
    k, j, i = (np.asarray(c, dtype=np.int64) for c in cells)
    cols, vals = _row_entries(p, t, k, j, i)
    xf = np.asarray(x, dtype=np.float64).reshape(-1)
    xi = xf[cols[0]]
    y = t.area[j, i] * t.mass[k] * xi
    for f in range(1, 7):
        y = y + (-vals[f]) * (xi - xf[cols[f]])
    return y


def column_blocks(a: sp.csr_matrix, p: Problem):
    """Tridiagonal column blocks of A (the matrix M of Section 4.2).

    Returns (lower, main, upper) of shape (n_y n_x, n_z) in column-contiguous
    order (the paper's CPU layout l = n_z nu(T) + k, Eq. (MemoryMappingCPU));
    ``lower[c, k]`` couples level k to k-1 and ``upper[c, k]`` couples k to k+1.
    Entries are read out of the assembled matrix, so M is block-diag(A) exactly.
    """
    nz, ncol = p.n_z, p.n_x * p.n_y
    plane = ncol
    idx = np.arange(p.n_cells, dtype=np.int64).reshape(nz, ncol)
    main = np.asarray(a[idx.ravel(), idx.ravel()]).reshape(nz, ncol).T
    upper = np.zeros((ncol, nz))
    lower = np.zeros((ncol, nz))
    if nz > 1:
        r = idx[:-1].ravel()
        upper[:, :-1] = np.asarray(a[r, r + plane]).reshape(nz - 1, ncol).T
        r = idx[1:].ravel()
        lower[:, 1:] = np.asarray(a[r, r - plane]).reshape(nz - 1, ncol).T
    return lower, main, upper
