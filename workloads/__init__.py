"""Seeded, synthetic problem inputs shared by the CUDA path and the CPU oracle.

This module holds only *problem data*: grid interfaces, coefficient fields
sampled where the solver library expects them, and right-hand sides drawn
from seeded generators.  It contains none of the method's arithmetic (no
metric terms, no stencil, no solver).  Both sides receive the arrays built
here and derive everything else on their own.

Problem classes follow the workloads of the paper (Section 7.2: a
256 x 256 x 128 column grid with strong vertical anisotropy) and the
model equation of Section 3, Eq. (ModelEquation), in the generalised form

    -div_h(alpha grad_h u) - (1/S) d_z(S beta d_z u) + lambda^2 u = f

on either a periodic unit square ("box") or a latitude-longitude band of a
thin spherical shell ("latlon", S = r^2).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

GEOM_BOX = 0
GEOM_LATLON = 1
GEOM_PANEL = 2      # one panel of an equidistant gnomonic cubed sphere, tangent coordinates [-1, 1]^2


@dataclasses.dataclass
class Problem:
    """One discrete elliptic problem on a tensor-product column grid.

    Arrays use the canonical layout of the library: horizontal fields are
    ``[n_y][n_x]`` (x fastest), vertical profiles are length ``n_z + 1``
    (values at the level interfaces ``z_0 .. z_{n_z}``).
    """

    kind: int
    n_x: int
    n_y: int
    n_z: int
    z_iface: np.ndarray          # (n_z+1,) increasing interface heights (box) or radii (latlon)
    beta_iface: np.ndarray       # (n_z+1,) vertical diffusion coefficient at the interfaces
    lambda2: float               # zero-order coefficient lambda^2
    alpha_e: Optional[np.ndarray] = None  # (n_y, n_x) alpha at the east face of cell (i, j); None = 1
    alpha_n: Optional[np.ndarray] = None  # (n_y, n_x) alpha at the north face of cell (i, j); None = 1
    lx: float = 1.0              # box: domain extent in x (periodic)
    ly: float = 1.0              # box: domain extent in y (periodic)
    lat0: float = 0.0            # latlon: southern edge latitude [rad] (Neumann)
    lat1: float = 0.0            # latlon: northern edge latitude [rad] (Neumann)
    name: str = ""

    @property
    def n_cells(self) -> int:
        return self.n_x * self.n_y * self.n_z

    @property
    def shape(self):
        return (self.n_z, self.n_y, self.n_x)


def graded_interfaces(n_z: int, thickness: float, ratio: float = 1.05, base: float = 0.0) -> np.ndarray:
    """Interfaces base = z_0 < ... < z_{n_z} = base + thickness whose spacings
    grow geometrically by ``ratio`` from the bottom (finest cells at the
    ground, as the paper asks of a meteorological grid in Section 3.1)."""
    k = np.arange(n_z + 1, dtype=np.float64)
    if ratio == 1.0:
        frac = k / n_z
    else:
        frac = (ratio ** k - 1.0) / (ratio ** n_z - 1.0)
    z = base + thickness * frac
    z[0] = base
    z[-1] = base + thickness
    return z


def smooth_graded_interfaces(n_z: int, thickness: float, q0: float = 1.05, span: float = 16.0) -> np.ndarray:
    """Interfaces z(s) = thickness (q0^(span s) - 1)/(q0^span - 1), s = k/n_z:
    a fixed smooth grading map, so that doubling n_z halves every spacing
    (used for grid-refinement studies)."""
    s = np.arange(n_z + 1, dtype=np.float64) / n_z
    z = thickness * (q0 ** (span * s) - 1.0) / (q0 ** span - 1.0)
    z[0] = 0.0
    z[-1] = thickness
    return z


def exp_profile(z: np.ndarray, scale: float, origin: float = 0.0) -> np.ndarray:
    """beta(z) = exp(-(z - origin)/scale) sampled at the given points."""
    return np.exp(-(np.asarray(z, dtype=np.float64) - origin) / scale)


def sinusoidal_alpha(n_x: int, n_y: int, amp: float = 0.5):
    """alpha(x, y) = 1 + amp sin(2 pi x) sin(2 pi y) on the unit square,
    sampled at the east-face and north-face midpoints of every cell."""
    i = np.arange(n_x, dtype=np.float64)
    j = np.arange(n_y, dtype=np.float64)
    hx, hy = 1.0 / n_x, 1.0 / n_y
    # east face of cell (i, j): x = (i+1) hx, y = (j+1/2) hy
    xe = (i + 1.0) * hx
    yc = (j + 0.5) * hy
    alpha_e = 1.0 + amp * np.outer(np.sin(2 * np.pi * yc), np.sin(2 * np.pi * xe))
    # north face of cell (i, j): x = (i+1/2) hx, y = (j+1) hy
    xc = (i + 0.5) * hx
    yn = (j + 1.0) * hy
    alpha_n = 1.0 + amp * np.outer(np.sin(2 * np.pi * yn), np.sin(2 * np.pi * xc))
    return np.ascontiguousarray(alpha_e), np.ascontiguousarray(alpha_n)


def box_problem(n_x, n_y, n_z, depth, *, ratio=1.05, beta_scale=0.005, lambda2=1e-2,
                alpha=None, name="") -> Problem:
    z = graded_interfaces(n_z, depth, ratio)
    ae = an = None
    if alpha == "sin":
        ae, an = sinusoidal_alpha(n_x, n_y)
    return Problem(kind=GEOM_BOX, n_x=n_x, n_y=n_y, n_z=n_z, z_iface=z,
                   beta_iface=exp_profile(z, beta_scale), lambda2=float(lambda2),
                   alpha_e=ae, alpha_n=an, name=name)


def latlon_problem(n_lon, n_lat, n_z, *, thickness=0.002, lat_deg=80.0, ratio=1.05,
                   beta_scale=0.005, lambda2=1e-2, name="") -> Problem:
    r = graded_interfaces(n_z, thickness, ratio, base=1.0)
    lat = math.radians(lat_deg)
    return Problem(kind=GEOM_LATLON, n_x=n_lon, n_y=n_lat, n_z=n_z, z_iface=r,
                   beta_iface=exp_profile(r, beta_scale, origin=1.0), lambda2=float(lambda2),
                   lat0=-lat, lat1=lat, name=name)


def panel_problem(n_x, n_y, n_z, *, thickness=0.01, omega2=6.71e-4, lambda2_vertical=3.32e-2,
                  name="") -> Problem:
    """The paper's test problem (Section 3, Eq. (ModelEquation); Section 7.2):
    -omega^2 (Lap_2d + lambda^2 r^-2 d_r(r^2 d_r)) u + u = f on one panel of a
    gnomonic cubed sphere times r in [1, 1 + H], with the quadratically graded
    levels r_k = 1 + (k/n_z)^2 H of Section 3.1.  In the library's form this
    is alpha = omega^2, beta = omega^2 lambda^2 and a zero-order coefficient 1.
    The paper does not give H; ``thickness`` is that reading."""
    k = np.arange(n_z + 1, dtype=np.float64)
    r = 1.0 + (k / n_z) ** 2 * thickness
    a = np.full((n_y, n_x), omega2)
    return Problem(kind=GEOM_PANEL, n_x=n_x, n_y=n_y, n_z=n_z, z_iface=r,
                   beta_iface=np.full(n_z + 1, omega2 * lambda2_vertical), lambda2=1.0,
                   alpha_e=a, alpha_n=a.copy(), name=name or f"panel{n_x}x{n_y}x{n_z}")


# ---------------------------------------------------------------------------
# Right-hand sides
# ---------------------------------------------------------------------------

def uniform_rhs(shape, seed: int) -> np.ndarray:
    """i.i.d. uniform[-1, 1] values from numpy's PCG64 generator with ``seed``."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=shape)


def smooth_mode(p: Problem) -> np.ndarray:
    """sin(2 pi x) cos(2 pi y) * zeta with zeta = (cell-centre height)/depth
    in [0, 1], sampled at cell centres of a box problem."""
    x = (np.arange(p.n_x) + 0.5) / p.n_x * p.lx
    y = (np.arange(p.n_y) + 0.5) / p.n_y * p.ly
    zc = 0.5 * (p.z_iface[:-1] + p.z_iface[1:])
    zeta = (zc - p.z_iface[0]) / (p.z_iface[-1] - p.z_iface[0])
    return zeta[:, None, None] * np.outer(np.cos(2 * np.pi * y), np.sin(2 * np.pi * x))[None, :, :]


def rhs_for(p: Problem, seed: int = 0, smooth: bool = False) -> np.ndarray:
    b = uniform_rhs(p.shape, seed)
    if smooth:
        b = b + smooth_mode(p)
    return np.ascontiguousarray(b)


def batched_rhs(p: Problem, seeds) -> np.ndarray:
    """One uniform right-hand side per seed, stacked as [nrhs][n_z][n_y][n_x]."""
    return np.ascontiguousarray(np.stack([uniform_rhs(p.shape, s) for s in seeds]))


# ---------------------------------------------------------------------------
# Named workloads (sizes of the full problems; ``scale`` shrinks the horizontal
# grid for tests while keeping the vertical structure)
# ---------------------------------------------------------------------------

def small_box(scale: int = 1) -> Problem:
    """32 x 32 x 16 periodic box, depth 0.01, grading 1.05, alpha = 1,
    beta = exp(-z/0.005), lambda^2 = 1e-2 (plain FP64 PCG, tol 1e-8)."""
    return box_problem(32 // scale, 32 // scale, 16, 0.01, name="box32x32x16")


def medium_box(scale: int = 1, n_z: int = 128) -> Problem:
    """256 x 256 x 128 periodic box, depth 0.004 (horizontal/vertical spacing
    ratio ~1e2); same coefficients as the small box (plain FP64, tol 1e-8)."""
    n = 256 // scale
    return box_problem(n, n, n_z, 0.004, name=f"box{n}x{n}x{n_z}")


def medium_box_rhs(p: Problem) -> np.ndarray:
    """Seed-0 uniform values plus the smooth mode sin(2 pi x) cos(2 pi y) zeta."""
    return rhs_for(p, seed=0, smooth=True)


def large_box(scale: int = 1, n_z: int = 128) -> Problem:
    """1024 x 1024 x 128 periodic box, depth 0.01, alpha = 1 + 0.5 sin sin,
    beta = exp(-z/0.005), lambda^2 = 1e-2 (mixed precision, tol 1e-8)."""
    n = 1024 // scale
    return box_problem(n, n, n_z, 0.01, alpha="sin", name=f"box{n}x{n}x{n_z}_sinalpha")


def shell_band(scale: int = 1, n_z: int = 64) -> Problem:
    """1440 x 640 latitude-longitude band (+-80 deg) of the shell
    r in [1, 1.002], n_z graded levels, alpha = 1, beta = exp(-(r-1)/0.005),
    lambda^2 = 1e-2."""
    return latlon_problem(1440 // scale, 640 // scale, n_z, name=f"latlon{1440 // scale}x{640 // scale}x{n_z}")


# ---------------------------------------------------------------------------
# Served request stream
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Request:
    index: int
    arrival_s: float
    problem: Problem
    rhs_seed: int
    tol: float = 1e-8


def request_stream(duration_s: float = 20.0, rate_hz: float = 200.0, seed: int = 1,
                   sizes=(64, 128, 256, 512), levels=(32, 64, 128), max_requests: Optional[int] = None):
    """Poisson arrivals of solves with random sizes and anisotropies.

    n_x and n_y are drawn independently from ``sizes``, n_z from ``levels``;
    log10(anisotropy) ~ U[2, 5] sets depth = n_z h / sqrt(anisotropy) with
    h = sqrt(hx hy); lambda^2 is log-uniform in [1e-4, 1]; request i uses the
    right-hand-side seed 1000 + i.
    """
    rng = np.random.default_rng(seed)
    out = []
    t = 0.0
    i = 0
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t > duration_s or (max_requests is not None and i >= max_requests):
            break
        n_x = int(rng.choice(sizes))
        n_y = int(rng.choice(sizes))
        n_z = int(rng.choice(levels))
        aniso = 10.0 ** rng.uniform(2.0, 5.0)
        lam2 = 10.0 ** rng.uniform(-4.0, 0.0)
        h = math.sqrt((1.0 / n_x) * (1.0 / n_y))
        depth = n_z * h / math.sqrt(aniso)
        p = box_problem(n_x, n_y, n_z, depth, lambda2=lam2, name=f"req{i}")
        out.append(Request(index=i, arrival_s=t, problem=p, rhs_seed=1000 + i))
        i += 1
    return out
