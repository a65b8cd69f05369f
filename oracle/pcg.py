"""Preconditioned conjugate gradients: textbook, interleaved (Algorithm 1) and
single-reduction (Chronopoulos-Gear).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings of the paper used here (each is also listed with the design notes):

* Initial state of Algorithm 1 (not given in the paper): u = u0 (zero unless a
  guess is passed), r = b - A u0, p = q = 0, alpha = 0, kappa_old = 1.  The
  first pass of the loop then yields p = z, q = A z.
* Stopping test of Algorithm 1 (Section 4.3): ||r|| / ||r_0|| < eps or
  ||r|| < tau.  With u0 = 0, ||r_0|| = ||b||; the reference norm is taken as
  ||b|| for every start, so that warm starts and iterative-refinement
  corrections stop on the same criterion.  tau defaults to 0.
* Algorithm 1 updates u one step behind r: when the test fires, u has not yet
  received the last alpha p.  That update is applied once after the loop, so
  the returned u matches the residual that passed the test.
* An iteration is one update of u (one application of A to a new search
  direction).  Exiting at the test of pass k of Algorithm 1 therefore counts
  k - 1 iterations; running out of passes counts ``maxiter``.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List, Optional

import numpy as np


@dataclasses.dataclass
class PCGResult:
    x: np.ndarray
    iterations: int
    converged: bool
    residual_history: List[float]      # ||r_k|| of the recursively updated residual, k = 0..
    final_true_relres: float


def _dot(a, b):
    return float(np.dot(a.ravel(), b.ravel()))


def _true_relres(A, b, x):
    bn = np.linalg.norm(b.ravel())
    r = b.ravel() - A @ x.ravel()
    return float(np.linalg.norm(r) / bn) if bn > 0 else float(np.linalg.norm(r))


def pcg_textbook(A, precond: Callable, b: np.ndarray, x0: Optional[np.ndarray] = None,
                 tol: float = 1e-8, maxit: int = 10000, tau: float = 0.0) -> PCGResult:
    """Left-preconditioned CG for SPD A and M (Section 4.1).

    Per iteration: q = A p, alpha = <r,z>/<p,q>, x += alpha p, r -= alpha q,
    stop if ||r|| < tol ||b|| (or < tau), z = M^{-1} r, beta = <r,z>_new/<r,z>_old,
    p = z + beta p.
    """
    shape = b.shape
    b = np.asarray(b, dtype=np.float64).ravel()
    x = np.zeros_like(b) if x0 is None else np.asarray(x0, dtype=np.float64).ravel().copy()
    bnorm = float(np.linalg.norm(b))
    r = b - A @ x
    hist = [float(np.linalg.norm(r))]
    it = 0

    def done(rn):
        return rn == 0.0 or rn < tol * bnorm or rn < tau

    if done(hist[-1]):
        return PCGResult(x.reshape(shape), 0, True, hist, _true_relres(A, b, x))
    z = precond(r.reshape(shape)).ravel()
    p = z.copy()
    rz = _dot(r, z)
    converged = False
    while it < maxit:
        q = A @ p
        alpha = rz / _dot(p, q)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        hist.append(float(np.linalg.norm(r)))
        if done(hist[-1]):
            converged = True
            break
        z = precond(r.reshape(shape)).ravel()
        rz_new = _dot(r, z)
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return PCGResult(x.reshape(shape), it, converged, hist, _true_relres(A, b, x))


def pcg_interleaved(A, precond: Callable, b: np.ndarray, u0: Optional[np.ndarray] = None,
                    eps: float = 1e-8, maxiter: int = 10000, tau: float = 0.0) -> PCGResult:
    """Algorithm 1 of the paper, two grid sweeps per pass.

    Sweep 1 (preconditioner kernel): r <- r - alpha q, z = M^{-1} r,
    ||r|| = sqrt(<r,r>), kappa = <r,z>; exit test; beta = kappa/kappa_old,
    kappa_old = kappa.  Sweep 2 (SpMV kernel): u <- u + alpha p,
    p <- z + beta p, q <- A z + beta q, sigma = <p,q>; alpha = kappa_old/sigma.
    """
    shape = b.shape
    b = np.asarray(b, dtype=np.float64).ravel()
    u = np.zeros_like(b) if u0 is None else np.asarray(u0, dtype=np.float64).ravel().copy()
    bnorm = float(np.linalg.norm(b))
    r = b - A @ u
    p = np.zeros_like(b)
    q = np.zeros_like(b)
    alpha = 0.0
    kappa_old = 1.0
    hist: List[float] = []
    converged = False
    passes = 0
    for k in range(1, maxiter + 2):
        # one more pass than maxiter so that maxiter full iterations are taken
        r = r - alpha * q
        z = precond(r.reshape(shape)).ravel()
        rnorm = float(np.sqrt(_dot(r, r)))
        kappa = _dot(r, z)
        hist.append(rnorm)
        if rnorm == 0.0 or rnorm < eps * bnorm or rnorm < tau:
            converged = True
            passes = k
            break
        if k == maxiter + 1:
            passes = k
            break
        beta = kappa / kappa_old
        kappa_old = kappa
        u = u + alpha * p
        p = z + beta * p
        q = (A @ z) + beta * q
        sigma = _dot(p, q)
        alpha = kappa_old / sigma
    u = u + alpha * p
    return PCGResult(u.reshape(shape), passes - 1, converged, hist, _true_relres(A, b, u))


def pcg_single_reduction(A, precond: Callable, b: np.ndarray, x0: Optional[np.ndarray] = None,
                         eps: float = 1e-8, maxiter: int = 10000, tau: float = 0.0) -> PCGResult:
    """PCG with one reduction phase per iteration (Chronopoulos and Gear, 1989).

    Section 4.3 of the paper points to this rearrangement of CG (fused loops
    with the inner products gathered in one place).  With u = M^{-1} r,
    w = A u, gamma = <r, u> and delta = <w, u>, the step lengths come from
    one reduction:
      beta  = gamma / gamma_old                                   (0 on the first step),
      alpha = gamma / (delta - beta gamma / alpha_old)            (gamma / delta on the first step),
    and the search direction p and s = A p follow by recurrence:
      p = u + beta p,  s = w + beta s,  x = x + alpha p,  r = r - alpha s.
    In exact arithmetic the iterates are those of textbook PCG (delta -
    beta gamma / alpha_old is <p, A p>).

    Written as the passes the one-sweep GPU form takes: every pass applies the
    previous pass's alpha and beta to p, s, x and r, then forms u = M^{-1} r,
    w = A u and the three inner products (||r||^2, gamma, delta), and the
    stopping test on ||r||.  The first pass starts from u = w = p = s = 0 and
    alpha = beta = 0, so it only forms u, w and the first products.  x is
    current when the test fires (no fix-up).  Iterations count the updates of
    x: exiting at the test of pass k counts k - 1.  The stopping reference is
    ||b|| (as in ``pcg_interleaved``).
    """
    shape = b.shape
    b = np.asarray(b, dtype=np.float64).ravel()
    x = np.zeros_like(b) if x0 is None else np.asarray(x0, dtype=np.float64).ravel().copy()
    bnorm = float(np.linalg.norm(b))
    r = b - A @ x
    u = np.zeros_like(b)
    w = np.zeros_like(b)
    p = np.zeros_like(b)
    s = np.zeros_like(b)
    alpha = beta = 0.0
    gamma_old = 1.0
    first = True
    hist: List[float] = []
    converged = False
    passes = 0
    for k in range(1, maxiter + 2):
        p = u + beta * p
        s = w + beta * s
        x = x + alpha * p
        r = r - alpha * s
        u = precond(r.reshape(shape)).ravel()
        w = A @ u
        rnorm = float(np.sqrt(_dot(r, r)))
        gamma = _dot(r, u)
        delta = _dot(w, u)
        hist.append(rnorm)
        if rnorm == 0.0 or rnorm < eps * bnorm or rnorm < tau:
            converged = True
            passes = k
            break
        if k == maxiter + 1:
            passes = k
            break
        if first:
            beta, alpha = 0.0, gamma / delta
            first = False
        else:
            beta = gamma / gamma_old
            alpha = gamma / (delta - beta * gamma / alpha)
        gamma_old = gamma
    return PCGResult(x.reshape(shape), passes - 1, converged, hist, _true_relres(A, b, x))


def rounding_floor(A, x: np.ndarray, b: np.ndarray) -> float:
    """Expected ||b - A fl(x)|| / ||b|| when x is rounded to FP64.

    Rounding perturbs each x_j by an independent error uniform in
    [-ulp(x_j)/2, ulp(x_j)/2] (variance ulp^2/12), so
    E ||A dx||^2 = sum_j ulp(x_j)^2/12 ||A e_j||^2.  No FP64 vector near the
    solution can show a smaller true residual than about this value.
    ``A`` is the assembled matrix (its column norms are used).
    """
    xf = np.asarray(x, dtype=np.float64).ravel()
    ulp = np.spacing(np.abs(xf))
    a2 = A.multiply(A)
    col2 = np.asarray(a2.sum(axis=0)).ravel()
    bn = float(np.linalg.norm(np.asarray(b).ravel()))
    return float(np.sqrt(np.sum(ulp * ulp / 12.0 * col2)) / bn) if bn > 0 else 0.0
