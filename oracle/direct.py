"""Exact small-system solvers and closed forms used to pin the oracle.

Test infrastructure only.  Each routine here is independent of
:mod:`oracle.bicgstab`, so agreement between them is evidence, not
repetition.
"""

from __future__ import annotations

import numpy as np

from . import stencil


def dense_solve(nx, ny, nz, coef, b):
    """Direct solve of the assembled matrix (LAPACK LU with partial pivoting)."""
    a = stencil.assemble_dense(nx, ny, nz, coef)
    return np.linalg.solve(a, np.asarray(b, dtype=np.float64))


def cg(nx, ny, nz, coef, b, tol=1e-14, maxit=10000):
    """Conjugate gradients (Hestenes-Stiefel) for a symmetric positive
    definite stencil operator, written independently of the BiCGStab code."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(r @ r)
    nb = np.sqrt(float(b @ b))
    for _ in range(maxit):
        if np.sqrt(rr) <= tol * nb:
            break
        ap = stencil.apply(nx, ny, nz, coef, p)
        a = rr / float(p @ ap)
        x += a * p
        r -= a * ap
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x


def thomas(lower, diag, upper, rhs):
    """Tridiagonal solve (Thomas algorithm).  ``lower[i]`` multiplies
    ``x[i-1]`` in row ``i`` (``lower[0]`` unused); ``upper[i]`` multiplies
    ``x[i+1]`` (``upper[-1]`` unused)."""
    n = len(diag)
    c = np.zeros(n)
    d = np.zeros(n)
    c[0] = upper[0] / diag[0]
    d[0] = rhs[0] / diag[0]
    for i in range(1, n):
        m = diag[i] - lower[i] * c[i - 1]
        c[i] = upper[i] / m if i < n - 1 else 0.0
        d[i] = (rhs[i] - lower[i] * d[i - 1]) / m
    x = np.zeros(n)
    x[-1] = d[-1]
    for i in range(n - 2, -1, -1):
        x[i] = d[i] - c[i] * x[i + 1]
    return x


def laplacian_eigenpair(nx, ny, nz, kx, ky, kz):
    """Closed-form eigenpair of the 7-point Dirichlet Laplacian
    (diagonal 6, off-diagonals -1): the separable sine mode with 1-based wave
    numbers ``(kx, ky, kz)`` and eigenvalue ``sum_d 2 (1 - cos(k_d pi/(n_d+1)))``.
    """
    x = np.arange(1, nx + 1)
    y = np.arange(1, ny + 1)
    z = np.arange(1, nz + 1)
    vx = np.sin(kx * np.pi * x / (nx + 1))
    vy = np.sin(ky * np.pi * y / (ny + 1))
    vz = np.sin(kz * np.pi * z / (nz + 1))
    v = (vz[:, None, None] * vy[None, :, None] * vx[None, None, :]).reshape(-1)
    lam = sum(2.0 * (1.0 - np.cos(k * np.pi / (m + 1)))
              for k, m in ((kx, nx), (ky, ny), (kz, nz)))
    return lam, v
