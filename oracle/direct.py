"""Exact small-system solvers and closed forms used to pin the oracle.

Test infrastructure only.  Each routine here is independent of
:mod:`oracle.bicgstab`, so agreement between them is evidence, not
repetition.
"""

from __future__ import annotations

import numpy as np

from . import stencil, stencil9


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


def dense_solve9(nx, ny, coef, b):
    """Direct solve of the assembled 2D 9-point matrix (LAPACK LU)."""
    a = stencil9.assemble_dense(nx, ny, coef)
    return np.linalg.solve(a, np.asarray(b, dtype=np.float64))


def ninepoint_eigenpair(nx, ny, a0, ax, ay, c, j, k):
    """Eigenpair of the constant 2D 9-point operator of tensor-product form.

    With ``T`` the 1D Dirichlet neighbour-sum operator (``(T u)_i = u_{i-1} +
    u_{i+1}``, zero outside), the operator with diagonal ``a0``, axis
    coefficients ``ax`` (x) and ``ay`` (y) and all four corner coefficients
    ``c`` is ``a0 I + ax T_x + ay T_y + c T_x T_y``.  The sine vectors
    ``sin(j pi (x+1)/(nx+1)) sin(k pi (y+1)/(ny+1))`` diagonalise every
    ``T``, with eigenvalue ``2 cos(j pi/(nx+1))`` (resp. k, ny), so the
    eigenvalue is ``a0 + 2 ax cx + 2 ay cy + 4 c cx cy``.
    Returns ``(lambda, v)`` with ``v`` of unit 2-norm, x-fastest.
    """
    tx = j * np.pi / (nx + 1)
    ty = k * np.pi / (ny + 1)
    vx = np.sin(tx * np.arange(1, nx + 1))
    vy = np.sin(ty * np.arange(1, ny + 1))
    v = np.outer(vy, vx).reshape(-1)
    v /= np.linalg.norm(v)
    cx, cy = np.cos(tx), np.cos(ty)
    return a0 + 2 * ax * cx + 2 * ay * cy + 4 * c * cx * cy, v
