"""Algorithm 1 (standard BiCGStab) in float64 (test infrastructure only).

The paper's iteration (Sec. III, Algorithm 1), with ``r0`` the fixed shadow
residual:

    s_i     = A p_i
    alpha_i = (r0, r_i) / (r0, s_i)
    q_i     = r_i - alpha_i s_i
    y_i     = A q_i
    omega_i = (q_i, y_i) / (y_i, y_i)
    x_{i+1} = x_i + alpha_i p_i + omega_i q_i
    r_{i+1} = q_i - omega_i y_i
    beta_i  = (alpha_i / omega_i) (r0, r_{i+1}) / (r0, r_i)
    p_{i+1} = r_{i+1} + beta_i (p_i - omega_i s_i)

Readings where the paper is silent or garbled (each is listed in the
project's design notes):

* The x update is printed with ``x_i`` on both sides; it is read as
  ``x_{i+1} = x_i + alpha_i p_i + omega_i q_i``.
* The algorithm starts from ``r0 = b`` (i.e. ``x0 = 0``); for a general
  ``x0`` the start is ``r_0 = b - A x0``, ``r0_hat = r_0``, ``p_0 = r_0``.
* No stopping rule is printed.  A solve stops after the full step in which
  the recurrence residual satisfies ``||r_{i+1}|| / ||b|| <= tol`` (2-norms),
  or after ``maxit`` steps; ``hist[k] = ||r_k|| / ||b||``.  With ``b = 0``
  the answer is ``x = 0`` after zero steps.  If ``hist[0] <= tol`` no step is
  taken.
* Breakdown (not discussed in the paper): ``(r0, s) = 0``, ``omega = 0``,
  ``(r0, r_{i+1}) = 0`` before convergence, or any non-finite scalar stops
  the solve with status BREAKDOWN.  If ``(y, y) = 0`` then ``q = 0``
  exactly; the half step ``x += alpha p`` is taken and the solve ends as
  converged if ``||q|| <= tol ||b||``.
* With ``jacobi=True`` the iteration runs on the diagonally preconditioned
  system ``D^-1 A x = D^-1 b`` (Sec. IV: the main diagonal is all ones and
  only six diagonals are stored); ``tol`` and ``hist`` refer to that system.

The same iteration serves the 3D 7-point operator (:func:`bicgstab`) and the
2D 9-point operator of Sec. IV-A (:func:`bicgstab9`); only the operator
differs.

Status codes follow the library's: 0 converged, 3 breakdown, 4 not
converged within ``maxit``.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import stencil, stencil9

OK, BREAKDOWN, NOTCONV = 0, 3, 4


class _Mesh3:
    """The 3D 7-point operator of :mod:`oracle.stencil` on an nx x ny x nz mesh."""

    def __init__(self, nx, ny, nz):
        self.dims = (nx, ny, nz)

    def system(self, coef, b, jacobi, storage):
        if jacobi:
            return (stencil.jacobi_scale(*self.dims, coef, storage),
                    stencil.scale_rhs(*self.dims, coef, b))
        return stencil.rounded(*self.dims, coef, storage), b.copy()

    def apply(self, op, v):
        return stencil.apply(*self.dims, op, v)


class _Mesh9:
    """The 2D 9-point operator of :mod:`oracle.stencil9` on an nx x ny mesh."""

    def __init__(self, nx, ny):
        self.dims = (nx, ny)

    def system(self, coef, b, jacobi, storage):
        if jacobi:
            return (stencil9.jacobi_scale(*self.dims, coef, storage),
                    stencil9.scale_rhs(*self.dims, coef, b))
        return stencil9.rounded(*self.dims, coef, storage), b.copy()

    def apply(self, op, v):
        return stencil9.apply(*self.dims, op, v)


@dataclass
class Result:
    x: np.ndarray
    iters: int
    hist: np.ndarray          # hist[0..iters]
    status: int
    true_resid: float         # ||b~ - A~ x|| / ||b~|| on the solved system
    true_resid_orig: float    # ||b - A x|| / ||b|| on the raw system


def _dot(a, b):
    return float(np.dot(a, b))


def bicgstab(nx, ny, nz, coef, b, x0=None, tol=1e-8, maxit=500,
             jacobi=True, storage="f64", half_step=False):
    """Solve ``A x = b`` by Algorithm 1 in float64.

    ``coef`` holds the raw operator (``diag`` and the six directions);
    ``storage`` is the type the scaled operator is rounded to (the system the
    GPU path actually holds).  Returns a :class:`Result`.
    """
    return _bicgstab(_Mesh3(nx, ny, nz), coef, b, x0, tol, maxit, jacobi, storage, half_step)


def bicgstab9(nx, ny, coef, b, x0=None, tol=1e-8, maxit=500,
              jacobi=True, storage="f64", half_step=False):
    """:func:`bicgstab` on the 2D 9-point operator (Sec. IV-A, "SpMV (2D)");
    ``coef`` holds ``diag`` and the eight directions of :mod:`oracle.stencil9`."""
    return _bicgstab(_Mesh9(nx, ny), coef, b, x0, tol, maxit, jacobi, storage, half_step)


def _bicgstab(mesh, coef, b, x0, tol, maxit, jacobi, storage, half_step):
    b = np.asarray(b, dtype=np.float64)
    n = b.size
    op, bt = mesh.system(coef, b, jacobi, storage)

    def A(v):
        return mesh.apply(op, v)

    x = np.zeros(n) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    bnorm = np.sqrt(_dot(bt, bt))
    hist = [0.0]
    if bnorm == 0.0:
        return _finish(mesh, coef, op, b, bt, np.zeros(n), 0, [0.0], OK)

    r = bt - A(x)
    rhat = r.copy()
    p = r.copy()
    rho = _dot(rhat, r)
    hist = [np.sqrt(_dot(r, r)) / bnorm]
    if hist[0] <= tol:
        return _finish(mesh, coef, op, b, bt, x, 0, hist, OK)

    status = NOTCONV
    it = 0
    for i in range(maxit):
        s = A(p)
        sigma = _dot(rhat, s)
        if sigma == 0.0 or not np.isfinite(sigma) or not np.isfinite(rho):
            status = BREAKDOWN
            break
        alpha = rho / sigma
        q = r - alpha * s
        if half_step:
            qn = np.sqrt(_dot(q, q)) / bnorm
            if qn <= tol:
                x = x + alpha * p
                hist.append(qn)
                it = i + 1
                status = OK
                break
        y = A(q)
        yy = _dot(y, y)
        qy = _dot(q, y)
        if yy == 0.0:
            x = x + alpha * p
            qn = np.sqrt(_dot(q, q)) / bnorm
            hist.append(qn)
            it = i + 1
            status = OK if qn <= tol else BREAKDOWN
            break
        omega = qy / yy
        if omega == 0.0 or not np.isfinite(omega):
            status = BREAKDOWN
            break
        x = x + alpha * p + omega * q
        r = q - omega * y
        rho_new = _dot(rhat, r)
        rr = _dot(r, r)
        hist.append(np.sqrt(rr) / bnorm)
        it = i + 1
        if hist[-1] <= tol:
            status = OK
            break
        if rho_new == 0.0 or not np.isfinite(rho_new):
            status = BREAKDOWN
            break
        beta = (alpha / omega) * (rho_new / rho)
        p = r + beta * (p - omega * s)
        rho = rho_new
    return _finish(mesh, coef, op, b, bt, x, it, hist, status)


def _finish(mesh, coef, op, b, bt, x, it, hist, status):
    def rel(res, rhs):
        nb = np.linalg.norm(rhs)
        return float(np.linalg.norm(res) / nb) if nb > 0 else float(np.linalg.norm(res))

    tr = rel(bt - mesh.apply(op, x), bt)
    tro = rel(b - mesh.apply(coef, x), b)
    return Result(x, it, np.asarray(hist, dtype=np.float64), status, tr, tro)


def true_residual(nx, ny, nz, coef, b, x):
    """``||b - A x|| / ||b||`` in float64 on the operator ``coef``."""
    r = np.asarray(b, dtype=np.float64) - stencil.apply(nx, ny, nz, coef, x)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(r) / nb) if nb > 0 else float(np.linalg.norm(r))


def true_residual9(nx, ny, coef, b, x):
    """:func:`true_residual` for the 2D 9-point operator."""
    r = np.asarray(b, dtype=np.float64) - stencil9.apply(nx, ny, coef, x)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(r) / nb) if nb > 0 else float(np.linalg.norm(r))


def _rho_next(rho, alpha, sigma, omega, ry):
    """(r0, r_{i+1}) from (r0, r_i), (r0, s_i), (r0, y_i) and the step's scalars."""
    return rho - alpha * sigma - omega * ry


def bicgstab_merged(nx, ny, nz, coef, b, x0=None, tol=1e-8, maxit=500, jacobi=True,
                    storage="f64"):
    """Algorithm 1 with two reduction phases per step instead of three.

    In exact arithmetic this produces the iterates of :func:`bicgstab`.  The
    inner product (r0, r_{i+1}) that defines beta_i is not reduced from
    r_{i+1}; it follows from the quantities of the step, since
    r_{i+1} = r_i - alpha_i s_i - omega_i y_i:

        (r0, r_{i+1}) = (r0, r_i) - alpha_i (r0, s_i) - omega_i (r0, y_i)

    so beta_i is known as soon as omega_i's reduction, which now also sums
    (r0, y_i), is done.  Then the x and r updates of step i and the p update
    and SpMV s_{i+1} = A p_{i+1} of step i+1 form one pass over the mesh,
    which also reduces (r0, s_{i+1}), (r_{i+1}, r_{i+1}) (the stopping rule
    of :func:`bicgstab`) and (r0, r_{i+1}) directly.  The recurrence value
    only predicts beta_i; alpha_{i+1} and the next prediction start from the
    directly reduced (r0, r_{i+1}), so rounding in the recurrence does not
    accumulate from step to step (carried alone, it stalls float32 solves).
    Breakdown readings as in :func:`bicgstab`, on the direct value.
    """
    return _bicgstab_merged(_Mesh3(nx, ny, nz), coef, b, x0, tol, maxit, jacobi, storage)


def bicgstab9_merged(nx, ny, coef, b, x0=None, tol=1e-8, maxit=500, jacobi=True,
                     storage="f64"):
    """:func:`bicgstab_merged` on the 2D 9-point operator."""
    return _bicgstab_merged(_Mesh9(nx, ny), coef, b, x0, tol, maxit, jacobi, storage)


def _bicgstab_merged(mesh, coef, b, x0, tol, maxit, jacobi, storage):
    b = np.asarray(b, dtype=np.float64)
    n = b.size
    op, bt = mesh.system(coef, b, jacobi, storage)

    def A(v):
        return mesh.apply(op, v)

    x = np.zeros(n) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    bnorm = np.sqrt(_dot(bt, bt))
    if bnorm == 0.0:
        return _finish(mesh, coef, op, b, bt, np.zeros(n), 0, [0.0], OK)
    r = bt - A(x)
    rhat = r.copy()
    p = r.copy()
    rho = _dot(rhat, r)
    hist = [np.sqrt(_dot(r, r)) / bnorm]
    if hist[0] <= tol:
        return _finish(mesh, coef, op, b, bt, x, 0, hist, OK)
    # first pass: s_0 = A p_0 and (r0, s_0)
    s = A(p)
    sigma = _dot(rhat, s)
    status = NOTCONV
    it = 0
    for i in range(maxit):
        if sigma == 0.0 or not np.isfinite(sigma) or not np.isfinite(rho):
            status = BREAKDOWN
            break
        alpha = rho / sigma
        # pass 1: q, y = A q, and (q, y), (y, y), (r0, y)
        q = r - alpha * s
        y = A(q)
        yy = _dot(y, y)
        qy = _dot(q, y)
        ry = _dot(rhat, y)
        if yy == 0.0:
            x = x + alpha * p
            qn = np.sqrt(_dot(q, q)) / bnorm
            hist.append(qn)
            it = i + 1
            status = OK if qn <= tol else BREAKDOWN
            break
        omega = qy / yy
        if omega == 0.0 or not np.isfinite(omega):
            status = BREAKDOWN
            break
        rho_new = _rho_next(rho, alpha, sigma, omega, ry)
        # pass 2: x, r updates of step i; p, s = A p of step i+1
        beta = (alpha / omega) * (rho_new / rho)
        x = x + alpha * p + omega * q
        r = q - omega * y
        p = r + beta * (p - omega * s)
        s = A(p)
        sigma = _dot(rhat, s)
        rr = _dot(r, r)
        rho_direct = _dot(rhat, r)
        hist.append(np.sqrt(rr) / bnorm)
        it = i + 1
        if hist[-1] <= tol:
            status = OK
            break
        if rho_direct == 0.0 or not np.isfinite(rho_direct):
            status = BREAKDOWN
            break
        rho = rho_direct
    return _finish(mesh, coef, op, b, bt, x, it, hist, status)
