"""Algorithm 1 with float32 vectors and float32 sums (test infrastructure only).

A float32 BiCGStab solve (Algorithm 1, Sec. III) does not follow the float64
iteration step for step: every vector it keeps is rounded to float32, every
stencil row and inner-product partial is summed in float32, and BiCGStab
amplifies those roundings.  Its step count to a tolerance therefore differs
from the float64 oracle's, and it depends on the *order* in which the sums
are rounded -- something no two correct implementations need share.

:func:`bicgstab_f32` runs Algorithm 1 (with the stopping rule and the
readings of :mod:`oracle.bicgstab`) under such a float32 rounding model, with
the summation order chosen by ``order``:

* the iterate ``x`` and the vectors ``r, p, s, q, y`` are held in float32;
  each vector update ``u + c v`` (and the nested ``r + beta (p - omega s)``)
  is formed exactly in float64 from float32 operands and rounded once to
  float32 per multiply-add;
* a stencil row ``(A v)_i`` starts from the diagonal term and adds the six
  neighbour terms in an order drawn from ``order``, rounding to float32
  after each addition;
* an inner product forms the float64 products of float32 values, rounds
  them to float32 and sums them in float32 over runs of 32 consecutive
  entries of a permutation drawn from ``order``; the run sums are added in
  float64.  The scalars alpha, omega, beta are float64 quotients of those
  sums, rounded to float32 where they multiply a vector.

It is a model of rounding, not a reference for values: the tests use the
spread of its step counts over several orders to bound the step count of a
float32 solve, while values are compared with :func:`oracle.bicgstab.bicgstab`.
"""

from __future__ import annotations

import numpy as np

from . import stencil
from .bicgstab import BREAKDOWN, NOTCONV, OK, Result

_F = np.float32
_RUN = 32


def _r32(a):
    return np.asarray(a, dtype=np.float64).astype(_F)


def _fma32(a, b, c):
    """round32(a * b + c) for float32 operands (the product is exact in float64)."""
    return _r32(np.float64(a) * np.asarray(b, dtype=np.float64) + np.asarray(c, dtype=np.float64))


class _Model:
    def __init__(self, nx, ny, nz, op, order):
        self.dims = (nx, ny, nz)
        self.n = nx * ny * nz
        rng = np.random.default_rng(order)
        self.dir_order = [stencil.DIRS[k] for k in rng.permutation(len(stencil.DIRS))]
        self.perm = rng.permutation(self.n)
        self.op = {k: (np.full(self.n, v, dtype=_F) if np.isscalar(v) else _r32(v))
                   for k, v in op.items()}

    def apply(self, v):
        nx, ny, nz = self.dims
        v3 = np.asarray(v, dtype=_F).reshape(nz, ny, nx)
        d = self.op.get("diag")
        acc = v3.reshape(-1).astype(_F) if d is None else _r32(d.astype(np.float64) * v3.reshape(-1))
        for name in self.dir_order:
            axis, off = stencil._NEIGH[name]
            nb = stencil.shifted(v3, axis, off).reshape(-1)
            acc = _fma32(1.0, self.op[name].astype(np.float64) * nb.astype(np.float64), acc)
        return acc

    def dot(self, a, b):
        pr = _r32(np.asarray(a, np.float64) * np.asarray(b, np.float64))[self.perm]
        k = pr.size // _RUN * _RUN
        run = np.zeros(k // _RUN, dtype=_F)
        blk = pr[:k].reshape(-1, _RUN)
        for j in range(_RUN):
            run = (run + blk[:, j]).astype(_F)
        return float(run.astype(np.float64).sum() + pr[k:].astype(np.float64).sum())


def bicgstab_f32(nx, ny, nz, coef, b, tol=1e-6, maxit=500, order=0, storage="f32"):
    """Algorithm 1 on the Jacobi-scaled system rounded to ``storage``, with
    float32 vectors and float32 sums in the order chosen by ``order`` (an
    integer seed).  Returns a :class:`oracle.bicgstab.Result` (``x`` as
    float64 holding float32 values; true residuals in float64)."""
    b = np.asarray(b, dtype=np.float64)
    op = stencil.jacobi_scale(nx, ny, nz, coef, storage)
    bt = stencil.scale_rhs(nx, ny, nz, coef, b)
    m = _Model(nx, ny, nz, op, order)
    n = m.n
    x = np.zeros(n, dtype=_F)
    r = _r32(bt)
    bnorm = np.sqrt(m.dot(r, r))
    if bnorm == 0.0:
        return _finish(nx, ny, nz, coef, op, b, bt, x, 0, [0.0], OK)
    rhat = r.copy()
    p = r.copy()
    rho = m.dot(rhat, r)
    hist = [np.sqrt(m.dot(r, r)) / bnorm]
    if hist[0] <= tol:
        return _finish(nx, ny, nz, coef, op, b, bt, x, 0, hist, OK)
    status, it = NOTCONV, 0
    for i in range(maxit):
        s = m.apply(p)
        sigma = m.dot(rhat, s)
        if sigma == 0.0 or not np.isfinite(sigma):
            status = BREAKDOWN
            break
        alpha = rho / sigma
        q = _fma32(-_F(alpha), s, r)
        y = m.apply(q)
        yy, qy = m.dot(y, y), m.dot(q, y)
        if yy == 0.0:
            x = _fma32(_F(alpha), p, x)
            hist.append(np.sqrt(m.dot(q, q)) / bnorm)
            it = i + 1
            status = OK if hist[-1] <= tol else BREAKDOWN
            break
        omega = qy / yy
        if omega == 0.0 or not np.isfinite(omega):
            status = BREAKDOWN
            break
        x = _fma32(_F(omega), q, _fma32(_F(alpha), p, x))
        r = _fma32(-_F(omega), y, q)
        rho_new = m.dot(rhat, r)
        hist.append(np.sqrt(m.dot(r, r)) / bnorm)
        it = i + 1
        if hist[-1] <= tol:
            status = OK
            break
        if rho_new == 0.0 or not np.isfinite(rho_new):
            status = BREAKDOWN
            break
        beta = (alpha / omega) * (rho_new / rho)
        p = _fma32(_F(beta), _fma32(-_F(omega), s, p), r)
        rho = rho_new
    return _finish(nx, ny, nz, coef, op, b, bt, x, it, hist, status)


def _finish(nx, ny, nz, coef, op, b, bt, x, it, hist, status):
    x = x.astype(np.float64)

    def rel(res, rhs):
        nb = np.linalg.norm(rhs)
        return float(np.linalg.norm(res) / nb) if nb > 0 else float(np.linalg.norm(res))

    tr = rel(bt - stencil.apply(nx, ny, nz, op, x), bt)
    tro = rel(b - stencil.apply(nx, ny, nz, coef, x), b)
    return Result(x, it, np.asarray(hist, dtype=np.float64), status, tr, tro)


def step_range(nx, ny, nz, coef, b, tol, maxit=1000, orders=6, storage="f32"):
    """(min, max) step count of :func:`bicgstab_f32` over ``orders`` summation
    orders (seeds 0 .. orders-1)."""
    its = [bicgstab_f32(nx, ny, nz, coef, b, tol=tol, maxit=maxit, order=k, storage=storage).iters
           for k in range(orders)]
    return min(its), max(its)
