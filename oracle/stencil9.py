"""The 2D 9-point stencil operator, in float64 (test infrastructure only).

Sec. IV-A ("SpMV (2D)") treats ``u = A v`` for a 9-point stencil on an
``X x Y`` mesh: row ``i`` of ``A`` couples cell ``(x, y)`` with itself, its
four axis neighbours and its four diagonal neighbours.  The off-diagonals
are named by the sign of the x and y offsets of the neighbour:

    (A v)_i = diag_i v_i + xm_i v_{i-1} + xp_i v_{i+1}
                         + ym_i v_{i-nx} + yp_i v_{i+nx}
                         + xmym_i v_{i-1-nx} + xpym_i v_{i+1-nx}
                         + xmyp_i v_{i-1+nx} + xpyp_i v_{i+1+nx}

with a neighbour outside the mesh contributing zero (homogeneous Dirichlet
boundary).  Storage is x-fastest: ``i = x + nx*y``.

The paper's mapping keeps, per core, the *columns* of ``A`` that belong to
its cells and scatters the products into an output halo that neighbouring
cores add up (Sec. IV-A).  :func:`apply_columns` is that formulation,
written independently of the row (gather) form :func:`apply`; the column of
cell ``j`` in direction ``e`` holds ``A_{j+e, j}``, the factor by which
``v_j`` enters ``u_{j+e}``.

Diagonal preconditioning (Sec. IV: unit main diagonal) is the same left
scaling ``D^-1 A`` as for the 3D operator, rounded once to storage.
"""

from __future__ import annotations

import numpy as np

from .stencil import _field, round_to

DIRS = ("xm", "xp", "ym", "yp", "xmym", "xpym", "xmyp", "xpyp")
# (dx, dy) of each direction's neighbour
OFFS = {"xm": (-1, 0), "xp": (1, 0), "ym": (0, -1), "yp": (0, 1),
        "xmym": (-1, -1), "xpym": (1, -1), "xmyp": (-1, 1), "xpyp": (1, 1)}
# the direction with the opposite offset
OPPOSITE = {d: next(e for e, o in OFFS.items() if o == (-dx, -dy))
            for d, (dx, dy) in OFFS.items()}


def shifted(v2, dx, dy):
    """``w[y, x] = v2[y + dy, x + dx]``, zero where that is off-mesh."""
    ny, nx = v2.shape
    w = np.zeros_like(v2)
    ys = slice(max(0, -dy), ny - max(0, dy))
    xs = slice(max(0, -dx), nx - max(0, dx))
    ysrc = slice(max(0, dy), ny + min(0, dy))
    xsrc = slice(max(0, dx), nx + min(0, dx))
    w[ys, xs] = v2[ysrc, xsrc]
    return w


def apply(nx, ny, coef, v):
    """``A v`` in float64 (row form).  ``coef`` maps ``diag`` (optional: unit)
    and the eight directions to scalars or length-N arrays; the sum is taken
    in the order diagonal, xm, xp, ym, yp, xmym, xpym, xmyp, xpyp."""
    n = nx * ny
    v2 = np.asarray(v, dtype=np.float64).reshape(ny, nx)
    out = _field(coef.get("diag", 1.0), n).reshape(ny, nx) * v2
    for name in DIRS:
        dx, dy = OFFS[name]
        out = out + _field(coef[name], n).reshape(ny, nx) * shifted(v2, dx, dy)
    return out.reshape(n)


def apply_columns(nx, ny, cols, v):
    """``A v`` from the columns of ``A`` (the paper's 2D formulation).

    Every cell ``j`` forms the products ``cols[e][j] * v_j`` and sends each to
    the output of its neighbour ``j + e``; products whose target is off-mesh
    are dropped, and each output sums what it receives.  Written as a loop
    over directions, each a scatter into the output array.
    """
    n = nx * ny
    v2 = np.asarray(v, dtype=np.float64).reshape(ny, nx)
    out = _field(cols.get("diag", 1.0), n).reshape(ny, nx) * v2
    for name in DIRS:
        dx, dy = OFFS[name]
        prod = _field(cols[name], n).reshape(ny, nx) * v2     # sent from cell j
        # received by cell j + (dx, dy)
        ys = slice(max(0, dy), ny + min(0, dy))
        xs = slice(max(0, dx), nx + min(0, dx))
        ysrc = slice(max(0, -dy), ny - max(0, dy))
        xsrc = slice(max(0, -dx), nx - max(0, dx))
        out[ys, xs] += prod[ysrc, xsrc]
    return out.reshape(n)


def rows_to_columns(nx, ny, coef):
    """Column storage of the operator given by rows: ``cols[e][j] =
    A_{j+e, j}``, zero where ``j + e`` is off-mesh.  The columns of ``A`` are
    the rows of ``A^T``, so this is :func:`transpose_coef`."""
    return transpose_coef(nx, ny, coef)


def apply_at(nx, ny, coef_rows, x_at, idx):
    """Rows ``idx`` of ``A v`` (and of ``|A||v|``) one row at a time, from the
    coefficients of those rows and nine values of v each (see the 3D
    ``stencil.apply_at``)."""
    idx = np.asarray(idx, dtype=np.int64)
    x = idx % nx
    y = idx // nx
    d = coef_rows.get("diag", None)
    vi = np.asarray(x_at(idx), dtype=np.float64)
    dv = np.ones(idx.shape) if d is None else np.asarray(d, dtype=np.float64)
    out = dv * vi
    mag = np.abs(dv * vi)
    for name in DIRS:
        dx, dy = OFFS[name]
        inside = (x + dx >= 0) & (x + dx < nx) & (y + dy >= 0) & (y + dy < ny)
        j = np.where(inside, idx + dx + nx * dy, idx)
        vj = np.where(inside, np.asarray(x_at(j), dtype=np.float64), 0.0)
        c = np.asarray(coef_rows[name], dtype=np.float64)
        out = out + c * vj
        mag = mag + np.abs(c * vj)
    return out, mag


def abs_apply(nx, ny, coef, v):
    """``|A| |v|``: the scale of each row's sum (per-row SpMV error metric)."""
    a = {k: (abs(c) if np.isscalar(c) else np.abs(np.asarray(c, dtype=np.float64)))
         for k, c in coef.items()}
    return apply(nx, ny, a, np.abs(np.asarray(v, dtype=np.float64)))


def jacobi_scale(nx, ny, coef, storage="f64"):
    """``D^-1 A`` (left scaling to a unit diagonal, Sec. IV), each scaled
    off-diagonal rounded once to ``storage``; ``diag`` omitted (= unit)."""
    n = nx * ny
    d = _field(coef["diag"], n)
    return {name: round_to(_field(coef[name], n) / d, storage) for name in DIRS}


def scale_rhs(nx, ny, coef, b):
    """``D^-1 b`` in float64."""
    return np.asarray(b, dtype=np.float64) / _field(coef["diag"], nx * ny)


def rounded(nx, ny, coef, storage):
    """The raw operator with every coefficient rounded to ``storage``."""
    n = nx * ny
    return {k: round_to(_field(c, n), storage) for k, c in coef.items()}


def assemble_dense(nx, ny, coef):
    """The N x N matrix, entry by entry with plain loops (N <= a few 1000)."""
    n = nx * ny
    f = {k: _field(c, n) for k, c in coef.items()}
    diag = f.get("diag", np.ones(n))
    a = np.zeros((n, n))
    for y in range(ny):
        for x in range(nx):
            i = x + nx * y
            a[i, i] = diag[i]
            for name in DIRS:
                dx, dy = OFFS[name]
                if 0 <= x + dx < nx and 0 <= y + dy < ny:
                    a[i, i + dx + nx * dy] = f[name][i]
    return a


def transpose_coef(nx, ny, coef):
    """Rows of ``A^T`` built from the stencil: the entry of row ``i`` of
    ``A^T`` towards ``i+e`` is the entry of row ``i+e`` of ``A`` towards
    ``i`` (direction ``-e``); off-mesh entries are zero."""
    n = nx * ny
    out = {"diag": _field(coef.get("diag", 1.0), n).copy()}
    for name in DIRS:
        dx, dy = OFFS[name]
        src = _field(coef[OPPOSITE[name]], n).reshape(ny, nx)
        out[name] = shifted(src, dx, dy).reshape(n)
    return out
