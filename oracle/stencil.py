"""The 7-point stencil operator, in float64 (test infrastructure only).

The paper's system ``A x = b`` (Sec. III, Eq. 1) comes from a 7-point finite
difference stencil on an ``X x Y x Z`` mesh (Sec. IV).  Row ``i`` of ``A`` has
the main diagonal and one coefficient per axis neighbour; the six
off-diagonal vectors are named by axis and sign (Sec. IV-A, "SpMV (3D)":
``x``/``y``/``z`` with ``p`` or ``m``), so

    (A v)_i = diag_i v_i + xm_i v_{i-1}  + xp_i v_{i+1}
                         + ym_i v_{i-nx} + yp_i v_{i+nx}
                         + zm_i v_{i-nx*ny} + zp_i v_{i+nx*ny}

with a neighbour outside the mesh contributing zero (homogeneous Dirichlet
boundary).  Storage is x-fastest: ``i = x + nx*(y + ny*z)``.

Sec. IV keeps the operator scaled by its diagonal, so the diagonal is one
everywhere and only the six off-diagonals need storing; :func:`jacobi_scale` forms that operator
as ``D^-1 A`` (left scaling) and rounds the scaled values once to the storage
type.
"""

from __future__ import annotations

import numpy as np

DIRS = ("xm", "xp", "ym", "yp", "zm", "zp")
# (axis in the (z, y, x) array, offset) of each direction's neighbour
_NEIGH = {"xm": (2, -1), "xp": (2, +1), "ym": (1, -1), "yp": (1, +1),
          "zm": (0, -1), "zp": (0, +1)}


def _field(c, n):
    """A coefficient as a float64 1-D array of length n (scalars broadcast)."""
    if np.isscalar(c):
        return np.full(n, float(c), dtype=np.float64)
    a = np.asarray(c, dtype=np.float64)
    if a.shape != (n,):
        raise ValueError("coefficient length %s != %d" % (a.shape, n))
    return a


def shifted(v3, axis, off):
    """``w[idx] = v3[idx + off along axis]``, zero where that is off-mesh."""
    w = np.zeros_like(v3)
    src = [slice(None)] * 3
    dst = [slice(None)] * 3
    if off > 0:
        dst[axis] = slice(0, v3.shape[axis] - off)
        src[axis] = slice(off, None)
    else:
        dst[axis] = slice(-off, None)
        src[axis] = slice(0, v3.shape[axis] + off)
    w[tuple(dst)] = v3[tuple(src)]
    return w


def apply(nx, ny, nz, coef, v):
    """``A v`` in float64 for the operator with coefficients ``coef``.

    ``coef`` maps ``diag`` and the six directions to scalars or length-N
    arrays; a missing ``diag`` means a unit diagonal (the stored form after
    diagonal preconditioning, Sec. IV).  The sum is taken in a fixed order:
    diagonal, then xm, xp, ym, yp, zm, zp.
    """
    n = nx * ny * nz
    v3 = np.asarray(v, dtype=np.float64).reshape(nz, ny, nx)
    d = coef.get("diag", 1.0)
    out = _field(d, n).reshape(nz, ny, nx) * v3
    for name in DIRS:
        axis, off = _NEIGH[name]
        out = out + _field(coef[name], n).reshape(nz, ny, nx) * shifted(v3, axis, off)
    return out.reshape(n)


def apply_at(nx, ny, nz, coef_rows, x_at, idx):
    """Rows ``idx`` of ``A v`` in float64, one row at a time.

    ``coef_rows`` maps ``diag`` (optional: unit) and the six directions to
    the coefficients *of those rows* (arrays aligned with ``idx``); ``x_at``
    returns v at an array of linear indices.  Used on meshes too large to
    hold in float64 on the host: each sampled row needs only its own
    coefficients and seven values of v.  Returns ``(A v)[idx]`` and
    ``(|A||v|)[idx]``.
    """
    idx = np.asarray(idx, dtype=np.int64)
    x = idx % nx
    y = (idx // nx) % ny
    z = idx // (nx * ny)
    d = coef_rows.get("diag", None)
    vi = np.asarray(x_at(idx), dtype=np.float64)
    dv = np.ones(idx.shape) if d is None else np.asarray(d, dtype=np.float64)
    out = dv * vi
    mag = np.abs(dv * vi)
    steps = {"xm": (x > 0, -1), "xp": (x < nx - 1, 1), "ym": (y > 0, -nx),
             "yp": (y < ny - 1, nx), "zm": (z > 0, -nx * ny), "zp": (z < nz - 1, nx * ny)}
    for name in DIRS:
        inside, off = steps[name]
        j = np.where(inside, idx + off, idx)            # any valid index where off-mesh
        vj = np.where(inside, np.asarray(x_at(j), dtype=np.float64), 0.0)
        c = np.asarray(coef_rows[name], dtype=np.float64)
        out = out + c * vj
        mag = mag + np.abs(c * vj)
    return out, mag


def abs_apply(nx, ny, nz, coef, v):
    """``|A| |v|`` (elementwise magnitudes): the scale of each row's sum.

    Used as the denominator of the per-row relative error of an SpMV,
    ``|y_gpu - y_ref|_i / (|A||v|)_i``, which stays meaningful where
    ``(A v)_i`` cancels to nearly zero.
    """
    a = {k: (abs(c) if np.isscalar(c) else np.abs(np.asarray(c, dtype=np.float64)))
         for k, c in coef.items()}
    return apply(nx, ny, nz, a, np.abs(np.asarray(v, dtype=np.float64)))


# ---------------------------------------------------------------------------
# rounding to storage types (round to nearest, ties to even)
# ---------------------------------------------------------------------------

def _round_bits(x, mant_bits, emin):
    """Round float64 ``x`` to a binary format with ``mant_bits`` significant
    bits and minimum normal exponent ``emin`` (values as ``m * 2**e`` with
    ``0.5 <= |m| < 1``), ties to even, subnormals on a fixed grid below the
    normal range.  Overflow is not handled (inputs here are O(1))."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)
    # below the normal range the grid spacing stops shrinking
    e = np.maximum(e, emin)
    scale = np.ldexp(1.0, (mant_bits - e).astype(np.int64))
    return np.rint(x * scale) / scale          # x*scale and /scale are exact


def round_to(x, storage):
    """Round float64 values once to ``storage`` ('f64','f32','bf16','f16')."""
    x = np.asarray(x, dtype=np.float64)
    if storage == "f64":
        return x.copy()
    if storage == "f32":
        return x.astype(np.float32).astype(np.float64)
    if storage == "f16":
        # binary16: 11 significant bits, smallest normal 2**-14 (= 0.5 * 2**-13)
        return _round_bits(x, 11, -13)
    if storage == "bf16":
        # bfloat16: 8 significant bits, exponent range of binary32
        return _round_bits(x, 8, -125)
    raise ValueError(storage)


def jacobi_scale(nx, ny, nz, coef, storage="f64"):
    """Diagonal preconditioning to a unit main diagonal (Sec. IV).

    Left scaling: ``A~ = D^-1 A`` with ``D = diag(A)``; each off-diagonal is
    divided by its row's diagonal in float64 and rounded once to the storage
    type.  Returns the six scaled off-diagonals (``diag`` omitted = unit).
    Constant coefficients stay constant.  The right-hand side is scaled by
    the caller as ``b~ = D^-1 b`` (see :func:`scale_rhs`).
    """
    n = nx * ny * nz
    d = coef["diag"]
    out = {}
    for name in DIRS:
        c = coef[name]
        if np.isscalar(c) and np.isscalar(d):
            out[name] = float(round_to(np.float64(c) / np.float64(d), storage))
        else:
            out[name] = round_to(_field(c, n) / _field(d, n), storage)
    return out


def scale_rhs(nx, ny, nz, coef, b):
    """``D^-1 b`` in float64 (no rounding)."""
    n = nx * ny * nz
    return np.asarray(b, dtype=np.float64) / _field(coef["diag"], n)


def rounded(nx, ny, nz, coef, storage):
    """The raw operator with every coefficient rounded to ``storage``."""
    out = {}
    for k, c in coef.items():
        out[k] = float(round_to(np.float64(c), storage)) if np.isscalar(c) else round_to(c, storage)
    return out


# ---------------------------------------------------------------------------
# dense assembly and transpose (small meshes only)
# ---------------------------------------------------------------------------

def assemble_dense(nx, ny, nz, coef):
    """The N x N matrix, entry by entry with plain loops (N <= a few 1000)."""
    n = nx * ny * nz
    f = {k: _field(c, n) for k, c in coef.items()}
    diag = f.get("diag", np.ones(n))
    a = np.zeros((n, n))
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                i = x + nx * (y + ny * z)
                a[i, i] = diag[i]
                if x > 0:
                    a[i, i - 1] = f["xm"][i]
                if x < nx - 1:
                    a[i, i + 1] = f["xp"][i]
                if y > 0:
                    a[i, i - nx] = f["ym"][i]
                if y < ny - 1:
                    a[i, i + nx] = f["yp"][i]
                if z > 0:
                    a[i, i - nx * ny] = f["zm"][i]
                if z < nz - 1:
                    a[i, i + nx * ny] = f["zp"][i]
    return a


def transpose_coef(nx, ny, nz, coef):
    """Diagonals of ``A^T``, built directly from the stencil.

    ``(A^T)_{i,j} = A_{j,i}``: the plus-x entry of row ``i`` of ``A^T`` is the
    minus-x entry of row ``i+1`` of ``A`` (and so on per axis).  Entries whose
    neighbour is off-mesh multiply zero, so they are set to zero here.
    """
    n = nx * ny * nz
    f = {k: _field(c, n).reshape(nz, ny, nx) for k, c in coef.items()}
    out = {"diag": f.get("diag", np.ones((nz, ny, nx))).reshape(n).copy()}
    pairs = {"xp": ("xm", 2), "xm": ("xp", 2), "yp": ("ym", 1), "ym": ("yp", 1),
             "zp": ("zm", 0), "zm": ("zp", 0)}
    for name, (src, axis) in pairs.items():
        off = +1 if name.endswith("p") else -1
        out[name] = shifted(f[src], axis, off).reshape(n)
    return out
