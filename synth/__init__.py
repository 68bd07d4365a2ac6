"""Seeded synthetic problem generator for the stencil systems (3D 7-point
and 2D 9-point).

This module is shared by the CPU oracle and by the GPU path's tests and
benchmark.  It produces *inputs only*: raw (unscaled) stencil coefficients,
right-hand sides, mesh sizes and request streams.  It holds none of the
solver's arithmetic -- no operator application, no Jacobi scaling, no Krylov
step -- so the two sides that it feeds stay independent.

Random numbers come from SplitMix64 (G. L. Steele, D. Lea, C. H. Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014) used as a
counter-based generator: the value at counter ``i`` of stream ``s`` under seed
``k`` is the SplitMix64 output function applied to ``key(k, s) + (i+1)*GAMMA``.
Any single value can therefore be regenerated on its own, which is what the
full-size sampled parity checks rely on.

Layout convention (the same everywhere in the project): a mesh of
``nx*ny*nz`` cells is stored x-fastest, linear index ``i = x + nx*(y + ny*z)``.
Coefficient direction order is ``xm, xp, ym, yp, zm, zp`` (the neighbour at
``x-1``, ``x+1``, ``y-1``, ``y+1``, ``z-1``, ``z+1``), following the paper's
naming of the six off-diagonal vectors by coordinate direction and
plus/minus (Sec. IV-A, "SpMV (3D)").  The 2D 9-point systems (Sec. IV-A,
"SpMV (2D)") live on an ``nx*ny`` mesh (``nz = 1``, ``i = x + nx*y``) with the
eight directions ``xm, xp, ym, yp, xmym, xpym, xmyp, xpyp`` (``DIRS9``: the
sign of the neighbour's x and y offsets).
"""

from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_TWO_M53 = float(2.0 ** -53)

DIRS = ("xm", "xp", "ym", "yp", "zm", "zp")
DIRS9 = ("xm", "xp", "ym", "yp", "xmym", "xpym", "xmyp", "xpyp")

# Stream numbers inside one seed.
STREAM_COEF = 0      # coefficient arrays (6 directions, then the diagonal margin)
STREAM_RHS = 1       # right-hand side
STREAM_SIZES = 2     # batched / served mesh sizes, tolerances, arrivals


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (the 'mix64' finaliser), on uint64 arrays."""
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _mix_scalar(v: int) -> int:
    with np.errstate(over="ignore"):
        return int(_mix(np.array([v & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0])


def stream_key(seed: int, stream: int) -> np.uint64:
    """Start state of stream ``stream`` under ``seed`` (both mixed once)."""
    return np.uint64(_mix_scalar(seed ^ _mix_scalar(stream + 0x632BE59BD9B4E019)))


_INNER = 1 << 16


def _mix_inplace(z: np.ndarray, t: np.ndarray) -> np.ndarray:
    """:func:`_mix` computed in place (``t`` is scratch of the same shape)."""
    for shift, mul in ((30, _M1), (27, _M2), (31, None)):
        np.right_shift(z, np.uint64(shift), out=t)
        np.bitwise_xor(z, t, out=z)
        if mul is not None:
            np.multiply(z, mul, out=z)
    return z


def raw_u64(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Counters ``start .. start+count-1`` of a stream, as raw 64-bit words."""
    key = stream_key(seed, stream)
    out = np.empty(count, dtype=np.uint64)
    m = min(_INNER, count)
    t = np.empty(m, dtype=np.uint64)
    base = np.arange(1, m + 1, dtype=np.uint64) * GAMMA
    with np.errstate(over="ignore"):
        for s in range(0, count, m):
            c = min(m, count - s)
            z = out[s:s + c]
            np.add(base[:c], key + np.uint64(start + s) * GAMMA, out=z)
            _mix_inplace(z, t[:c])
    return out


def uniform(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """U[0,1) doubles with 53 random bits: ``(word >> 11) * 2**-53``."""
    w = raw_u64(seed, stream, start, count)
    np.right_shift(w, np.uint64(11), out=w)
    u = w.astype(np.float64)
    u *= _TWO_M53
    return u


def uniform_at(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """U[0,1) at arbitrary counters ``idx`` (for sampled checks)."""
    key = stream_key(seed, stream)
    ctr = np.asarray(idx, dtype=np.uint64) + np.uint64(1)
    with np.errstate(over="ignore"):
        w = _mix(key + ctr * GAMMA)
    return (w >> np.uint64(11)).astype(np.float64) * _TWO_M53


# ---------------------------------------------------------------------------
# chunked, threaded fill for large meshes (numpy releases the GIL)
# ---------------------------------------------------------------------------

_CHUNK = 1 << 22


def _threads() -> int:
    return max(1, min(32, os.cpu_count() or 1))


def _fill(out: np.ndarray, fn) -> np.ndarray:
    """Fill ``out`` (1-D) chunk by chunk with ``fn(start, count)``."""
    n = out.shape[0]
    starts = list(range(0, n, _CHUNK))

    def work(s):
        c = min(_CHUNK, n - s)
        out[s:s + c] = fn(s, c)

    if len(starts) <= 1:
        for s in starts:
            work(s)
    else:
        with ThreadPoolExecutor(_threads()) as ex:
            list(ex.map(work, starts))
    return out


# ---------------------------------------------------------------------------
# problem recipes
# ---------------------------------------------------------------------------

@dataclass
class Problem:
    """One linear system ``A x = b`` on an ``nx*ny*nz`` mesh (raw, unscaled).

    ``coef`` maps ``diag`` and the six directions to either a 1-D array of
    ``n`` values (per-cell coefficients) or a Python float (constant
    coefficients).  Arrays are already rounded to ``dtype`` (the storage type
    of the raw inputs: ``float64`` or ``float32``).  ``b`` is a 1-D array.
    Off-diagonals that point outside the mesh are present in the arrays (they
    multiply the zero Dirichlet value), so the value distribution does not
    depend on the cell's position.
    """

    nx: int
    ny: int
    nz: int
    coef: dict
    b: np.ndarray
    constant: bool
    seed: int
    recipe: str
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz


def _as_dtype(a, dtype):
    return np.asarray(a, dtype=np.float64).astype(dtype)


def convdiff_constant(nx, ny, nz, seed=0, dtype=np.float64) -> Problem:
    """Constant-coefficient convection-diffusion operator.

    ``c_d ~ U[0,0.3]`` once per axis d; minus-side coefficient ``-1 - c_d``,
    plus-side ``-1 + c_d``, diagonal ``6.1``; ``b ~ U[-1,1]``.  Off-diagonal
    magnitudes sum to 6 < 6.1, so A is strictly diagonally dominant.
    """
    c = 0.3 * uniform(seed, STREAM_COEF, 0, 3)
    coef = {"diag": 6.1}
    for a, ax in enumerate("xyz"):
        coef[ax + "m"] = float(np.float64(-1.0 - c[a]).astype(dtype))
        coef[ax + "p"] = float(np.float64(-1.0 + c[a]).astype(dtype))
    coef["diag"] = float(np.float64(6.1).astype(dtype))
    n = nx * ny * nz
    b = np.empty(n, dtype=dtype)
    _fill(b, lambda s, k: (2.0 * uniform(seed, STREAM_RHS, s, k) - 1.0).astype(dtype))
    return Problem(nx, ny, nz, coef, b, True, seed, "convdiff_constant",
                   {"c": c.tolist()})


def laplacian(nx, ny, nz, dtype=np.float64, b=None) -> Problem:
    """The 7-point Dirichlet Laplacian: diagonal 6, off-diagonals -1."""
    coef = {"diag": 6.0}
    for d in DIRS:
        coef[d] = -1.0
    n = nx * ny * nz
    if b is None:
        b = np.zeros(n, dtype=dtype)
    return Problem(nx, ny, nz, coef, np.asarray(b, dtype=dtype), True, 0, "laplacian")


def _offdiag_chunk(seed, k, n, s, c, dtype):
    # direction k occupies counters [k*n, (k+1)*n) of the coefficient stream
    return _as_dtype(-(0.5 + uniform(seed, STREAM_COEF, k * n + s, c)), dtype)


def _normal_chunk(seed, stream, s, c):
    """Box-Muller on the counter pair (2i, 2i+1); cosine branch only."""
    u = uniform(seed, stream, 2 * s, 2 * c)
    u1 = 1.0 - u[0::2]          # (0, 1]: log is finite
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def varcoef(nx, ny, nz, seed=0, dtype=np.float32, rhs="normal") -> Problem:
    """Per-cell variable coefficients, diagonally dominant and nonsymmetric.

    Off-diagonals ``-U[0.5,1.5]`` independently per cell and direction; the
    diagonal is ``sum |off| + U[0.01,0.1]`` (the sum over the six rounded
    off-diagonals, in float64, then rounded once).  With all off-diagonals
    negative and strict dominance, A is a nonsingular M-matrix.
    ``b ~ N(0,1)`` (Box-Muller) or ``U[-1,1]``.
    """
    n = nx * ny * nz
    coef = {}
    for k, d in enumerate(DIRS):
        arr = np.empty(n, dtype=dtype)
        coef[d] = _fill(arr, lambda s, c, k=k: _offdiag_chunk(seed, k, n, s, c, dtype))
    diag = np.empty(n, dtype=dtype)

    def diag_chunk(s, c):
        acc = np.zeros(c, dtype=np.float64)
        for d in DIRS:
            acc += np.abs(coef[d][s:s + c].astype(np.float64))
        acc += 0.01 + 0.09 * uniform(seed, STREAM_COEF, 6 * n + s, c)
        return acc.astype(dtype)

    coef["diag"] = _fill(diag, diag_chunk)
    b = np.empty(n, dtype=dtype)
    if rhs == "normal":
        _fill(b, lambda s, c: _normal_chunk(seed, STREAM_RHS, s, c).astype(dtype))
    else:
        _fill(b, lambda s, c: (2.0 * uniform(seed, STREAM_RHS, s, c) - 1.0).astype(dtype))
    return Problem(nx, ny, nz, coef, b, False, seed, "varcoef")


def varcoef_at(nx, ny, nz, idx, seed=0, dtype=np.float32):
    """Coefficients and b of :func:`varcoef` at cells ``idx`` only.

    Returns ``(coef, b)`` with the same values, bit for bit, as the full
    generator at those cells (used by sampled checks on meshes too large to
    generate on the host twice).
    """
    idx = np.asarray(idx, dtype=np.int64)
    n = nx * ny * nz
    coef = {}
    acc = np.zeros(idx.shape, dtype=np.float64)
    for k, d in enumerate(DIRS):
        v = _as_dtype(-(0.5 + uniform_at(seed, STREAM_COEF, k * n + idx)), dtype)
        coef[d] = v
        acc += np.abs(v.astype(np.float64))
    acc += 0.01 + 0.09 * uniform_at(seed, STREAM_COEF, 6 * n + idx)
    coef["diag"] = acc.astype(dtype)
    u1 = 1.0 - uniform_at(seed, STREAM_RHS, 2 * idx)
    u2 = uniform_at(seed, STREAM_RHS, 2 * idx + 1)
    b = (np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)).astype(dtype)
    return coef, b


def varcoef9(nx, ny, seed=0, dtype=np.float32, rhs="normal") -> Problem:
    """The 2D 9-point analogue of :func:`varcoef`: off-diagonals
    ``-U[0.5,1.5]`` per cell and direction (``DIRS9``), diagonal ``sum |off|
    + U[0.01,0.1]``, ``b ~ N(0,1)`` or ``U[-1,1]``.  Direction k of the
    coefficient stream occupies counters ``[k*n, (k+1)*n)``, the diagonal
    margin ``[8n, 9n)``."""
    n = nx * ny
    coef = {}
    for k, d in enumerate(DIRS9):
        arr = np.empty(n, dtype=dtype)
        coef[d] = _fill(arr, lambda s, c, k=k: _offdiag_chunk(seed, k, n, s, c, dtype))
    diag = np.empty(n, dtype=dtype)

    def diag_chunk(s, c):
        acc = np.zeros(c, dtype=np.float64)
        for d in DIRS9:
            acc += np.abs(coef[d][s:s + c].astype(np.float64))
        acc += 0.01 + 0.09 * uniform(seed, STREAM_COEF, 8 * n + s, c)
        return acc.astype(dtype)

    coef["diag"] = _fill(diag, diag_chunk)
    b = np.empty(n, dtype=dtype)
    if rhs == "normal":
        _fill(b, lambda s, c: _normal_chunk(seed, STREAM_RHS, s, c).astype(dtype))
    else:
        _fill(b, lambda s, c: (2.0 * uniform(seed, STREAM_RHS, s, c) - 1.0).astype(dtype))
    return Problem(nx, ny, 1, coef, b, False, seed, "varcoef9")


def varcoef9_at(nx, ny, idx, seed=0, dtype=np.float32):
    """Coefficients and b of :func:`varcoef9` at cells ``idx`` only (bit for
    bit the full generator's values)."""
    idx = np.asarray(idx, dtype=np.int64)
    n = nx * ny
    coef = {}
    acc = np.zeros(idx.shape, dtype=np.float64)
    for k, d in enumerate(DIRS9):
        v = _as_dtype(-(0.5 + uniform_at(seed, STREAM_COEF, k * n + idx)), dtype)
        coef[d] = v
        acc += np.abs(v.astype(np.float64))
    acc += 0.01 + 0.09 * uniform_at(seed, STREAM_COEF, 8 * n + idx)
    coef["diag"] = acc.astype(dtype)
    u1 = 1.0 - uniform_at(seed, STREAM_RHS, 2 * idx)
    u2 = uniform_at(seed, STREAM_RHS, 2 * idx + 1)
    b = (np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)).astype(dtype)
    return coef, b


def random_vector(n, seed, stream, dtype=np.float32, kind="normal"):
    """A seeded test vector (``N(0,1)`` or ``U[-1,1]``)."""
    out = np.empty(n, dtype=dtype)
    if kind == "normal":
        return _fill(out, lambda s, c: _normal_chunk(seed, stream, s, c).astype(dtype))
    return _fill(out, lambda s, c: (2.0 * uniform(seed, stream, s, c) - 1.0).astype(dtype))


def random_vector_at(idx, seed, stream, dtype=np.float32):
    """Values of ``random_vector(n, seed, stream, dtype, kind="uniform")`` at
    indices ``idx`` (bit for bit)."""
    u = uniform_at(seed, stream, np.asarray(idx, dtype=np.int64))
    return (2.0 * u - 1.0).astype(dtype)


# ---------------------------------------------------------------------------
# batched and served workloads
# ---------------------------------------------------------------------------

def batched_edges(count=512, seed=1, lo=16, hi=128):
    """Cube edges ``round(lo * (hi/lo)**u)``, ``u ~ U[0,1]`` (log-uniform)."""
    u = uniform(seed, STREAM_SIZES, 0, count)
    return [int(round(lo * (hi / lo) ** v)) for v in u]


def system_seed(base_seed: int, j: int) -> int:
    """Seed of the j-th independent system of a batch or request stream."""
    return _mix_scalar(base_seed * 0x10001 + 7919 * (j + 1)) & 0x7FFFFFFFFFFFFFFF


@dataclass
class Request:
    rid: int
    nx: int
    ny: int
    nz: int
    tol: float
    arrival: float
    seed: int


def request_stream(count=20000, rate=100.0, seed=3, lo=32, hi=384,
                   aspect=(0.5, 2.0), tols=(1e-4, 1e-6, 1e-8)):
    """Poisson arrivals of solve requests with log-uniform mesh sizes.

    Edge ``e ~ logU[lo,hi]``; ``nx = e``, ``ny = round(e*a1)``,
    ``nz = round(e*a2)`` with ``a ~ logU[aspect]``; tolerance uniform over
    ``tols``; inter-arrival times exponential with mean ``1/rate`` seconds.
    """
    u = uniform(seed, STREAM_SIZES, 0, 5 * count).reshape(count, 5)
    out = []
    t = 0.0
    alo, ahi = aspect
    for j in range(count):
        e = lo * (hi / lo) ** u[j, 0]
        a1 = alo * (ahi / alo) ** u[j, 1]
        a2 = alo * (ahi / alo) ** u[j, 2]
        tol = tols[min(len(tols) - 1, int(u[j, 3] * len(tols)))]
        t += -math.log(1.0 - u[j, 4]) / rate
        out.append(Request(j, max(1, int(round(e))), max(1, int(round(e * a1))),
                           max(1, int(round(e * a2))), tol, t, system_seed(seed, j)))
    return out
