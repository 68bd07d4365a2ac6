"""BiCGStab for 7-point stencil systems on one GB300 GPU.

Python binding of ``libstencil7.so``, whose C ABI is ``include/stencil7.h``.
The functions here carry the C names and only marshal arguments: every step
of the solve runs in the library's CUDA kernels.  Buffers may be torch
tensors (CUDA or CPU) or NumPy arrays; CUDA tensors are passed to the
library by pointer on the current torch stream, host buffers are staged by
the library.  There is no CPU fallback: if the library is not built, or no
GPU is visible, calls raise.

Layout: a mesh vector has ``nx*ny*nz`` elements, x fastest
(``i = x + nx*(y + ny*z)``).  Coefficients: ``diag`` and the six
off-diagonals ``xm, xp, ym, yp, zm, zp`` (Sec. IV-A of the paper names them by
axis and sign).  :func:`stencil9_create` builds the 2D 9-point operator of
Sec. IV-A on an ``nx*ny`` mesh (``i = x + nx*y``; directions ``DIRS9``); its
handle works with every single-system entry point.
"""

from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import _build

__all__ = [
    "S7_F64", "S7_F32", "S7_BF16", "S7_F16", "S7Error", "Operator", "lib", "EXPORTS",
    "stencil7_create", "stencil9_create", "stencil7_destroy", "stencil7_info", "stencil7_apply",
    "stencil7_residual", "stencil7_residual_noalloc", "bicgstab_solve",
    "bicgstab_solve_refined", "bicgstab_solve_batched", "bicgstab_batched_policy",
    "stencil7_profile", "s7_last_error",
    "s7_version", "Server", "s7_server_create", "s7_server_submit", "s7_server_poll",
    "s7_server_wait", "s7_server_release", "s7_server_get_stats", "s7_server_destroy",
    "s7_mem_stats", "s7_mem_trim", "s7_mem_set_cache",
]

S7_F64, S7_F32, S7_BF16, S7_F16 = 0, 1, 2, 3
OK, EINVAL, ENOMEM, EBREAKDOWN, ENOTCONV, ETIMEOUT, ECUDA, EAGAIN, ECANCELED = range(9)
STATUS_NAMES = {0: "ok", 1: "einval", 2: "enomem", 3: "breakdown", 4: "notconv",
                5: "timeout", 6: "ecuda", 7: "eagain", 8: "canceled"}
DIRS = ("xm", "xp", "ym", "yp", "zm", "zp")
DIRS9 = ("xm", "xp", "ym", "yp", "xmym", "xpym", "xmyp", "xpyp")
S9_ROWS, S9_COLUMNS = 0, 1
_STORAGE = {"f64": S7_F64, "f32": S7_F32, "bf16": S7_BF16, "f16": S7_F16}

# Entry points declared in include/stencil7.h (checked by the tests).
EXPORTS = (
    "stencil7_create", "stencil9_create", "stencil7_destroy", "stencil7_info", "stencil7_apply",
    "stencil7_residual", "stencil7_residual_noalloc", "bicgstab_solve",
    "bicgstab_solve_refined", "bicgstab_solve_batched", "bicgstab_batched_policy",
    "stencil7_profile", "s7_last_error",
    "s7_version", "s7_server_create", "s7_server_submit", "s7_server_poll", "s7_server_wait",
    "s7_server_release", "s7_server_get_stats", "s7_server_destroy", "s7_mem_stats",
    "s7_mem_trim", "s7_mem_set_cache",
)
PROF_KINDS = ("spmv_p_dot", "spmv_q_dots", "update_dots", "start_residual", "true_residual",
              "other")


class S7Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (STATUS_NAMES.get(code, "?"), code, msg))
        self.code = code


class s7_coeffs(C.Structure):
    _fields_ = [("diag", C.c_void_p), ("xm", C.c_void_p), ("xp", C.c_void_p),
                ("ym", C.c_void_p), ("yp", C.c_void_p), ("zm", C.c_void_p),
                ("zp", C.c_void_p), ("dtype", C.c_int), ("constant", C.c_int)]


class s9_coeffs(C.Structure):
    _fields_ = [("diag", C.c_void_p)] + [(k, C.c_void_p) for k in DIRS9] + \
               [("dtype", C.c_int), ("layout", C.c_int)]


class s7_opts(C.Structure):
    _fields_ = [("storage", C.c_int), ("no_jacobi", C.c_int), ("keep_true", C.c_int),
                ("bx", C.c_int), ("by", C.c_int), ("zchunk", C.c_int),
                ("check_every", C.c_int), ("stages", C.c_int), ("pipe_kinds", C.c_int),
                ("variant", C.c_int), ("step_cells", C.c_int), ("residual_f64", C.c_int),
                ("tma", C.c_int)]


class s7_batch_opts(C.Structure):
    _fields_ = [("threads", C.c_int), ("zchunk", C.c_int), ("check_every", C.c_int),
                ("no_autotune", C.c_int), ("schedule", C.c_int), ("wait_cycles", C.c_longlong),
                ("choose_variant", C.c_int)]


class s7_server_opts(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("storage", C.c_int), ("max_active", C.c_int),
                ("steps_per_tick", C.c_int), ("threads", C.c_int), ("zchunk", C.c_int),
                ("inner_tol", C.c_double), ("inner_maxit", C.c_int), ("max_outer", C.c_int),
                ("three_pass", C.c_int), ("residual_f64", C.c_int)]


class s7_request(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("coeffs", s7_coeffs),
                ("b", C.c_void_p), ("x", C.c_void_p), ("dt", C.c_int), ("tol", C.c_double)]


class s7_result(C.Structure):
    _fields_ = [("status", C.c_int), ("outer", C.c_int), ("inner_iters", C.c_int),
                ("resid", C.c_double), ("t_arrive", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double)]


class s7_server_stats(C.Structure):
    _fields_ = [("completed", C.c_longlong), ("failed", C.c_longlong), ("queued", C.c_longlong),
                ("active", C.c_longlong), ("mem_used", C.c_size_t), ("mem_peak", C.c_size_t),
                ("cell_iters", C.c_double), ("busy_s", C.c_double)]


_lib = None


def lib_path():
    return _build.LIB


def lib():
    """Load the CUDA library (it must have been built; see ``_build``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError("libstencil7.so is not built: run __graft_entry__.build() "
                           "or python -m paper_2010_03660_gb300._build")
    L = C.CDLL(path)
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    P = C.POINTER
    sig = {
        "stencil7_create": (i, [P(vp), i, i, i, P(s7_coeffs), P(s7_opts)]),
        "stencil9_create": (i, [P(vp), i, i, P(s9_coeffs), P(s7_opts)]),
        "stencil7_destroy": (i, [vp]),
        "stencil7_info": (i, [vp, P(i), P(i), P(i), P(i), P(C.c_size_t)]),
        "stencil7_apply": (i, [vp, vp, vp, i, vp]),
        "stencil7_residual": (i, [vp, vp, vp, vp, i, P(d), P(d), vp]),
        "stencil7_residual_noalloc": (i, [vp, vp, vp, vp, i, P(d), P(d), vp]),
        "bicgstab_solve": (i, [vp, vp, vp, i, d, i, P(i), P(d), P(d), vp]),
        "bicgstab_solve_refined": (i, [vp, vp, vp, d, i, i, d, P(i), P(i), P(d), vp]),
        "stencil7_profile": (i, [vp, i, P(d), P(C.c_longlong)]),
        "bicgstab_solve_batched": (i, [i, P(vp), P(vp), P(vp), i, P(d), P(i), P(i), P(i), P(d),
                                       P(s7_batch_opts), vp]),
        "bicgstab_batched_policy": (i, [P(i), P(i), P(i), P(i), P(i)]),
        "s7_server_create": (i, [P(vp), P(s7_server_opts)]),
        "s7_server_submit": (i, [vp, P(s7_request), P(C.c_uint64)]),
        "s7_server_poll": (i, [vp, C.c_uint64, P(s7_result)]),
        "s7_server_wait": (i, [vp, C.c_uint64, P(s7_result), d]),
        "s7_server_release": (i, [vp, C.c_uint64]),
        "s7_server_get_stats": (i, [vp, P(s7_server_stats)]),
        "s7_server_destroy": (i, [vp]),
        "s7_mem_stats": (i, [i, P(C.c_size_t), P(C.c_size_t)]),
        "s7_mem_trim": (i, [i, C.c_size_t]),
        "s7_mem_set_cache": (i, [C.c_size_t]),
        "s7_last_error": (C.c_char_p, []),
        "s7_version": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def s7_last_error():
    return lib().s7_last_error().decode()


def s7_version():
    return lib().s7_version().decode()


def _check(rc, allow=()):
    if rc != OK and rc not in allow:
        raise S7Error(rc, s7_last_error())
    return rc


# ---------------------------------------------------------------------------
# buffer marshalling
# ---------------------------------------------------------------------------

def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _dtype_code(a):
    if _is_torch(a):
        import torch
        m = {torch.float64: S7_F64, torch.float32: S7_F32, torch.bfloat16: S7_BF16,
             torch.float16: S7_F16}
        return m[a.dtype]
    m = {np.dtype(np.float64): S7_F64, np.dtype(np.float32): S7_F32,
         np.dtype(np.float16): S7_F16}
    return m[np.asarray(a).dtype]


def _ptr(a):
    if a is None:
        return None
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if not (isinstance(a, np.ndarray) and a.flags["C_CONTIGUOUS"]):
        raise ValueError("array must be a C-contiguous numpy array")
    return a.ctypes.data


def _stream(*bufs):
    for a in bufs:
        if a is not None and _is_torch(a) and a.is_cuda:
            import torch
            return torch.cuda.current_stream(a.device).cuda_stream
    return None


def _numel(a):
    return a.numel() if _is_torch(a) else np.asarray(a).size


def _vectors(what, n, first, *others, dtype=None):
    """Check the vectors of one call: the C entry points take a single
    element type for all of them and no sizes, so a buffer of another type
    would be read as the wrong type and a short one past its end.  Returns
    the common type code."""
    code = _dtype_code(first)
    if dtype is not None and code != dtype:
        raise ValueError("%s: vectors must be float64" % what)
    for a in (first,) + others:
        if a is None:
            continue
        if _dtype_code(a) != code:
            raise ValueError("%s: all vectors must have the same dtype" % what)
        if _numel(a) != n:
            raise ValueError("%s: a vector has %d elements, the operator %d" % (what, _numel(a), n))
    return code


def _empty_like(a, dtype_code=None):
    if _is_torch(a):
        import torch
        m = {S7_F64: torch.float64, S7_F32: torch.float32, S7_BF16: torch.bfloat16,
             S7_F16: torch.float16}
        return torch.empty(a.shape, dtype=m[dtype_code] if dtype_code is not None else a.dtype,
                           device=a.device)
    m = {S7_F64: np.float64, S7_F32: np.float32, S7_F16: np.float16}
    return np.empty(np.asarray(a).shape, dtype=m[dtype_code] if dtype_code is not None
                    else np.asarray(a).dtype)


# ---------------------------------------------------------------------------
# the operator handle
# ---------------------------------------------------------------------------

class Operator:
    """An owned ``stencil7_t`` (see :func:`stencil7_create`)."""

    def __init__(self, handle, nx, ny, nz, storage):
        self._h = C.c_void_p(handle)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.storage = storage

    @property
    def n(self):
        return self.nx * self.ny * self.nz

    @property
    def handle(self):
        if not self._h:
            raise ValueError("operator destroyed")
        return self._h

    def close(self):
        if self._h:
            lib().stencil7_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def stencil7_create(nx, ny, nz, coef, storage="f32", jacobi=True, keep_true=False,
                    bx=0, by=0, zchunk=0, check_every=0, constant=None, stages=0,
                    pipe_kinds=0, variant=0, step_cells=0, residual_f64=False, tma=False):
    """Create an operator from raw coefficients.

    ``coef`` maps ``diag, xm, xp, ym, yp, zm, zp`` to arrays/tensors of
    ``nx*ny*nz`` float32 or float64 values (all the same type), or all to
    Python floats for a constant-coefficient operator.  ``residual_f64``
    runs the float64-accuracy residual sweeps in binary64 instead of double
    words.
    """
    names = ("diag",) + DIRS
    if constant is None:
        constant = all(np.isscalar(coef[k]) for k in names)
    keep = []
    ptrs = {}
    if constant:
        raw_dt = S7_F64
        for k in names:
            a = np.array([float(coef[k])], dtype=np.float64)
            keep.append(a)
            ptrs[k] = a.ctypes.data
    else:
        raw_dt = _dtype_code(coef["diag"])
        for k in names:
            a = coef[k]
            if _numel(a) != nx * ny * nz:
                raise ValueError("coefficient %s has %d elements, expected %d"
                                 % (k, _numel(a), nx * ny * nz))
            if _dtype_code(a) != raw_dt:
                raise ValueError("all coefficients must have the same dtype")
            keep.append(a)
            ptrs[k] = _ptr(a)
    cs = s7_coeffs(ptrs["diag"], ptrs["xm"], ptrs["xp"], ptrs["ym"], ptrs["yp"],
                   ptrs["zm"], ptrs["zp"], raw_dt, 1 if constant else 0)
    st = _STORAGE[storage] if isinstance(storage, str) else int(storage)
    op = s7_opts(st, 0 if jacobi else 1, 1 if keep_true else 0, bx, by, zchunk, check_every,
                 stages, pipe_kinds, variant, step_cells, 1 if residual_f64 else 0,
                 1 if tma else 0)
    h = C.c_void_p()
    _check(lib().stencil7_create(C.byref(h), nx, ny, nz, C.byref(cs), C.byref(op)))
    del keep
    return Operator(h.value, nx, ny, nz, st)


def stencil9_create(nx, ny, coef, storage="f32", jacobi=True, keep_true=False, bx=0,
                    zchunk=0, check_every=0, variant=0, layout="rows", residual_f64=False):
    """Create a 2D 9-point operator from raw coefficients.

    ``coef`` maps ``diag`` and the eight directions of ``DIRS9`` to
    arrays/tensors of ``nx*ny`` float32 or float64 values (all the same
    type).  ``layout="rows"``: array e holds row i's coefficient of its
    neighbour i+e; ``"columns"``: array e holds, at cell j, the factor by
    which v_j enters the output at j+e (the paper's column storage).  The
    returned :class:`Operator` has ``nz = 1``.
    """
    names = ("diag",) + DIRS9
    raw_dt = _dtype_code(coef["diag"])
    keep, ptrs = [], {}
    for k in names:
        a = coef[k]
        if _numel(a) != nx * ny:
            raise ValueError("coefficient %s has %d elements, expected %d" % (k, _numel(a), nx * ny))
        if _dtype_code(a) != raw_dt:
            raise ValueError("all coefficients must have the same dtype")
        keep.append(a)
        ptrs[k] = _ptr(a)
    lay = {"rows": S9_ROWS, "columns": S9_COLUMNS}[layout] if isinstance(layout, str) else layout
    cs = s9_coeffs(ptrs["diag"], *[ptrs[k] for k in DIRS9], raw_dt, lay)
    st = _STORAGE[storage] if isinstance(storage, str) else int(storage)
    op = s7_opts(st, 0 if jacobi else 1, 1 if keep_true else 0, bx, 0, zchunk, check_every,
                 0, 0, variant, 0, 1 if residual_f64 else 0)
    h = C.c_void_p()
    _check(lib().stencil9_create(C.byref(h), nx, ny, C.byref(cs), C.byref(op)))
    del keep
    return Operator(h.value, nx, ny, 1, st)


def stencil7_destroy(op):
    op.close()


def stencil7_info(op):
    nx, ny, nz, st = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    nb = C.c_size_t()
    _check(lib().stencil7_info(op.handle, C.byref(nx), C.byref(ny), C.byref(nz), C.byref(st),
                               C.byref(nb)))
    return {"nx": nx.value, "ny": ny.value, "nz": nz.value, "storage": st.value,
            "device_bytes": nb.value}


def stencil7_apply(op, x, y=None):
    """``y = A~ x`` with the stored operator; returns y."""
    if y is None:
        y = _empty_like(x)
    dt = _vectors("stencil7_apply", op.n, x, y)
    _check(lib().stencil7_apply(op.handle, _ptr(x), _ptr(y), dt, _stream(x, y)))
    return y


def stencil7_residual(op, b, x, r=None):
    """``r = b - A x`` on the raw system; returns ``(rnorm, bnorm)``."""
    rn, bn = C.c_double(), C.c_double()
    dt = _vectors("stencil7_residual", op.n, b, x, r)
    _check(lib().stencil7_residual(op.handle, _ptr(b), _ptr(x), _ptr(r), dt,
                                   C.byref(rn), C.byref(bn), _stream(b, x, r)))
    return rn.value, bn.value


def stencil7_profile(op, enable):
    """Turn per-kernel timing on/off; returns the totals since the last call
    as ``{kind: (milliseconds, launches)}``."""
    ms = (C.c_double * 6)()
    n = (C.c_longlong * 6)()
    _check(lib().stencil7_profile(op.handle, 1 if enable else 0, ms, n))
    return {k: (ms[j], n[j]) for j, k in enumerate(PROF_KINDS)}


def s7_mem_stats(device=0):
    """(reserved, used) bytes of the library's device memory pool."""
    r, u = C.c_size_t(), C.c_size_t()
    _check(lib().s7_mem_stats(int(device), C.byref(r), C.byref(u)))
    return r.value, u.value


def s7_mem_trim(device=0, keep=0):
    """Return the pool's cached blocks to the device, keeping ``keep`` bytes."""
    _check(lib().s7_mem_trim(int(device), int(keep)))


def s7_mem_set_cache(nbytes):
    """Most bytes a pool keeps reserved after a release (default 64 GiB)."""
    _check(lib().s7_mem_set_cache(int(nbytes)))


def stencil7_residual_noalloc(op, b, x, r=None):
    """:func:`stencil7_residual` without any allocation (device buffers only);
    for callers that may not allocate device memory at call time."""
    rn, bn = C.c_double(), C.c_double()
    dt = _vectors("stencil7_residual_noalloc", op.n, b, x, r)
    _check(lib().stencil7_residual_noalloc(op.handle, _ptr(b), _ptr(x), _ptr(r), dt,
                                           C.byref(rn), C.byref(bn), _stream(b, x, r)))
    return rn.value, bn.value


@dataclass
class SolveResult:
    x: object
    iters: int
    hist: np.ndarray
    true_resid: float
    status: int


def bicgstab_solve(op, b, x=None, tol=1e-6, maxit=500, history=True, true_resid=True):
    """BiCGStab (Algorithm 1) on the operator; ``x`` holds x0 and is overwritten.

    Returns a :class:`SolveResult`; breakdown and non-convergence are
    reported in ``status`` (3, 4), other errors raise :class:`S7Error`.
    """
    if x is None:
        x = _empty_like(b)
        if _is_torch(x):
            x.zero_()
        else:
            x[...] = 0
    dt = _vectors("bicgstab_solve", op.n, b, x)
    it = C.c_int()
    hist = np.zeros(maxit + 1) if history else None
    tr = C.c_double()
    rc = lib().bicgstab_solve(op.handle, _ptr(b), _ptr(x), dt, float(tol),
                              int(maxit), C.byref(it),
                              hist.ctypes.data_as(C.POINTER(C.c_double)) if history else None,
                              C.byref(tr) if true_resid else None, _stream(b, x))
    _check(rc, allow=(EBREAKDOWN, ENOTCONV))
    return SolveResult(x, it.value, hist[:it.value + 1] if history else None,
                       tr.value if true_resid else float("nan"), rc)


@dataclass
class RefinedResult:
    x: object
    outer: int
    inner_total: int
    hist: np.ndarray
    status: int


def bicgstab_solve_refined(op, b, x=None, tol=1e-10, max_outer=30, inner_maxit=200,
                           inner_tol=1e-2):
    """Mixed-precision solve with float64 iterative refinement (float64 b, x)."""
    if x is None:
        x = _empty_like(b)
        if _is_torch(x):
            x.zero_()
        else:
            x[...] = 0
    _vectors("bicgstab_solve_refined", op.n, b, x, dtype=S7_F64)
    outer, inner = C.c_int(), C.c_int()
    hist = np.zeros(max_outer + 1)
    rc = lib().bicgstab_solve_refined(op.handle, _ptr(b), _ptr(x), float(tol), int(max_outer),
                                      int(inner_maxit), float(inner_tol), C.byref(outer),
                                      C.byref(inner), hist.ctypes.data_as(C.POINTER(C.c_double)),
                                      _stream(b, x))
    _check(rc, allow=(EBREAKDOWN, ENOTCONV))
    return RefinedResult(x, outer.value, inner.value, hist[:outer.value + 1], rc)


@dataclass
class BatchResult:
    x: list
    iters: list
    status: list
    resid: list
    rc: int
    policy: dict = None


def bicgstab_solve_batched(ops, bs, xs=None, tol=1e-6, maxit=500, threads=0, zchunk=0,
                           check_every=0, autotune=True, schedule=0, wait_cycles=0,
                           allow_timeout=False, choose_variant=False):
    """Solve independent systems together (one persistent launch, or one
    launch per step kernel, covers all).

    ``ops``: operators (same storage type); ``bs``: right-hand sides (all the
    same dtype); ``xs``: start vectors (default zeros), overwritten with the
    results.  ``tol`` and ``maxit`` may be scalars or per-system sequences.
    ``schedule``: 0 chosen, 1 persistent, -1 one launch per step kernel;
    ``wait_cycles``: bound of the persistent launch's barrier waits (0 =
    default).  With ``allow_timeout`` an S7_ETIMEOUT return is reported in
    the result instead of raised.  ``choose_variant``: the autotuner may run
    the other variant of the step.  ``policy`` of the result: the block
    shape and fusion schedule the solve ran with (:func:`bicgstab_batched_policy`).
    """
    n = len(ops)
    if xs is None:
        xs = []
        for b in bs:
            x = _empty_like(b)
            if _is_torch(x):
                x.zero_()
            else:
                x[...] = 0
            xs.append(x)
    if len(bs) != n or len(xs) != n:
        raise ValueError("bicgstab_solve_batched: one b and one x per operator")
    dt = _dtype_code(bs[0])
    for op, b, x in zip(ops, bs, xs):
        if _vectors("bicgstab_solve_batched", op.n, b, x) != dt:
            raise ValueError("bicgstab_solve_batched: all vectors must have the same dtype")
    tols = [float(tol)] * n if np.isscalar(tol) else [float(t) for t in tol]
    mits = [int(maxit)] * n if np.isscalar(maxit) else [int(m) for m in maxit]
    H = (C.c_void_p * n)(*[op.handle.value for op in ops])
    B = (C.c_void_p * n)(*[_ptr(b) for b in bs])
    X = (C.c_void_p * n)(*[_ptr(x) for x in xs])
    T = (C.c_double * n)(*tols)
    M = (C.c_int * n)(*mits)
    it = (C.c_int * n)()
    stt = (C.c_int * n)()
    rs = (C.c_double * n)()
    o = s7_batch_opts(threads, zchunk, check_every, 0 if autotune else 1, int(schedule),
                      int(wait_cycles), int(bool(choose_variant)))
    rc = lib().bicgstab_solve_batched(n, H, B, X, dt, T, M, it, stt, rs,
                                      C.byref(o), _stream(*bs))
    _check(rc, allow=(EBREAKDOWN, ENOTCONV) + ((ETIMEOUT,) if allow_timeout else ()))
    return BatchResult(xs, list(it), list(stt), list(rs), rc, bicgstab_batched_policy())


def bicgstab_batched_policy():
    """Block shape and fusion schedule of this thread's last batched solve:
    ``threads``, ``zchunk``, ``schedule`` (1 persistent, -1 launch per step
    kernel), ``pipelined`` (pipelined step sweeps or register sweeps),
    ``variant`` (0 Algorithm 1, 1 two-reduction)."""
    v = [C.c_int() for _ in range(5)]
    _check(lib().bicgstab_batched_policy(*[C.byref(a) for a in v]))
    return dict(zip(("threads", "zchunk", "schedule", "pipelined", "variant"),
                    [a.value for a in v]))


def _result_dict(r):
    return {"status": r.status, "outer": r.outer, "inner_iters": r.inner_iters,
            "resid": r.resid, "t_arrive": r.t_arrive, "t_admit": r.t_admit,
            "t_done": r.t_done, "latency": r.t_done - r.t_arrive}


def s7_server_create(hbm_budget_bytes=0, storage="bf16", max_active=0, steps_per_tick=0,
                     threads=0, zchunk=0, inner_tol=0.0, inner_maxit=0, max_outer=0,
                     three_pass=False, residual_f64=False):
    st = _STORAGE[storage] if isinstance(storage, str) else int(storage)
    o = s7_server_opts(int(hbm_budget_bytes), st, max_active, steps_per_tick, threads, zchunk,
                       float(inner_tol), inner_maxit, max_outer, 1 if three_pass else 0,
                       1 if residual_f64 else 0)
    h = C.c_void_p()
    _check(lib().s7_server_create(C.byref(h), C.byref(o)))
    return h


def s7_server_submit(srv, nx, ny, nz, coef, b, x, tol):
    """Queue a request.  ``coef`` holds arrays of nx*ny*nz values, or of one
    value each for a constant-coefficient operator."""
    names = ("diag",) + DIRS
    raw_dt = _dtype_code(coef["diag"])
    constant = 1 if nx * ny * nz > 1 and all(_numel(coef[k]) == 1 for k in names) else 0
    cs = s7_coeffs(*[_ptr(coef[k]) for k in names], raw_dt, constant)
    dt = _vectors("s7_server_submit", nx * ny * nz, b, x)
    req = s7_request(nx, ny, nz, cs, _ptr(b), _ptr(x), dt, float(tol))
    rid = C.c_uint64()
    _check(lib().s7_server_submit(srv, C.byref(req), C.byref(rid)))
    return rid.value


def s7_server_poll(srv, rid):
    r = s7_result()
    rc = lib().s7_server_poll(srv, rid, C.byref(r))
    if rc == EAGAIN:
        return None
    _check(rc)
    return _result_dict(r)


def s7_server_wait(srv, rid, timeout=-1.0):
    r = s7_result()
    _check(lib().s7_server_wait(srv, rid, C.byref(r), float(timeout)))
    return _result_dict(r)


def s7_server_release(srv, rid):
    _check(lib().s7_server_release(srv, rid))


def s7_server_get_stats(srv):
    s = s7_server_stats()
    _check(lib().s7_server_get_stats(srv, C.byref(s)))
    return {k: getattr(s, k) for k, _ in s7_server_stats._fields_}


def s7_server_destroy(srv):
    return lib().s7_server_destroy(srv)


class Server:
    """A solve server (continuous batching).  Keeps each request's buffers
    alive until the request has finished."""

    def __init__(self, **kw):
        self._h = s7_server_create(**kw)
        self._keep = {}

    def submit(self, nx, ny, nz, coef, b, x=None, tol=1e-6):
        if x is None:
            x = _empty_like(b)
        rid = s7_server_submit(self._h, nx, ny, nz, coef, b, x, tol)
        self._keep[rid] = (coef, b, x)
        return rid

    def result(self, rid):
        return self._keep[rid][2]

    def poll(self, rid):
        return s7_server_poll(self._h, rid)

    def wait(self, rid, timeout=-1.0):
        return s7_server_wait(self._h, rid, timeout)

    def release(self, rid):
        s7_server_release(self._h, rid)
        return self._keep.pop(rid)[2]

    def stats(self):
        return s7_server_get_stats(self._h)

    def close(self):
        if self._h:
            s7_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
