"""Helpers shared by the GPU parity tests."""

import numpy as np

import synth
from oracle import stencil

STORAGE_NP = {"f64": np.float64, "f32": np.float32}
# per-row relative SpMV bound |y - y_ref|_i / (|A||x|)_i, derived from the
# accumulation precision (7 terms) plus the final rounding of y to storage
SPMV_TOL = {"f64": 1e-14, "f32": 2e-6, "bf16": 2 ** -8 + 2e-6, "f16": 2 ** -11 + 2e-6}


def torch_dev():
    import torch
    return torch.device("cuda:0")


def to_dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(torch_dev())


def torch_dtype(storage):
    import torch
    return {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16,
            "f16": torch.float16}[storage]


def coef_on_device(p):
    if p.constant:
        return dict(p.coef)
    return {k: to_dev(v) for k, v in p.coef.items()}


def stored_vector(v, storage):
    """A float64 vector rounded to the storage type, as float64 (oracle side)
    and as a device tensor of that type (GPU side), holding the same values."""
    v64 = stencil.round_to(np.asarray(v, dtype=np.float64), storage)
    return v64, to_dev(v64, torch_dtype(storage))


def spmv_row_error(nx, ny, nz, op_coef, x64, y_gpu):
    ref = stencil.apply(nx, ny, nz, op_coef, x64)
    den = stencil.abs_apply(nx, ny, nz, op_coef, x64)
    den = np.where(den == 0, 1.0, den)
    return float(np.max(np.abs(np.asarray(y_gpu, dtype=np.float64) - ref) / den))


def problem(kind, nx, ny, nz, seed, dtype=np.float32):
    if kind == "varcoef":
        return synth.varcoef(nx, ny, nz, seed=seed, dtype=dtype)
    if kind == "const":
        return synth.convdiff_constant(nx, ny, nz, seed=seed, dtype=dtype)
    raise ValueError(kind)


def fp32_step_window(nx, ny, nz, coef, b, tol, maxit, oracle_iters, orders=6):
    """Step-count window of a float32 solve: the range of the float32 rounding
    model's step counts over `orders` summation orders, joined with the
    float64 oracle's count, widened by max(2, 10%) (a handful of orders
    samples, not bounds, the orders a float32 implementation may take)."""
    from oracle import fp32model
    lo, hi = fp32model.step_range(nx, ny, nz, coef, b, tol, maxit=maxit, orders=orders)
    lo, hi = min(lo, oracle_iters), max(hi, oracle_iters)
    m = max(2, lo // 10)
    return lo - m, hi + m
