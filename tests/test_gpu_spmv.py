"""GPU parity of the stencil SpMV (stencil7_apply) against the FP64 oracle.

The library stores A~ = D^-1 A rounded once to the storage type; the oracle
forms the same operator in float64 (Sec. IV: unit main diagonal) and applies
it to the same stored input values.  The error metric is per row,
|y_gpu - y_ref|_i / (|A~||x|)_i, which stays meaningful where a row's sum
cancels; the bound comes from float32 accumulation of 7 terms (float64 for
F64 storage) plus the final rounding of y to the storage type.
"""

import numpy as np
import pytest

import synth
from oracle import stencil
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

SHAPES = [
    (17, 9, 33),    # nx not a multiple of any vector width: element-wise path
    (64, 48, 40),   # several tiles in x and y, several z chunks
    (40, 31, 70),   # ragged y tiles, nz not a multiple of the chunk
    (1, 1, 7),      # a single column
    (3, 1, 1),      # a single row
    (1, 5, 1),
    (8, 8, 8),
    (128, 20, 9),
]


@pytest.fixture(scope="module")
def s7():
    import paper_2010_03660_gb300 as m
    m.lib()
    return m


@pytest.mark.parametrize("storage", ["f32", "f64", "bf16", "f16"])
@pytest.mark.parametrize("shape", SHAPES)
def test_spmv_varcoef(s7, storage, shape):
    import torch
    nx, ny, nz = shape
    raw = np.float64 if storage == "f64" else np.float32
    p = synth.varcoef(nx, ny, nz, seed=3, dtype=raw)
    op_coef = stencil.jacobi_scale(nx, ny, nz, p.coef, storage)
    x64, xd = gu.stored_vector(synth.random_vector(p.n, 5, 4, np.float64), storage)
    with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage=storage) as op:
        y = s7.stencil7_apply(op, xd)
        torch.cuda.synchronize()
        err = gu.spmv_row_error(nx, ny, nz, op_coef, x64, y.double().cpu().numpy())
    assert err <= gu.SPMV_TOL[storage], err


@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_spmv_constant_and_raw_diagonal(s7, storage):
    import torch
    nx, ny, nz = 33, 17, 12
    raw = np.float64 if storage == "f64" else np.float32
    pc = synth.convdiff_constant(nx, ny, nz, seed=0, dtype=raw)
    x64, xd = gu.stored_vector(synth.random_vector(pc.n, 8, 4, np.float64), storage)
    with s7.stencil7_create(nx, ny, nz, pc.coef, storage=storage) as op:
        y = s7.stencil7_apply(op, xd)
        torch.cuda.synchronize()
        err = gu.spmv_row_error(nx, ny, nz, stencil.jacobi_scale(nx, ny, nz, pc.coef, storage),
                                x64, y.double().cpu().numpy())
    assert err <= gu.SPMV_TOL[storage]
    # raw seven-diagonal operator (no Jacobi scaling)
    p = synth.varcoef(nx, ny, nz, seed=9, dtype=raw)
    with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage=storage,
                            jacobi=False) as op:
        y = s7.stencil7_apply(op, xd)
        torch.cuda.synchronize()
        err = gu.spmv_row_error(nx, ny, nz, stencil.rounded(nx, ny, nz, p.coef, storage),
                                x64, y.double().cpu().numpy())
    assert err <= gu.SPMV_TOL[storage]


def test_spmv_host_buffers_match_device(s7):
    import torch
    nx, ny, nz = 24, 11, 13
    p = synth.varcoef(nx, ny, nz, seed=4)
    x = synth.random_vector(p.n, 1, 1, np.float32)
    with s7.stencil7_create(nx, ny, nz, p.coef, storage="f32") as op:   # host coefficients
        yh = s7.stencil7_apply(op, x)                                    # numpy in, numpy out
        yd = s7.stencil7_apply(op, gu.to_dev(x))
        torch.cuda.synchronize()
        assert np.array_equal(yh, yd.cpu().numpy())


def test_spmv_launch_shapes_agree_bitwise(s7):
    # the tile shape and z chunk change the schedule, not the arithmetic of a row
    import torch
    nx, ny, nz = 96, 40, 50
    p = synth.varcoef(nx, ny, nz, seed=12)
    x = gu.to_dev(synth.random_vector(p.n, 2, 2, np.float32))
    outs = []
    for bx, by, zc in [(0, 0, 0), (8, 4, 5), (24, 16, 50), (3, 7, 1)]:
        with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage="f32",
                                bx=bx, by=by, zchunk=zc) as op:
            outs.append(s7.stencil7_apply(op, x).cpu().numpy())
    torch.cuda.synchronize()
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_spmv_laplacian_eigenvector(s7):
    # closed form on the GPU too: A v = lambda v for the Dirichlet Laplacian
    import torch
    from oracle import direct
    nx, ny, nz = 30, 20, 24
    lap = synth.laplacian(nx, ny, nz)
    lam, v = direct.laplacian_eigenpair(nx, ny, nz, 2, 3, 5)
    with s7.stencil7_create(nx, ny, nz, lap.coef, storage="f64", jacobi=False) as op:
        y = s7.stencil7_apply(op, gu.to_dev(v)).cpu().numpy()
    assert np.max(np.abs(y - lam * v)) < 1e-13


def test_zero_diagonal_is_rejected(s7):
    p = synth.varcoef(8, 8, 8, seed=1)
    p.coef["diag"] = p.coef["diag"].copy()
    p.coef["diag"][100] = 0.0
    with pytest.raises(s7.S7Error) as e:
        s7.stencil7_create(8, 8, 8, p.coef, storage="f32")
    assert e.value.code == s7.EINVAL


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_16bit_output_rounding_is_nearest_even_bitwise(s7, storage):
    """y = c x with a raw diagonal c and zero off-diagonals: c and x are 16-bit
    values, so c*x is exact in float32 and the only rounding is the final one
    to the storage type, which must equal the oracle's round-to-nearest-even
    bit for bit (ties included)."""
    import torch
    nx, ny, nz = 64, 16, 8
    n = nx * ny * nz
    c = float(stencil.round_to(np.float64(1.3), storage))
    coef = {"diag": c, **{d: 0.0 for d in synth.DIRS}}
    x64 = stencil.round_to(synth.random_vector(n, 21, 3, np.float64), storage)
    x64[:64] = stencil.round_to(np.linspace(-3, 3, 64), storage)
    with s7.stencil7_create(nx, ny, nz, coef, storage=storage, jacobi=False) as op:
        y = s7.stencil7_apply(op, gu.to_dev(x64, gu.torch_dtype(storage)))
        torch.cuda.synchronize()
        got = y.double().cpu().numpy()
    want = stencil.round_to(c * x64, storage)
    assert np.array_equal(got, want)
