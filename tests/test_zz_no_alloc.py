"""stencil7_residual_noalloc, the residual entry point that allocates nothing.

It serves callers that may not allocate device memory at call time (a
service whose pool owns the whole memory budget, a loop that cannot absorb
cudaMalloc's synchronisation).  Checked through the C ABI against
stencil7_residual, on two calls in a row (the static scratch keeps the
previous call's contents, so the second call shows it is cleared properly).
This file is named to be collected last.
"""

import ctypes

import numpy as np
import pytest

import synth
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def s7():
    import paper_2010_03660_gb300 as m
    m.lib()
    return m


def _norms(lib, fn, op, b, x, r, dt):
    rn, bn = ctypes.c_double(), ctypes.c_double()
    rc = fn(op.handle, b.data_ptr(), x.data_ptr(), r.data_ptr() if r is not None else None, dt,
            ctypes.byref(rn), ctypes.byref(bn), None)
    return rc, rn.value, bn.value


@pytest.mark.parametrize("storage,keep_true,dtype", [
    ("f32", True, "f32"), ("f32", False, "f32"), ("f32", True, "f64"), ("f32", False, "f64"),
    # 16-bit storage without the raw copy: the residual comes from the stored
    # 16-bit operator times the kept diagonal
    ("bf16", False, "f32"), ("f16", False, "f64"), ("bf16", True, "f64")])
def test_noalloc_matches_residual_twice(s7, storage, keep_true, dtype):
    """Both entry points run the same sweep with the same launch shape and the
    same fixed-order sums, so the residual vector and the norms agree bit for
    bit."""
    import torch
    nx, ny, nz = 37, 29, 23
    p = synth.varcoef(nx, ny, nz, seed=51)
    npdt = np.float64 if dtype == "f64" else np.float32
    dt = s7.S7_F64 if dtype == "f64" else s7.S7_F32
    lib = s7.lib()
    with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage=storage,
                            keep_true=keep_true) as op:
        for call in range(2):
            x = gu.to_dev(synth.random_vector(p.n, 60 + call, 1, npdt))
            b = gu.to_dev(p.b.astype(npdt))
            r_ref = torch.zeros_like(b)
            r_new = torch.full_like(b, float("nan"))
            rc0, rn0, bn0 = _norms(lib, lib.stencil7_residual, op, b, x, r_ref, dt)
            rc1, rn1, bn1 = _norms(lib, lib.stencil7_residual_noalloc, op, b, x, r_new, dt)
            torch.cuda.synchronize()
            assert rc0 == 0 and rc1 == 0, s7.s7_last_error()
            assert torch.equal(r_ref, r_new)
            assert rn1 == rn0 and bn1 == bn0


def test_noalloc_allocates_nothing_after_setup(s7):
    import torch
    nx, ny, nz = 40, 30, 20
    p = synth.varcoef(nx, ny, nz, seed=52)
    with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage="f32",
                            keep_true=True) as op:
        b = gu.to_dev(p.b)
        x = gu.to_dev(synth.random_vector(p.n, 70, 1, np.float32))
        s7.stencil7_residual_noalloc(op, b, x)          # first call: per-device set-up
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        info0 = s7.stencil7_info(op)["device_bytes"]
        pool0 = s7.s7_mem_stats(0)                      # the library's own pool
        for _ in range(3):
            s7.stencil7_residual_noalloc(op, b, x)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert s7.stencil7_info(op)["device_bytes"] == info0
        assert s7.s7_mem_stats(0) == pool0


def test_noalloc_rejects_host_buffers_and_oversize(s7):
    nx, ny, nz = 16, 8, 8
    p = synth.varcoef(nx, ny, nz, seed=53)
    with s7.stencil7_create(nx, ny, nz, p.coef, storage="f32") as op:
        with pytest.raises(s7.S7Error) as e:
            s7.stencil7_residual_noalloc(op, p.b, p.b)      # numpy: host memory
        assert e.value.code == s7.EINVAL
    # one z plane per block on a tall column: more blocks than the scratch holds
    nz = 70000
    c = {"diag": 4.0, **{d: -0.5 for d in synth.DIRS}}
    with s7.stencil7_create(4, 1, nz, c, storage="f32", zchunk=1) as op:
        b = gu.to_dev(np.ones(4 * nz, np.float32))
        with pytest.raises(s7.S7Error) as e:
            s7.stencil7_residual_noalloc(op, b, b)
        assert e.value.code == s7.EINVAL and "blocks" in str(e.value)


def test_noalloc_refuses_a_capturing_stream(s7):
    """The call waits on the host for its norms, so on a stream that is being
    captured it returns S7_EINVAL before any other CUDA call on that stream,
    and the capture stays valid."""
    import torch
    nx, ny, nz = 16, 8, 8
    p = synth.varcoef(nx, ny, nz, seed=54)
    with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage="f32") as op:
        b = gu.to_dev(p.b)
        x = gu.to_dev(p.b)
        s7.stencil7_residual_noalloc(op, b, x)          # set-up outside any capture
        torch.cuda.synchronize()
        y = torch.zeros(4, device=b.device)
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                y.add_(1)
                with pytest.raises(s7.S7Error) as e:
                    s7.stencil7_residual_noalloc(op, b, x)
                y.add_(1)
        assert e.value.code == s7.EINVAL and "capturing" in str(e.value)
        g.replay()
        torch.cuda.synchronize()
        assert float(y[0]) == 2.0
