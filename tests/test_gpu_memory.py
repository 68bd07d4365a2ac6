"""Device memory pool and host-buffer paths of the C ABI.

Handles take their memory from the library's stream-ordered pool; a
destroyed handle's blocks stay cached for the next one.  Coefficients in
pinned host memory are read in place by the scaling kernels, pageable host
memory is staged through pool blocks, and a solve with host b / x copies x
out on a second stream beside the true residual.  All of these must give the
same bits as the device-buffer paths.
"""

import numpy as np
import pytest

import synth
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

MiB = 1 << 20


@pytest.fixture(scope="module")
def s7():
    import paper_2010_03660_gb300 as m
    m.lib()
    return m


def _pinned(p):
    import torch
    return {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in p.coef.items()}


def test_pool_caches_and_trims(s7):
    nx, ny, nz = 96, 64, 48
    p = synth.varcoef(nx, ny, nz, seed=3)
    coef = gu.coef_on_device(p)
    b = gu.to_dev(p.b)
    r0, u0 = s7.s7_mem_stats(0)
    with s7.stencil7_create(nx, ny, nz, coef, storage="f32") as op:
        s7.bicgstab_solve(op, b, tol=0.0, maxit=3)
        held = s7.stencil7_info(op)["device_bytes"]
        r1, u1 = s7.s7_mem_stats(0)
        assert held > 10 * nx * ny * nz * 4
        assert u1 - u0 >= held
    r2, u2 = s7.s7_mem_stats(0)
    assert u2 == u0                      # every block came back
    assert r2 >= u0 + held               # and stays cached (limit 64 GiB)
    with s7.stencil7_create(nx, ny, nz, coef, storage="f32") as op:
        s7.bicgstab_solve(op, b, tol=0.0, maxit=3)
        r3, _ = s7.s7_mem_stats(0)
    assert r3 < r2 + held // 2           # the second handle reused them
    s7.s7_mem_trim(0, 0)
    r4, u4 = s7.s7_mem_stats(0)
    assert u4 == u0
    assert r4 <= u4 + 64 * MiB


def test_pool_cache_limit_zero_releases(s7):
    nx, ny, nz = 64, 64, 64
    p = synth.varcoef(nx, ny, nz, seed=4)
    s7.s7_mem_trim(0, 0)
    try:
        s7.s7_mem_set_cache(0)
        with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage="f32") as op:
            s7.bicgstab_solve(op, gu.to_dev(p.b), tol=0.0, maxit=2)
        # a later synchronisation returns the free blocks
        with s7.stencil7_create(4, 4, 4, gu.coef_on_device(synth.varcoef(4, 4, 4, seed=1)),
                                storage="f32"):
            pass
        s7.s7_mem_trim(0, 1 << 62)       # synchronises, trims nothing itself
        r, u = s7.s7_mem_stats(0)
        assert r <= u + 64 * MiB
    finally:
        s7.s7_mem_set_cache(64 << 30)


def test_mem_stats_bad_device(s7):
    with pytest.raises(s7.S7Error):
        s7.s7_mem_stats(-1)
    with pytest.raises(s7.S7Error):
        s7.s7_mem_trim(64, 0)


@pytest.mark.parametrize("storage,raw", [("f32", np.float32), ("f32", np.float64),
                                         ("bf16", np.float32), ("f64", np.float64)])
@pytest.mark.parametrize("keep_true", [False, True])
def test_create_from_pinned_and_pageable_host(s7, storage, raw, keep_true):
    """Same stored operator from device, pinned-host (read in place) and
    pageable-host (staged) coefficients: A~ x agrees bit for bit."""
    import torch
    nx, ny, nz = 45, 22, 17
    p = synth.varcoef(nx, ny, nz, seed=8, dtype=raw)
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f64": torch.float64}[storage]
    x = torch.from_numpy(np.random.default_rng(2).standard_normal(p.n)).to(tdt).to(gu.torch_dev())
    outs = []
    for coef in (gu.coef_on_device(p), _pinned(p), dict(p.coef)):
        with s7.stencil7_create(nx, ny, nz, coef, storage=storage, keep_true=keep_true) as op:
            outs.append(s7.stencil7_apply(op, x).double().cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(outs[0], outs[2])


def test_create_9pt_from_host(s7):
    import torch
    nx, ny = 130, 77
    q = synth.varcoef9(nx, ny, seed=5)
    x = torch.from_numpy(np.random.default_rng(3).standard_normal(q.n).astype(np.float32))
    x = x.to(gu.torch_dev())
    outs = []
    for coef in ({k: gu.to_dev(v) for k, v in q.coef.items()}, _pinned(q), dict(q.coef)):
        with s7.stencil9_create(nx, ny, coef, storage="f32") as op:
            outs.append(s7.stencil7_apply(op, x).cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(outs[0], outs[2])


@pytest.mark.parametrize("storage", ["f32", "f64", "bf16"])
def test_solve_with_host_buffers_matches_device(s7, storage):
    """Pinned and pageable host b / x (x copied out beside the true residual)
    give the device-buffer result bit for bit."""
    import torch
    nx, ny, nz = 40, 36, 30
    raw = np.float64 if storage == "f64" else np.float32
    p = synth.varcoef(nx, ny, nz, seed=12, dtype=raw)
    with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage=storage) as op:
        bd = gu.to_dev(p.b)
        xd = torch.zeros_like(bd)
        rd = s7.bicgstab_solve(op, bd, xd, tol=1e-5, maxit=300)
        ref = xd.cpu().numpy()
        bp = torch.from_numpy(p.b).pin_memory()
        xp = torch.zeros_like(bp).pin_memory()
        rp = s7.bicgstab_solve(op, bp, xp, tol=1e-5, maxit=300)
        xn = np.zeros_like(p.b)
        rn = s7.bicgstab_solve(op, p.b, xn, tol=1e-5, maxit=300)
        # without the true residual the copy-out stays on the handle's stream
        xq = np.zeros_like(p.b)
        rq = s7.bicgstab_solve(op, p.b, xq, tol=1e-5, maxit=300, true_resid=False)
    assert rd.status == 0 and rd.iters == rp.iters == rn.iters == rq.iters
    assert np.array_equal(ref, xp.numpy())
    assert np.array_equal(ref, xn)
    assert np.array_equal(ref, xq)
    assert rd.true_resid == rp.true_resid == rn.true_resid
    assert np.array_equal(rd.hist, rn.hist)
