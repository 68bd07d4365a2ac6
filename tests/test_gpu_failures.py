"""Failure paths, injected on the host; nothing faults, traps or hangs the
GPU.  Non-finite input ends a solve with a breakdown status after bounded
work; an allocation that cannot be met returns S7_ENOMEM and leaks nothing;
bad arguments are rejected before any launch."""

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


def test_nan_rhs_is_a_breakdown_not_a_hang(s7):
    p = synth.varcoef(20, 12, 9, seed=3)
    b = p.b.copy()
    b[17] = np.nan
    with s7.stencil7_create(20, 12, 9, gu.coef_on_device(p), storage="f32") as op:
        r = s7.bicgstab_solve(op, gu.to_dev(b), tol=1e-6, maxit=50)
        assert r.status == s7.EBREAKDOWN and r.iters == 0
        # the handle stays usable
        ok = s7.bicgstab_solve(op, gu.to_dev(p.b), tol=1e-6, maxit=500)
        assert ok.status == 0


def test_nan_in_batch_stops_only_that_system(s7):
    probs = [synth.varcoef(16, 16, 16, seed=40 + j) for j in range(3)]
    bs = [gu.to_dev(p.b) for p in probs]
    bs[1][5] = float("nan")
    ops = [s7.stencil7_create(16, 16, 16, gu.coef_on_device(p), storage="f32") for p in probs]
    try:
        res = s7.bicgstab_solve_batched(ops, bs, tol=1e-6, maxit=500)
        assert res.rc == s7.EBREAKDOWN
        assert res.status == [0, s7.EBREAKDOWN, 0]
    finally:
        for op in ops:
            op.close()


def test_out_of_memory_is_reported_and_nothing_leaks(s7):
    import torch
    # a 5000^3 constant-coefficient operator that also keeps the true
    # operator: its first per-cell array (500 GB) cannot be allocated, so
    # creation fails at once with nothing else held
    e = 5000
    c = {"diag": 6.0, **{d: -1.0 for d in synth.DIRS}}
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    with pytest.raises(s7.S7Error) as err:
        s7.stencil7_create(e, e, e, c, storage="f32", keep_true=True)
    assert err.value.code == s7.ENOMEM
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (16 << 20)
    # the library still works afterwards
    p = synth.varcoef(12, 10, 8, seed=5)
    with s7.stencil7_create(12, 10, 8, p.coef, storage="f32") as op:
        assert s7.bicgstab_solve(op, p.b.copy(), tol=1e-6, maxit=300).status == 0


def test_bad_arguments_rejected(s7):
    p = synth.varcoef(8, 8, 8, seed=1)
    with s7.stencil7_create(8, 8, 8, p.coef, storage="f32") as op:
        x = gu.to_dev(p.b)
        with pytest.raises(s7.S7Error) as e:
            s7.stencil7_apply(op, x, x)                      # overlapping in/out
        assert e.value.code == s7.EINVAL
        with pytest.raises(s7.S7Error) as e:
            s7.stencil7_apply(op, gu.to_dev(p.b.astype(np.float64)))   # wrong dtype
        assert e.value.code == s7.EINVAL
        with pytest.raises(s7.S7Error) as e:
            s7.bicgstab_solve(op, gu.to_dev(p.b), tol=-1.0)
        assert e.value.code == s7.EINVAL
        # refinement with 16-bit storage needs the true operator
    with s7.stencil7_create(8, 8, 8, p.coef, storage="bf16") as op:
        with pytest.raises(s7.S7Error) as e:
            s7.bicgstab_solve_refined(op, gu.to_dev(p.b.astype(np.float64)))
        assert e.value.code == s7.EINVAL
