"""GPU parity of bicgstab_solve against the FP64 oracle (Algorithm 1).

Both sides run Algorithm 1 on the same stored operator (A~ = D^-1 A rounded
to the storage type) and the same right-hand side, with the same stopping
rule.  BiCGStab amplifies rounding differences: in the oracle alone, changing
only the rounding order of the inner products moves the FP64 residual
history by ~3% after 60 steps while x still agrees to ~1e-9
(tests/test_oracle.py::test_history_sensitivity_to_dot_rounding).  So the
bars are: the first steps of the history agree tightly, the final x agrees
within the bound the tolerance allows, the true residual meets the
tolerance, and step counts agree within a small window.  FP32 solves to 1e-6
agree in x within 1e-4 relative.
"""

import numpy as np
import pytest

import synth
from oracle import bicgstab as ob
from oracle import stencil
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def s7():
    import paper_2010_03660_gb300 as m
    m.lib()
    return m


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def test_config1_fp64_constant_convdiff_32cubed(s7):
    """32^3 convection-diffusion, FP64, tol 1e-8, maxit 500."""
    p = synth.convdiff_constant(32, 32, 32, seed=0)
    orc = ob.bicgstab(32, 32, 32, p.coef, p.b, tol=1e-8, maxit=500, storage="f64")
    with s7.stencil7_create(32, 32, 32, p.coef, storage="f64") as op:
        res = s7.bicgstab_solve(op, gu.to_dev(p.b), tol=1e-8, maxit=500)
        x = res.x.cpu().numpy()
    assert res.status == 0 and orc.status == 0
    assert abs(res.iters - orc.iters) <= 3
    assert np.max(np.abs(res.hist[:15] - orc.hist[:15]) / orc.hist[:15]) < 1e-9
    assert rel(x, orc.x) < 1e-7
    assert res.true_resid <= 1.01e-8
    sc = stencil.jacobi_scale(32, 32, 32, p.coef, "f64")
    bt = stencil.scale_rhs(32, 32, 32, p.coef, p.b)
    tr = np.linalg.norm(bt - stencil.apply(32, 32, 32, sc, x)) / np.linalg.norm(bt)
    assert abs(tr - res.true_resid) <= 1e-6 * tr


@pytest.mark.parametrize("shape", [(64, 48, 40), (61, 37, 29), (17, 9, 33), (1, 1, 50)])
def test_fp32_varcoef_solve(s7, shape):
    nx, ny, nz = shape
    p = synth.varcoef(nx, ny, nz, seed=21)
    orc = ob.bicgstab(nx, ny, nz, p.coef, p.b, tol=1e-6, maxit=1000, storage="f32")
    with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage="f32") as op:
        res = s7.bicgstab_solve(op, gu.to_dev(p.b), tol=1e-6, maxit=1000)
        x = res.x.cpu().numpy()
    assert res.status == 0
    assert res.hist[-1] <= 1e-6 and res.hist[0] == pytest.approx(1.0, rel=1e-6)
    assert abs(res.iters - orc.iters) <= max(3, orc.iters // 10)
    assert rel(x, orc.x) <= 1e-4
    assert res.true_resid <= 2e-6
    # the residual reported by the oracle for the GPU's x agrees
    sc = stencil.jacobi_scale(nx, ny, nz, p.coef, "f32")
    bt = stencil.scale_rhs(nx, ny, nz, p.coef, p.b)
    tr = np.linalg.norm(bt - stencil.apply(nx, ny, nz, sc, x.astype(np.float64))) / np.linalg.norm(bt)
    assert abs(tr - res.true_resid) <= 1e-3 * tr + 1e-9


def test_fp64_varcoef_matches_oracle_step_by_step(s7):
    nx, ny, nz = 45, 30, 26
    p = synth.varcoef(nx, ny, nz, seed=5, dtype=np.float64)
    orc = ob.bicgstab(nx, ny, nz, p.coef, p.b, tol=1e-10, maxit=400, storage="f64")
    with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage="f64") as op:
        res = s7.bicgstab_solve(op, gu.to_dev(p.b), tol=1e-10, maxit=400)
    assert res.status == 0 and abs(res.iters - orc.iters) <= max(3, orc.iters // 20)
    assert np.max(np.abs(res.hist[:15] - orc.hist[:15]) / orc.hist[:15]) < 1e-9
    assert rel(res.x.cpu().numpy(), orc.x) < 1e-8
    assert res.true_resid <= 1.01e-10


def test_general_x0_and_degenerate_cases(s7):
    import torch
    nx, ny, nz = 20, 10, 12
    p = synth.varcoef(nx, ny, nz, seed=31, dtype=np.float64)
    x0 = synth.random_vector(p.n, 4, 4, np.float64)
    orc = ob.bicgstab(nx, ny, nz, p.coef, p.b, x0=x0, tol=1e-9, maxit=300)
    with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage="f64") as op:
        res = s7.bicgstab_solve(op, gu.to_dev(p.b), gu.to_dev(x0), tol=1e-9, maxit=300)
        assert res.status == 0 and abs(res.iters - orc.iters) <= 3
        assert rel(res.x.cpu().numpy(), orc.x) < 5e-8
        assert res.hist[0] == pytest.approx(orc.hist[0], rel=1e-10)
        assert np.max(np.abs(res.hist[:10] - orc.hist[:10]) / orc.hist[:10]) < 1e-9
        # b = 0: x = 0 after zero steps, whatever x0
        z = torch.zeros(p.n, dtype=torch.float64, device="cuda:0")
        r0 = s7.bicgstab_solve(op, z, gu.to_dev(x0), tol=1e-8, maxit=10)
        assert r0.iters == 0 and r0.status == 0 and float(r0.x.abs().max()) == 0.0
        # exact start: no step
        xe = gu.to_dev(orc.x)
        r1 = s7.bicgstab_solve(op, gu.to_dev(p.b), xe, tol=1e-8, maxit=10)
        assert r1.iters == 0 and r1.status == 0
        # maxit reached: NOTCONV with a full history
        r2 = s7.bicgstab_solve(op, gu.to_dev(p.b), tol=1e-30, maxit=7)
        assert r2.status == s7.ENOTCONV and r2.iters == 7 and len(r2.hist) == 8
        o2 = ob.bicgstab(nx, ny, nz, p.coef, p.b, tol=1e-30, maxit=7)
        assert np.max(np.abs(r2.hist - o2.hist) / o2.hist) < 1e-10
        # maxit = 0
        r3 = s7.bicgstab_solve(op, gu.to_dev(p.b), tol=1e-8, maxit=0)
        assert r3.iters == 0 and r3.status == s7.ENOTCONV


def test_single_cell_and_single_row(s7):
    c1 = {"diag": 2.5, **{d: 0.0 for d in synth.DIRS}}
    with s7.stencil7_create(1, 1, 1, c1, storage="f64") as op:
        res = s7.bicgstab_solve(op, gu.to_dev(np.array([5.0])), tol=1e-12, maxit=5)
        assert res.status == 0 and res.x.item() == pytest.approx(2.0)
    p = synth.varcoef(1, 1, 40, seed=2, dtype=np.float64)
    orc = ob.bicgstab(1, 1, 40, p.coef, p.b, tol=1e-12, maxit=200)
    with s7.stencil7_create(1, 1, 40, gu.coef_on_device(p), storage="f64") as op:
        res = s7.bicgstab_solve(op, gu.to_dev(p.b), tol=1e-12, maxit=200)
    assert res.status == 0 and abs(res.iters - orc.iters) <= 3
    assert rel(res.x.cpu().numpy(), orc.x) < 1e-10


def test_host_buffers_and_mixed_types(s7):
    nx, ny, nz = 30, 21, 17
    p = synth.varcoef(nx, ny, nz, seed=41)
    with s7.stencil7_create(nx, ny, nz, p.coef, storage="f32") as op:
        rh = s7.bicgstab_solve(op, p.b.copy(), tol=1e-6, maxit=500)            # numpy f32
        rd = s7.bicgstab_solve(op, gu.to_dev(p.b), tol=1e-6, maxit=500)       # torch f32
        r64 = s7.bicgstab_solve(op, p.b.astype(np.float64), tol=1e-6, maxit=500)  # numpy f64
    assert rh.iters == rd.iters == r64.iters
    assert np.array_equal(rh.x, rd.x.cpu().numpy())
    assert np.array_equal(rh.x.astype(np.float64), r64.x)


def test_solves_are_deterministic(s7):
    nx, ny, nz = 50, 41, 37
    p = synth.varcoef(nx, ny, nz, seed=42)
    with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage="f32") as op:
        a = s7.bicgstab_solve(op, gu.to_dev(p.b), tol=1e-7, maxit=500)
        b = s7.bicgstab_solve(op, gu.to_dev(p.b), tol=1e-7, maxit=500)
    assert a.iters == b.iters
    assert np.array_equal(a.hist, b.hist)
    assert np.array_equal(a.x.cpu().numpy(), b.x.cpu().numpy())


def test_graph_step_count_does_not_change_results(s7):
    nx, ny, nz = 40, 33, 21
    p = synth.varcoef(nx, ny, nz, seed=43)
    outs = []
    for ce in (1, 3, 16):
        with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage="f32",
                                check_every=ce) as op:
            outs.append(s7.bicgstab_solve(op, gu.to_dev(p.b), tol=1e-6, maxit=500))
    for o in outs[1:]:
        assert o.iters == outs[0].iters
        assert np.array_equal(o.x.cpu().numpy(), outs[0].x.cpu().numpy())


@pytest.mark.parametrize("shape", [(64, 48, 40), (40, 31, 70), (8, 3, 5)])
def test_pipeline_depth_does_not_change_results(s7, shape):
    # the shared-memory pipelined sweeps (2 or 3 stages) and the direct-load
    # sweeps (stages = 1) do the same arithmetic in the same order
    nx, ny, nz = shape
    p = synth.varcoef(nx, ny, nz, seed=44)
    outs = []
    for stages, by, kinds in ((1, 0, 0), (2, 0, 0), (3, 0, 3), (2, 3, 3), (3, 1, 2), (2, 8, 1)):
        with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage="f32",
                                stages=stages, by=by, pipe_kinds=kinds) as op:
            outs.append(s7.bicgstab_solve(op, gu.to_dev(p.b), tol=1e-6, maxit=300))
    for o in outs[1:]:
        assert o.iters == outs[0].iters
        assert np.array_equal(o.hist, outs[0].hist)
        assert np.array_equal(o.x.cpu().numpy(), outs[0].x.cpu().numpy())


@pytest.mark.parametrize("storage", ["f32", "f64", "bf16", "f16"])
@pytest.mark.parametrize("shape", [(64, 48, 40), (40, 31, 70), (8, 3, 5)])
def test_pipeline_depth_two_reduction_variant(s7, storage, shape):
    # the pipelined q/y and fused passes (kinds 2 and 3) against the
    # direct-load sweeps with the same policies and tile: bit for bit.  (A
    # different tile regroups the float64 block sums of the sweeps; in this
    # variant (r0, r) is one of them, and its partials need not sum exactly.
    # 16-bit storage is compared at 4 cells per thread, the register form's
    # grouping of the float32 partial sums.)
    nx, ny, nz = shape
    raw = np.float64 if storage == "f64" else np.float32
    p = synth.varcoef(nx, ny, nz, seed=46, dtype=raw)
    tol = 1e-6 if storage in ("f32", "f64") else 1e-3
    outs = []
    for stages, by, kinds in ((1, 0, 0), (2, 0, 3), (3, 0, 1), (2, 0, 2), (4, 0, 3), (3, 0, 3)):
        with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage=storage, variant=1,
                                stages=stages, by=by, pipe_kinds=kinds,
                                step_cells=4 if storage in ("bf16", "f16") else 0) as op:
            outs.append(s7.bicgstab_solve(op, gu.to_dev(p.b), tol=tol, maxit=300))
    assert outs[0].status == 0
    for o in outs[1:]:
        assert o.iters == outs[0].iters and o.status == outs[0].status
        assert np.array_equal(o.hist, outs[0].hist)
        assert np.array_equal(o.x.cpu().numpy(), outs[0].x.cpu().numpy())


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16", "f16"])
@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("shape", [(64, 48, 40), (136, 21, 37), (8, 5, 70), (256, 8, 16)])
def test_tma_staging_equals_cp_async(s7, storage, variant, shape):
    """The pipelined sweeps staged by per-thread cp.async copies (the default)
    and by TMA tensor copies fill the same shared-memory tiles with the same
    values (zeros past the mesh edges), so the solves agree bit for bit:
    several x tiles, odd y extents, many z chunks, a tile wider than the
    mesh.  16-bit storage at 8 cells per thread (the width TMA applies to)."""
    nx, ny, nz = shape
    raw = np.float64 if storage == "f64" else np.float32
    p = synth.varcoef(nx, ny, nz, seed=48, dtype=raw)
    tol = 1e-6 if storage in ("f32", "f64") else 1e-3
    outs = []
    for tma in (False, True):
        with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage=storage,
                                variant=variant, zchunk=7, tma=tma) as op:
            outs.append(s7.bicgstab_solve(op, gu.to_dev(p.b), tol=tol, maxit=300))
    assert outs[0].status == 0
    assert outs[1].iters == outs[0].iters and outs[1].status == outs[0].status
    assert np.array_equal(outs[1].hist, outs[0].hist)
    assert np.array_equal(outs[1].x.cpu().numpy(), outs[0].x.cpu().numpy())


@pytest.mark.parametrize("storage", ["bf16", "f16"])
@pytest.mark.parametrize("variant", [0, 1])
def test_16bit_eight_cells_per_thread(s7, storage, variant):
    """The pipelined sweeps at 8 cells (16 bytes) per thread: the same
    method; only the grouping of the float32 partial sums changes, so the
    history agrees with the 4-cell form to the storage precision, the
    solution to what the tolerance allows, and a refined solve reaches
    1e-10 on the true operator."""
    nx, ny, nz = 64, 40, 36
    p = synth.varcoef(nx, ny, nz, seed=47)
    # plain solves stop above each format's plateau (bf16 stalls near 1e-3)
    tol = 1e-2 if storage == "bf16" else 1e-3
    res = {}
    for cells in (4, 8):
        with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage=storage,
                                keep_true=True, variant=variant, step_cells=cells) as op:
            r = s7.bicgstab_solve(op, gu.to_dev(p.b), tol=tol, maxit=200)
            again = s7.bicgstab_solve(op, gu.to_dev(p.b), tol=tol, maxit=200)
            assert np.array_equal(r.x.cpu().numpy(), again.x.cpu().numpy())
            rr = s7.bicgstab_solve_refined(op, gu.to_dev(p.b.astype(np.float64)), tol=1e-10,
                                           max_outer=40, inner_maxit=100, inner_tol=1e-2)
            assert rr.status == 0 and rr.hist[-1] <= 1e-10
            xr = rr.x.cpu().numpy()
            assert ob.true_residual(nx, ny, nz, p.coef, p.b.astype(np.float64), xr) <= 1.5e-10
            res[cells] = r
    a, b = res[4], res[8]
    assert a.status == b.status == 0 and abs(a.iters - b.iters) <= max(3, a.iters // 4)
    k = min(len(a.hist), len(b.hist), 6)
    u = 2.0 ** -8 if storage == "bf16" else 2.0 ** -11
    assert np.max(np.abs(a.hist[:k] - b.hist[:k]) / a.hist[:k]) < 50 * u
    assert rel(b.x.cpu().numpy(), a.x.cpu().numpy().astype(np.float64)) < 0.05


@pytest.mark.parametrize("storage", ["f64", "bf16", "f16"])
def test_pipeline_depth_other_storage(s7, storage):
    nx, ny, nz = 48, 20, 30
    raw = np.float64 if storage == "f64" else np.float32
    p = synth.varcoef(nx, ny, nz, seed=45, dtype=raw)
    outs = []
    for stages, kinds in ((1, 0), (2, 3), (3, 3), (2, 1)):
        # 4 cells per thread: the register form's grouping of partial sums
        with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage=storage,
                                stages=stages, pipe_kinds=kinds,
                                step_cells=4 if storage in ("bf16", "f16") else 0) as op:
            outs.append(s7.bicgstab_solve(op, gu.to_dev(p.b), tol=1e-3, maxit=60))
    for o in outs[1:]:
        assert o.iters == outs[0].iters
        assert np.array_equal(o.x.cpu().numpy(), outs[0].x.cpu().numpy())


def test_residual_entry_point(s7):
    nx, ny, nz = 26, 19, 15
    p = synth.varcoef(nx, ny, nz, seed=44)
    x = synth.random_vector(p.n, 9, 1, np.float32)
    ref = p.b.astype(np.float64) - stencil.apply(nx, ny, nz, p.coef, x.astype(np.float64))
    for keep in (True, False):
        with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage="f32",
                                keep_true=keep) as op:
            r = gu.to_dev(np.zeros(p.n, np.float32))
            rn, bn = s7.stencil7_residual(op, gu.to_dev(p.b), gu.to_dev(x), r)
            rr = r.cpu().numpy().astype(np.float64)
        den = stencil.abs_apply(nx, ny, nz, p.coef, x) + np.abs(p.b)
        tol = 1e-6 if keep else 1e-5     # without keep_true A is rebuilt from rounded A~ and d
        assert np.max(np.abs(rr - ref) / den) < tol
        assert rn == pytest.approx(np.linalg.norm(ref), rel=tol * 10)
        assert bn == pytest.approx(np.linalg.norm(p.b.astype(np.float64)), rel=1e-12)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_refined_solve_reaches_1e12(s7, storage):
    """The outer residual in double words (about 48 bits) still carries the
    refinement to 1e-12 relative, checked by the oracle's float64 residual."""
    nx, ny, nz = 40, 33, 29
    p = synth.varcoef(nx, ny, nz, seed=6)
    b64 = p.b.astype(np.float64)
    with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage=storage,
                            keep_true=True) as op:
        res = s7.bicgstab_solve_refined(op, gu.to_dev(b64), tol=1e-12, max_outer=60,
                                        inner_maxit=100, inner_tol=1e-2)
        x = res.x.cpu().numpy()
    assert res.status == 0 and res.hist[-1] <= 1e-12
    assert ob.true_residual(nx, ny, nz, p.coef, b64, x) <= 1.5e-12


@pytest.mark.parametrize("storage", ["bf16", "f16", "f32"])
def test_refined_solve_reaches_1e10(s7, storage):
    nx, ny, nz = 48, 40, 36
    p = synth.varcoef(nx, ny, nz, seed=2)
    b64 = p.b.astype(np.float64)
    # oracle: the same (float32-coefficient) system solved in float64
    orc = ob.bicgstab(nx, ny, nz, p.coef, b64, tol=1e-13, maxit=2000, storage="f64")
    with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage=storage,
                            keep_true=True) as op:
        res = s7.bicgstab_solve_refined(op, gu.to_dev(b64), tol=1e-10, max_outer=40,
                                        inner_maxit=100, inner_tol=1e-2)
        x = res.x.cpu().numpy()
    assert res.status == 0 and res.hist[-1] <= 1e-10
    assert ob.true_residual(nx, ny, nz, p.coef, b64, x) <= 1.5e-10
    assert rel(x, orc.x) < 1e-8


@pytest.mark.parametrize("keep_true", [True, False])
def test_double_word_residual_under_cancellation(s7, keep_true):
    """b = A x rounded to float32, so every residual entry b - A x is the
    rounding error of A x: about 1e-8 of the terms that cancel.  The residual
    sweeps sum the terms in double words (binary32 pairs); their error must
    stay within a few u^2 (u = 2^-24) of the terms' magnitude, where a lost
    low part anywhere would leave errors near u."""
    nx, ny, nz = 33, 20, 18
    p = synth.varcoef(nx, ny, nz, seed=31)
    x = synth.random_vector(p.n, 5, 2, np.float32)
    ax = stencil.apply(nx, ny, nz, p.coef, x.astype(np.float64))
    b = ax.astype(np.float32)
    ref = b.astype(np.float64) - ax
    mag = stencil.abs_apply(nx, ny, nz, p.coef, x) + np.abs(b)
    assert 1e-10 < np.median(np.abs(ref) / mag) < 1e-7   # cancellation, not zero
    with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage="f32",
                            keep_true=keep_true) as op:
        r64 = gu.to_dev(np.zeros(p.n))
        rn, bn = s7.stencil7_residual(op, gu.to_dev(b.astype(np.float64)),
                                      gu.to_dev(x.astype(np.float64)), r64)
        r32 = gu.to_dev(np.zeros(p.n, np.float32))
        rn32, _ = s7.stencil7_residual(op, gu.to_dev(b), gu.to_dev(x), r32)
    r64 = r64.cpu().numpy()
    if keep_true:
        # the raw operator as given: only the summation error remains
        assert np.max(np.abs(r64 - ref) / mag) < 2e-13
        assert rn == pytest.approx(np.linalg.norm(ref), rel=1e-5)
        r32 = r32.cpu().numpy().astype(np.float64)
        assert np.max(np.abs(r32 - ref) / (np.abs(ref) * 6e-8 + mag * 2e-13)) <= 1.0
    else:
        # A rebuilt as d * A~ with A~ rounded to float32: entries off by ~u
        assert np.max(np.abs(r64 - ref) / mag) < 1e-6
    assert rn32 == pytest.approx(rn, rel=1e-5 if keep_true else 1e-2)


def test_binary64_residual_option_under_cancellation(s7):
    """residual_f64 = 1 runs the same sweeps in binary64: the cancellation case
    then resolves to binary64 rounding of the terms (about 1e-16)."""
    nx, ny, nz = 33, 20, 18
    p = synth.varcoef(nx, ny, nz, seed=31)
    x = synth.random_vector(p.n, 5, 2, np.float32)
    ax = stencil.apply(nx, ny, nz, p.coef, x.astype(np.float64))
    b = ax.astype(np.float32)
    ref = b.astype(np.float64) - ax
    mag = stencil.abs_apply(nx, ny, nz, p.coef, x) + np.abs(b)
    with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage="f32", keep_true=True,
                            residual_f64=True) as op:
        r64 = gu.to_dev(np.zeros(p.n))
        rn, _ = s7.stencil7_residual(op, gu.to_dev(b.astype(np.float64)),
                                     gu.to_dev(x.astype(np.float64)), r64)
    assert np.max(np.abs(r64.cpu().numpy() - ref) / mag) < 2e-15
    assert rn == pytest.approx(np.linalg.norm(ref), rel=1e-9)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_true_residual_modes_agree(s7, storage):
    """The true residual a solve reports is the same quantity in both modes:
    double words and binary64 agree far below the solve's tolerance."""
    nx, ny, nz = 48, 36, 30
    p = synth.varcoef(nx, ny, nz, seed=13)
    out = []
    for f64 in (False, True):
        with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage=storage,
                                residual_f64=f64) as op:
            out.append(s7.bicgstab_solve(op, gu.to_dev(p.b), tol=1e-5, maxit=400))
    assert out[0].iters == out[1].iters
    assert np.array_equal(out[0].x.cpu().numpy(), out[1].x.cpu().numpy())
    assert out[0].true_resid == pytest.approx(out[1].true_resid, rel=1e-6)


def test_refined_solve_binary64_residuals(s7):
    nx, ny, nz = 40, 33, 29
    p = synth.varcoef(nx, ny, nz, seed=6)
    b64 = p.b.astype(np.float64)
    with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage="f16", keep_true=True,
                            residual_f64=True) as op:
        res = s7.bicgstab_solve_refined(op, gu.to_dev(b64), tol=1e-12, max_outer=60,
                                        inner_maxit=100, inner_tol=1e-2)
        x = res.x.cpu().numpy()
    assert res.status == 0 and res.hist[-1] <= 1e-12
    assert ob.true_residual(nx, ny, nz, p.coef, b64, x) <= 1.5e-12


def test_double_word_residual9_under_cancellation(s7):
    from oracle import stencil9
    nx, ny = 90, 61
    p = synth.varcoef9(nx, ny, seed=32)
    x = synth.random_vector(p.n, 6, 2, np.float32)
    ax = stencil9.apply(nx, ny, p.coef, x.astype(np.float64))
    b = ax.astype(np.float32)
    ref = b.astype(np.float64) - ax
    mag = stencil9.abs_apply(nx, ny, p.coef, x) + np.abs(b)
    with s7.stencil9_create(nx, ny, {k: gu.to_dev(v) for k, v in p.coef.items()},
                            storage="f32", keep_true=True) as op:
        r64 = gu.to_dev(np.zeros(p.n))
        s7.stencil7_residual(op, gu.to_dev(b.astype(np.float64)),
                             gu.to_dev(x.astype(np.float64)), r64)
    assert np.max(np.abs(r64.cpu().numpy() - ref) / mag) < 2e-13


@pytest.mark.parametrize("f64", [False, True])
def test_float64_residual_of_float32_data_is_exact(s7, f64):
    """The residual sweeps take float32 data exactly (double words whose low
    part is zero; products of two float32 numbers are exact double words), so
    the residual norm of float32 data matches the oracle's to the double-word
    summation error, special values (zero, subnormal, large) included."""
    nx, ny, nz = 64, 48, 40
    p = synth.varcoef(nx, ny, nz, seed=9)
    x = synth.random_vector(p.n, 3, 3, np.float32)
    x[:100] = 0.0
    x[100:200] = np.float32(1e-40)          # binary32 subnormal
    x[200:300] = np.float32(-2.5e30)        # large
    x[300:400] = np.float32(-0.0)
    ref = p.b.astype(np.float64) - stencil.apply(nx, ny, nz, p.coef, x.astype(np.float64))
    for keep in (True, False):
        with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage="f32",
                                keep_true=keep, residual_f64=f64) as op:
            r = gu.to_dev(np.zeros(p.n, np.float32))
            rn, bn = s7.stencil7_residual(op, gu.to_dev(p.b), gu.to_dev(x), r)
        if keep:
            assert rn == pytest.approx(np.linalg.norm(ref), rel=1e-13)
            rr = r.cpu().numpy().astype(np.float64)
            assert np.max(np.abs(rr - ref) / (np.abs(ref) + 1e-300)) <= 6e-8   # one rounding
        else:
            assert rn == pytest.approx(np.linalg.norm(ref), rel=1e-6)


def test_mixed_precision_plateau_and_refinement(s7):
    """Sec. VI-B analogue, against the FP64 oracle: plain BiCGStab with 16-bit
    storage first follows the oracle's history on the same stored operator,
    then stalls at a plateau set by the storage precision, and its solution
    error against the oracle's float64 solution of the true system is set by
    that precision; float64 refinement on the true operator reaches 1e-10 and
    the oracle's solution to 1e-8."""
    nx, ny, nz = 50, 100, 25
    p = synth.varcoef(nx, ny, nz, seed=4)
    b64 = p.b.astype(np.float64)
    # the true (float32-coefficient) system solved in float64 by the oracle
    x_ref = ob.bicgstab(nx, ny, nz, p.coef, b64, tol=1e-13, maxit=3000, storage="f64").x
    coef = gu.coef_on_device(p)
    b = gu.to_dev(p.b)
    h, err = {}, {}
    for storage in ("f32", "bf16", "f16"):
        with s7.stencil7_create(nx, ny, nz, coef, storage=storage, keep_true=True) as op:
            r = s7.bicgstab_solve(op, b, tol=1e-12, maxit=80)
            rn, bn = s7.stencil7_residual(op, b, r.x)
            h[storage] = (np.asarray(r.hist), rn / bn)
            err[storage] = rel(r.x.cpu().numpy(), x_ref)
            # the oracle's Algorithm 1 on the same stored operator: early steps
            orc = ob.bicgstab(nx, ny, nz, p.coef, p.b, tol=1e-12, maxit=6, storage=storage)
            assert np.max(np.abs(r.hist[:6] - orc.hist[:6]) / orc.hist[:6]) < 1e-3
            if storage != "f32":
                rr = s7.bicgstab_solve_refined(op, b.double(), tol=1e-10, max_outer=40,
                                               inner_maxit=100, inner_tol=1e-2)
                assert rr.status == 0 and rr.hist[-1] <= 1e-10
                assert ob.true_residual(nx, ny, nz, p.coef, b64, rr.x.cpu().numpy()) <= 1.5e-10
                assert rel(rr.x.cpu().numpy(), x_ref) < 1e-8
    f32 = h["f32"][0]
    for storage, floor in (("bf16", 1e-4), ("f16", 1e-6)):
        hist, true_raw = h[storage]
        # the first steps track float32 closely
        assert np.max(np.abs(hist[:4] - f32[:4]) / f32[:4]) < 0.05
        # the true residual stalls far above what float32 reaches
        assert true_raw > floor
        assert true_raw > 100 * h["f32"][1]
    # the solution error follows the storage precision
    assert err["f32"] <= 1e-4 and err["f32"] < err["f16"] < err["bf16"], err


def test_two_reduction_variant_fp64_matches_its_oracle(s7):
    """variant 1 (beta from the rho recurrence, fused passes) against the oracle's
    bicgstab_merged, and both against Algorithm 1's solution."""
    p = synth.convdiff_constant(32, 32, 32, seed=0)
    orc = ob.bicgstab_merged(32, 32, 32, p.coef, p.b, tol=1e-8, maxit=500)
    std = ob.bicgstab(32, 32, 32, p.coef, p.b, tol=1e-8, maxit=500)
    with s7.stencil7_create(32, 32, 32, p.coef, storage="f64", variant=1) as op:
        res = s7.bicgstab_solve(op, gu.to_dev(p.b), tol=1e-8, maxit=500)
    x = res.x.cpu().numpy()
    assert res.status == 0 and abs(res.iters - orc.iters) <= 3
    assert np.max(np.abs(res.hist[:15] - orc.hist[:15]) / orc.hist[:15]) < 1e-9
    assert rel(x, orc.x) < 1e-7 and rel(x, std.x) < 1e-7
    assert res.true_resid <= 1.01e-8
    nx, ny, nz = 45, 30, 26
    q = synth.varcoef(nx, ny, nz, seed=5, dtype=np.float64)
    orc = ob.bicgstab_merged(nx, ny, nz, q.coef, q.b, tol=1e-10, maxit=400)
    with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(q), storage="f64", variant=1) as op:
        res = s7.bicgstab_solve(op, gu.to_dev(q.b), tol=1e-10, maxit=400)
    # beta comes from a recurrence, not a reduction: near 1e-10 the step count
    # moves more than for Algorithm 1 (solution and true residual still hold)
    assert res.status == 0 and abs(res.iters - orc.iters) <= max(6, orc.iters // 6)
    assert np.max(np.abs(res.hist[:15] - orc.hist[:15]) / orc.hist[:15]) < 1e-9
    assert rel(res.x.cpu().numpy(), orc.x) < 1e-8
    assert res.true_resid <= 1.01e-10


@pytest.mark.parametrize("shape", [(64, 48, 40), (61, 37, 29), (17, 9, 33)])
def test_two_reduction_variant_fp32(s7, shape):
    nx, ny, nz = shape
    p = synth.varcoef(nx, ny, nz, seed=21)
    orc = ob.bicgstab(nx, ny, nz, p.coef, p.b, tol=1e-6, maxit=1000, storage="f32")
    with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage="f32", variant=1) as op:
        res = s7.bicgstab_solve(op, gu.to_dev(p.b), tol=1e-6, maxit=1000)
        again = s7.bicgstab_solve(op, gu.to_dev(p.b), tol=1e-6, maxit=1000)
    assert res.status == 0 and res.hist[-1] <= 1e-6
    assert abs(res.iters - orc.iters) <= max(6, orc.iters // 4)
    assert rel(res.x.cpu().numpy(), orc.x) <= 1e-4
    assert res.true_resid <= 2e-6
    assert again.iters == res.iters
    assert np.array_equal(again.x.cpu().numpy(), res.x.cpu().numpy())


def test_two_reduction_variant_degenerate_cases(s7):
    import torch
    nx, ny, nz = 20, 10, 12
    p = synth.varcoef(nx, ny, nz, seed=31, dtype=np.float64)
    with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage="f64", variant=1) as op:
        z = torch.zeros(p.n, dtype=torch.float64, device="cuda:0")
        r0 = s7.bicgstab_solve(op, z, tol=1e-8, maxit=10)
        assert r0.iters == 0 and r0.status == 0 and float(r0.x.abs().max()) == 0.0
        r2 = s7.bicgstab_solve(op, gu.to_dev(p.b), tol=1e-30, maxit=7)
        o2 = ob.bicgstab_merged(nx, ny, nz, p.coef, p.b, tol=1e-30, maxit=7)
        assert r2.status == s7.ENOTCONV and r2.iters == 7 and len(r2.hist) == 8
        assert np.max(np.abs(r2.hist - o2.hist) / o2.hist) < 1e-10
        r3 = s7.bicgstab_solve(op, gu.to_dev(p.b), tol=1e-8, maxit=0)
        assert r3.iters == 0 and r3.status == s7.ENOTCONV
    for ce in (1, 5):
        with s7.stencil7_create(nx, ny, nz, gu.coef_on_device(p), storage="f64", variant=1,
                                check_every=ce) as op:
            r = s7.bicgstab_solve(op, gu.to_dev(p.b), tol=1e-9, maxit=300)
            assert r.status == 0
