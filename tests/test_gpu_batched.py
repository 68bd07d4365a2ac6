"""GPU parity of bicgstab_solve_batched.

Each system of a batch runs Algorithm 1 with its own grid combine, scalars
and stop flag, so (i) every system matches the FP64 oracle at its own
tolerance, (ii) with a fixed launch policy a system's result is bitwise the
same alone and inside any batch, and (iii) the batch of 512 systems of
log-uniform cube edges 16..128 converges system by system.
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


SHAPES = [(16, 16, 16), (17, 9, 33), (40, 31, 25), (1, 1, 50), (24, 24, 24), (5, 7, 3),
          (64, 20, 12), (33, 33, 8), (8, 8, 64), (3, 1, 1), (28, 19, 22), (1, 12, 1)]


def make(shapes, seed0):
    return [synth.varcoef(nx, ny, nz, seed=seed0 + j) for j, (nx, ny, nz) in enumerate(shapes)]


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def scaled_true_residual(p, x, storage="f32"):
    """||b~ - A~ x|| / ||b~|| on the system a solve iterates on: the Jacobi-scaled
    operator rounded to the storage type, in float64 (the oracle)."""
    sc = stencil.jacobi_scale(p.nx, p.ny, p.nz, p.coef, storage)
    bt = stencil.scale_rhs(p.nx, p.ny, p.nz, p.coef, p.b)
    r = bt - stencil.apply(p.nx, p.ny, p.nz, sc, np.asarray(x, dtype=np.float64))
    return float(np.linalg.norm(r) / np.linalg.norm(bt))


def test_batched_matches_oracle_per_system(s7):
    probs = make(SHAPES, 100)
    tols = [1e-6 if j % 3 else 1e-5 for j in range(len(probs))]
    ops = [s7.stencil7_create(p.nx, p.ny, p.nz, gu.coef_on_device(p), storage="f32")
           for p in probs]
    try:
        bs = [gu.to_dev(p.b) for p in probs]
        res = s7.bicgstab_solve_batched(ops, bs, tol=tols, maxit=1000)
        assert all(st == 0 for st in res.status), res.status
        for j, p in enumerate(probs):
            orc = ob.bicgstab(p.nx, p.ny, p.nz, p.coef, p.b, tol=tols[j], maxit=1000,
                              storage="f32")
            x = res.x[j].cpu().numpy()
            assert res.resid[j] <= tols[j]
            # the bars of a single-system float32 solve: step count within the
            # float32 rounding window, x within 100 tol, true residual of the
            # solved (scaled, stored) system within 2 tol
            lo, hi = gu.fp32_step_window(p.nx, p.ny, p.nz, p.coef, p.b, tols[j], 1000, orc.iters)
            assert lo <= res.iters[j] <= hi, (j, res.iters[j], lo, hi, orc.iters)
            assert rel(x, orc.x) <= 100 * tols[j], (j, rel(x, orc.x))
            assert scaled_true_residual(p, x) <= 2 * tols[j], (j, scaled_true_residual(p, x))
    finally:
        for op in ops:
            op.close()


def test_alone_and_in_the_mix_are_identical(s7):
    probs = make(SHAPES, 200)
    ops = [s7.stencil7_create(p.nx, p.ny, p.nz, gu.coef_on_device(p), storage="f32")
           for p in probs]
    try:
        kw = dict(tol=1e-7, maxit=500, threads=128, zchunk=16)
        mix = s7.bicgstab_solve_batched(ops, [gu.to_dev(p.b) for p in probs], **kw)
        for j in (0, 2, 5, 9):
            alone = s7.bicgstab_solve_batched([ops[j]], [gu.to_dev(probs[j].b)], **kw)
            assert alone.iters[0] == mix.iters[j]
            assert alone.status[0] == mix.status[j]
            assert np.array_equal(alone.x[0].cpu().numpy(), mix.x[j].cpu().numpy())
        # a different subset and order
        sub = [7, 1, 4]
        part = s7.bicgstab_solve_batched([ops[j] for j in sub],
                                         [gu.to_dev(probs[j].b) for j in sub], **kw)
        for k, j in enumerate(sub):
            assert np.array_equal(part.x[k].cpu().numpy(), mix.x[j].cpu().numpy())
    finally:
        for op in ops:
            op.close()


def test_batched_deterministic_and_autotuned(s7):
    probs = make(SHAPES[:6], 300)
    ops = [s7.stencil7_create(p.nx, p.ny, p.nz, gu.coef_on_device(p), storage="f32")
           for p in probs]
    try:
        a = s7.bicgstab_solve_batched(ops, [gu.to_dev(p.b) for p in probs], tol=1e-6)
        b = s7.bicgstab_solve_batched(ops, [gu.to_dev(p.b) for p in probs], tol=1e-6)
        assert a.iters == b.iters
        for xa, xb in zip(a.x, b.x):
            assert np.array_equal(xa.cpu().numpy(), xb.cpu().numpy())
    finally:
        for op in ops:
            op.close()


def test_batched_mixed_limits_and_host_buffers(s7):
    probs = make(SHAPES[:5], 400)
    ops = [s7.stencil7_create(p.nx, p.ny, p.nz, p.coef, storage="f32") for p in probs]
    try:
        # maxit 0, 3 (not converged), and converged systems in one batch
        res = s7.bicgstab_solve_batched(ops, [p.b.copy() for p in probs], tol=1e-6,
                                        maxit=[0, 3, 500, 500, 2])
        assert res.rc == s7.ENOTCONV
        assert res.iters[0] == 0 and res.status[0] == s7.ENOTCONV
        assert res.iters[1] == 3 and res.status[1] == s7.ENOTCONV
        assert res.status[2] == 0 and res.status[3] == 0
        assert res.iters[4] == 2
        single = s7.bicgstab_solve(ops[2], probs[2].b.copy(), tol=1e-6, maxit=500)
        assert abs(single.iters - res.iters[2]) <= 3
        assert rel(res.x[2], single.x.astype(np.float64)) <= 1e-4
        # duplicate handle rejected
        with pytest.raises(s7.S7Error):
            s7.bicgstab_solve_batched([ops[0], ops[0]], [probs[0].b, probs[0].b])
    finally:
        for op in ops:
            op.close()


def test_config4_512_systems(s7):
    """512 systems, cube edges log-uniform in [16,128] (seed 1), FP32, tol 1e-6."""
    import torch
    edges = synth.batched_edges(512, seed=1)
    ops, bs, probs, diags = [], [], [], []
    try:
        for j, e in enumerate(edges):
            p = synth.varcoef(e, e, e, seed=synth.system_seed(1, j))
            ops.append(s7.stencil7_create(e, e, e, gu.coef_on_device(p), storage="f32"))
            bs.append(gu.to_dev(p.b))
            diags.append(gu.to_dev(p.coef["diag"].astype(np.float64)))
            if j % 97 == 0:
                probs.append((j, p))
        res = s7.bicgstab_solve_batched(ops, bs, tol=1e-6, maxit=2000)
        assert res.rc == 0 and all(s == 0 for s in res.status)
        assert max(res.resid) <= 1e-6
        # spot-check systems against the oracle, with the single-system bars
        for j, p in probs:
            orc = ob.bicgstab(p.nx, p.ny, p.nz, p.coef, p.b, tol=1e-6, maxit=2000, storage="f32")
            x = res.x[j].cpu().numpy()
            assert rel(x, orc.x) <= 1e-4
            lo, hi = gu.fp32_step_window(p.nx, p.ny, p.nz, p.coef, p.b, 1e-6, 2000, orc.iters,
                                         orders=4)
            assert lo <= res.iters[j] <= hi, (j, res.iters[j], lo, hi, orc.iters)
            assert scaled_true_residual(p, x) <= 2e-6
        # every system's true residual of the scaled system b~ - A~ x =
        # D^-1 (b - A x): the raw residual from the GPU's float64-accuracy
        # sweep, divided by the diagonal (test-side, on the device)
        worst = 0.0
        for j, op in enumerate(ops):
            r = torch.empty_like(bs[j], dtype=torch.float64)
            s7.stencil7_residual(op, bs[j].double(), res.x[j].double(), r)
            bt = bs[j].double() / diags[j]
            worst = max(worst, float(torch.linalg.norm(r / diags[j]) / torch.linalg.norm(bt)))
        assert worst <= 2e-6, worst
    finally:
        for op in ops:
            op.close()
        torch.cuda.empty_cache()


def test_pipelined_batch_matches_register_batch(s7):
    """A batch whose systems all have whole-vector rows runs the pipelined
    step sweeps; one ragged system sends the whole batch to the register
    sweeps.  In float32 the two give the same bits (same arithmetic and
    order, 4 cells per thread either way)."""
    aligned = [(16, 12, 20), (40, 31, 25), (64, 20, 12), (8, 8, 64)]
    probs = make(aligned + [(17, 9, 33)], 500)
    ops = [s7.stencil7_create(p.nx, p.ny, p.nz, gu.coef_on_device(p), storage="f32")
           for p in probs]
    try:
        kw = dict(tol=1e-7, maxit=500, threads=128, zchunk=16)
        piped = s7.bicgstab_solve_batched(ops[:4], [gu.to_dev(p.b) for p in probs[:4]], **kw)
        mixed = s7.bicgstab_solve_batched(ops, [gu.to_dev(p.b) for p in probs], **kw)
        assert all(s == 0 for s in piped.status)
        for j in range(4):
            assert piped.iters[j] == mixed.iters[j]
            assert np.array_equal(piped.x[j].cpu().numpy(), mixed.x[j].cpu().numpy())
            orc = ob.bicgstab(probs[j].nx, probs[j].ny, probs[j].nz, probs[j].coef, probs[j].b,
                              tol=1e-7, maxit=500, storage="f32")
            assert rel(piped.x[j].cpu().numpy(), orc.x) <= 1e-3
    finally:
        for op in ops:
            op.close()


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_pipelined_16bit_batch(s7, storage):
    """16-bit batches with rows of whole 8-cell vectors run the 8-cell
    pipelined sweeps; their results agree with the register sweeps of a
    ragged batch to what the storage precision allows, and each system
    meets its tolerance."""
    aligned = [(16, 12, 20), (40, 31, 25), (64, 20, 12)]
    probs = make(aligned + [(17, 9, 33)], 600)
    ops = [s7.stencil7_create(p.nx, p.ny, p.nz, gu.coef_on_device(p), storage=storage)
           for p in probs]
    try:
        kw = dict(tol=1e-2, maxit=300, threads=128, zchunk=16)
        piped = s7.bicgstab_solve_batched(ops[:3], [gu.to_dev(p.b) for p in probs[:3]], **kw)
        mixed = s7.bicgstab_solve_batched(ops, [gu.to_dev(p.b) for p in probs], **kw)
        for j in range(3):
            p = probs[j]
            assert piped.status[j] == 0 and mixed.status[j] == 0
            assert piped.resid[j] <= 1e-2
            assert abs(piped.iters[j] - mixed.iters[j]) <= max(3, mixed.iters[j] // 4)
            # the true residual of each x on the stored (scaled) operator
            sc = stencil.jacobi_scale(p.nx, p.ny, p.nz, p.coef, storage)
            bt = stencil.scale_rhs(p.nx, p.ny, p.nz, p.coef, p.b)
            for res in (piped, mixed):
                x = res.x[j].cpu().numpy().astype(np.float64)
                tr = np.linalg.norm(bt - stencil.apply(p.nx, p.ny, p.nz, sc, x)) / np.linalg.norm(bt)
                assert tr <= 3e-2, (j, tr)
    finally:
        for op in ops:
            op.close()


@pytest.mark.parametrize("storage,shapes", [
    ("f32", SHAPES),                                              # ragged: register sweeps
    ("f32", [(16, 16, 16), (24, 20, 12), (32, 9, 30), (8, 8, 64)]),   # whole rows: pipelined
    ("bf16", [(16, 16, 16), (24, 20, 12), (32, 9, 30), (8, 8, 64)]),
])
def test_batched_two_reduction_variant(s7, storage, shapes):
    """Handles created with variant 1 run the two-reduction form in the batch:
    every system matches the oracle's form of that variant at its tolerance,
    and alone or in the mix it gives the same bits (fixed launch policy)."""
    probs = make(shapes, 300)
    tol = 1e-6 if storage == "f32" else 1e-2
    ops = [s7.stencil7_create(p.nx, p.ny, p.nz, gu.coef_on_device(p), storage=storage,
                              variant=1) for p in probs]
    try:
        kw = dict(tol=tol, maxit=1000, threads=128, zchunk=16)
        res = s7.bicgstab_solve_batched(ops, [gu.to_dev(p.b) for p in probs], **kw)
        assert all(st == 0 for st in res.status), res.status
        for j, p in enumerate(probs):
            orc = ob.bicgstab_merged(p.nx, p.ny, p.nz, p.coef, p.b, tol=tol, maxit=1000,
                                     storage=storage)
            x = res.x[j].cpu().numpy()
            assert res.resid[j] <= tol
            win = max(6, orc.iters // 4) if storage == "f32" else max(10, orc.iters // 2)
            assert abs(res.iters[j] - orc.iters) <= win, j
            if storage == "f32":
                assert rel(x, orc.x) <= 100 * tol, (j, rel(x, orc.x))
                assert scaled_true_residual(p, x) <= 2 * tol
        alone = s7.bicgstab_solve_batched([ops[1]], [gu.to_dev(probs[1].b)], **kw)
        assert alone.iters[0] == res.iters[1]
        assert np.array_equal(alone.x[0].cpu().numpy(), res.x[1].cpu().numpy())
    finally:
        for op in ops:
            op.close()


def test_batched_variants_must_agree(s7):
    probs = make([(12, 10, 8), (9, 9, 9)], 400)
    ops = [s7.stencil7_create(p.nx, p.ny, p.nz, gu.coef_on_device(p), storage="f32",
                              variant=j) for j, p in enumerate(probs)]
    try:
        with pytest.raises(s7.S7Error) as e:
            s7.bicgstab_solve_batched(ops, [gu.to_dev(p.b) for p in probs], tol=1e-6, maxit=100)
        assert e.value.code == s7.EINVAL
    finally:
        for op in ops:
            op.close()


@pytest.mark.parametrize("storage,variant", [("f32", 0), ("f32", 1), ("bf16", 1)])
def test_persistent_launch_matches_launch_per_kernel(s7, storage, variant):
    """One persistent launch (resident blocks claiming tiles from per-system
    work queues) and one launch per step kernel: both meet the single-system
    bars against the oracle (the update's partial sums are grouped by the
    launch's block size, so the two are not the same bits, and float32 step
    counts move with such regroupings); in the persistent launch a system's
    result is the same bits alone and in the mix."""
    shapes = SHAPES if storage == "f32" else [(16, 16, 16), (24, 20, 12), (32, 9, 30), (8, 8, 64)]
    probs = make(shapes, 800)
    tol = 1e-6 if storage == "f32" else 1e-2
    ops = [s7.stencil7_create(p.nx, p.ny, p.nz, gu.coef_on_device(p), storage=storage,
                              variant=variant) for p in probs]
    try:
        kw = dict(tol=tol, maxit=1000, threads=128, zchunk=16)
        per = s7.bicgstab_solve_batched(ops, [gu.to_dev(p.b) for p in probs], schedule=1, **kw)
        lpk = s7.bicgstab_solve_batched(ops, [gu.to_dev(p.b) for p in probs], schedule=-1, **kw)
        for j, p in enumerate(probs):
            assert per.status[j] == 0 and lpk.status[j] == 0
            if storage != "f32":
                assert rel(per.x[j].cpu().numpy(), lpk.x[j].cpu().numpy().astype(np.float64)) <= 0.1
                continue
            orc = (ob.bicgstab_merged if variant else ob.bicgstab)(
                p.nx, p.ny, p.nz, p.coef, p.b, tol=tol, maxit=1000, storage="f32")
            lo, hi = gu.fp32_step_window(p.nx, p.ny, p.nz, p.coef, p.b, tol, 1000, orc.iters)
            if variant:   # beta from the rho recurrence: the window of that variant's tests
                lo, hi = orc.iters - max(6, orc.iters // 4), orc.iters + max(6, orc.iters // 4)
            for res in (per, lpk):
                x = res.x[j].cpu().numpy()
                assert lo <= res.iters[j] <= hi, (j, res.iters[j], lo, hi)
                assert rel(x, orc.x) <= 100 * tol
                assert scaled_true_residual(p, x) <= 2 * tol
        alone = s7.bicgstab_solve_batched([ops[2]], [gu.to_dev(probs[2].b)], schedule=1, **kw)
        assert alone.iters[0] == per.iters[2]
        assert np.array_equal(alone.x[0].cpu().numpy(), per.x[2].cpu().numpy())
    finally:
        for op in ops:
            op.close()


def test_persistent_wait_bound_gives_timeout(s7):
    """A wait budget of one cycle: the first block of the persistent launch
    that finds every open tile taken gives up at once and aborts the launch;
    the solve returns S7_ETIMEOUT with the unfinished systems' status, no
    wait outlives its budget, and the device stays usable (the same batch
    then solves normally)."""
    probs = make([(64, 64, 48), (40, 31, 25)], 900)
    ops = [s7.stencil7_create(p.nx, p.ny, p.nz, gu.coef_on_device(p), storage="f32")
           for p in probs]
    try:
        kw = dict(tol=1e-6, maxit=500, threads=128, zchunk=16, schedule=1)
        res = s7.bicgstab_solve_batched(ops, [gu.to_dev(p.b) for p in probs], wait_cycles=1,
                                        allow_timeout=True, **kw)
        assert res.rc == s7.ETIMEOUT
        assert res.status[0] == s7.ETIMEOUT
        ok = s7.bicgstab_solve_batched(ops, [gu.to_dev(p.b) for p in probs], **kw)
        assert ok.rc == 0 and all(st == 0 for st in ok.status)
    finally:
        for op in ops:
            op.close()


def test_autotuner_picks_fusion_schedule(s7):
    """Without a fixed block shape the autotuner also times the fusion
    schedules (the persistent launch or one launch per step kernel, the
    pipelined step sweeps or the register sweeps) over a few steps of the solve
    from x0, and puts x0 back before solving: the solve is bit for bit an
    explicit-policy solve with the block shape and schedule it reports (in
    float32 the pipelined and register sweeps give the same bits), and every
    system, started from a nonzero x0, meets the oracle bars."""
    probs = make([(16, 12, 20), (40, 31, 24), (64, 20, 12), (8, 8, 64), (32, 32, 32)], 1000)
    ops = [s7.stencil7_create(p.nx, p.ny, p.nz, gu.coef_on_device(p), storage="f32")
           for p in probs]
    x0 = [(0.3 * np.cos(0.01 * np.arange(p.nx * p.ny * p.nz))).astype(p.b.dtype) for p in probs]
    tol = 1e-6
    try:
        def solve(**kw):
            return s7.bicgstab_solve_batched(ops, [gu.to_dev(p.b) for p in probs],
                                             xs=[gu.to_dev(v) for v in x0], tol=tol, maxit=1000,
                                             **kw)
        auto = solve()
        pol = auto.policy
        assert pol["schedule"] in (1, -1) and pol["pipelined"] in (0, 1) and pol["variant"] == 0
        assert pol["threads"] in (64, 128, 256) and pol["zchunk"] in (16, 32, 64)
        again = solve()
        assert again.policy == pol and again.iters == auto.iters
        fixed = solve(threads=pol["threads"], zchunk=pol["zchunk"], schedule=pol["schedule"])
        assert fixed.iters == auto.iters
        for j, p in enumerate(probs):
            xa = auto.x[j].cpu().numpy()
            assert np.array_equal(xa, fixed.x[j].cpu().numpy())
            assert np.array_equal(xa, again.x[j].cpu().numpy())
            assert auto.status[j] == 0
            orc = ob.bicgstab(p.nx, p.ny, p.nz, p.coef, p.b, x0=x0[j].astype(np.float64),
                              tol=tol, maxit=1000, storage="f32")
            assert rel(xa, orc.x) <= 100 * tol
            assert scaled_true_residual(p, xa) <= 2 * tol
    finally:
        for op in ops:
            op.close()


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_autotuner_may_choose_the_variant(s7, storage):
    """With choose_variant the autotuner times both variants of the step (the
    handles were created with Algorithm 1) and runs the faster; either way
    each system meets the bars of the variant it ran."""
    shapes = [(16, 16, 16), (24, 20, 12), (32, 9, 30), (8, 8, 64), (48, 40, 24)]
    probs = make(shapes, 1100)
    tol = 1e-6 if storage == "f32" else 1e-2
    ops = [s7.stencil7_create(p.nx, p.ny, p.nz, gu.coef_on_device(p), storage=storage)
           for p in probs]
    try:
        res = s7.bicgstab_solve_batched(ops, [gu.to_dev(p.b) for p in probs], tol=tol,
                                        maxit=1000, choose_variant=True)
        pol = res.policy
        assert pol["variant"] in (0, 1) and pol["schedule"] in (1, -1)
        for j, p in enumerate(probs):
            assert res.status[j] == 0 and res.resid[j] <= tol
            x = res.x[j].cpu().numpy().astype(np.float64)
            assert scaled_true_residual(p, x, storage) <= (2 * tol if storage == "f32" else 3e-2)
            if storage == "f32":
                orc = (ob.bicgstab_merged if pol["variant"] else ob.bicgstab)(
                    p.nx, p.ny, p.nz, p.coef, p.b, tol=tol, maxit=1000, storage="f32")
                assert rel(x, orc.x) <= 100 * tol
    finally:
        for op in ops:
            op.close()
