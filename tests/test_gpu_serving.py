"""The solve server: continuous batching of refined BF16 solves.

Checks: every request meets its own tolerance on the true float32 operator
(float64 residual, recomputed by the oracle from the returned x); a request
gives the same result alone and in a mix of concurrently running requests
(its arithmetic is independent of the batch); admission never exceeds the
memory budget; waits are bounded; destroying a busy server cancels cleanly.
"""

import time

import numpy as np
import pytest

import synth
from oracle import bicgstab as ob
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def s7():
    import paper_2010_03660_gb300 as m
    m.lib()
    return m


REQS = [((40, 32, 28), 1e-8), ((24, 50, 20), 1e-6), ((64, 30, 16), 1e-4), ((17, 23, 40), 1e-8),
        ((48, 48, 48), 1e-6), ((9, 70, 11), 1e-8), ((36, 20, 44), 1e-4)]


def problems(seed0):
    return [synth.varcoef(nx, ny, nz, seed=seed0 + j) for j, ((nx, ny, nz), _) in enumerate(REQS)]


def submit(srv, p, tol):
    x = np.zeros(p.n, np.float64)
    return srv.submit(p.nx, p.ny, p.nz, p.coef, p.b.astype(np.float64), x, tol)


def test_requests_meet_tolerance_and_match_oracle(s7):
    probs = problems(500)
    with s7.Server(storage="bf16") as srv:
        ids = [submit(srv, p, tol) for p, (_, tol) in zip(probs, REQS)]
        for rid, p, (_, tol) in zip(ids, probs, REQS):
            r = srv.wait(rid, timeout=120)
            assert r["status"] == 0, r
            x = srv.result(rid)
            b = p.b.astype(np.float64)
            assert r["resid"] <= tol
            tr = ob.true_residual(p.nx, p.ny, p.nz, p.coef, b, x)
            assert tr <= tol * 1.01, (tr, tol)
            assert r["t_arrive"] <= r["t_admit"] <= r["t_done"]
            if tol <= 1e-8:
                ref = ob.bicgstab(p.nx, p.ny, p.nz, p.coef, b, tol=1e-12, maxit=3000)
                assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) < 1e-5
        st = srv.stats()
        assert st["completed"] == len(REQS) and st["failed"] == 0


def test_alone_and_in_the_mix(s7):
    probs = problems(600)
    target = 3
    with s7.Server(storage="bf16") as srv:
        rid = submit(srv, probs[target], REQS[target][1])
        srv.wait(rid, timeout=120)
        alone = srv.release(rid).copy()
        # the same request again, arriving while others are already running,
        # followed by more arrivals
        ids = [submit(srv, p, tol) for p, (_, tol) in list(zip(probs, REQS))[:3]]
        time.sleep(0.02)
        mine = submit(srv, probs[target], REQS[target][1])
        ids += [submit(srv, p, tol) for p, (_, tol) in list(zip(probs, REQS))[4:]]
        r = srv.wait(mine, timeout=120)
        for i in ids:
            assert srv.wait(i, timeout=120)["status"] == 0
        mixed = srv.result(mine)
        assert r["status"] == 0
        # within the request's tolerance, and in fact bit for bit
        assert np.linalg.norm(mixed - alone) / np.linalg.norm(alone) <= REQS[target][1]
        assert np.array_equal(mixed, alone)


def test_admission_respects_budget(s7):
    probs = problems(700)
    sizes = [p.n for p in probs]
    # about two average requests fit at once (bytes per held cell as the
    # server counts them: bf16 storage, eight Krylov vectors, float32 raw
    # coefficients)
    per_cell = 6 * 2 + 4 + 28 + 8 * 2 + 8 + 24 + 32
    budget = int(2.2 * np.mean(sizes) * per_cell) + (4 << 20)
    budget = max(budget, int(max(sizes) * per_cell) + (2 << 20))
    with s7.Server(storage="bf16", hbm_budget_bytes=budget) as srv:
        ids = [submit(srv, p, 1e-6) for p in probs]
        for i in ids:
            assert srv.wait(i, timeout=300)["status"] == 0
        st = srv.stats()
        assert st["mem_peak"] <= budget
        assert st["completed"] == len(probs)
    # a request larger than the whole budget is refused at submission
    with s7.Server(storage="bf16", hbm_budget_bytes=1 << 20) as srv:
        with pytest.raises(s7.S7Error) as e:
            submit(srv, probs[0], 1e-6)
        assert e.value.code == s7.ENOMEM


def test_bounded_wait_and_cancel(s7):
    p = synth.varcoef(96, 96, 96, seed=800)
    srv = s7.Server(storage="bf16")
    rid = submit(srv, p, 1e-10)
    with pytest.raises(s7.S7Error) as e:
        srv.wait(rid, timeout=0.0)          # host-side bounded wait
    assert e.value.code == s7.ETIMEOUT
    others = [submit(srv, p, 1e-10) for _ in range(3)]
    srv.close()                              # running and queued requests are cancelled
    assert others


@pytest.mark.parametrize("three_pass,f64", [(False, False), (True, False), (False, True)])
def test_constant_and_padded_requests_both_forms(s7, three_pass, f64):
    """A constant-coefficient request (expanded to per-cell arrays) and
    requests whose x extent is padded to whole vectors, with the inner steps
    in either form and the outer residuals in double words or binary64: each
    meets its tolerance on the true operator, and the padding leaves the
    solution on the real cells unchanged (oracle)."""
    cases = [synth.convdiff_constant(21, 13, 17, seed=0, dtype=np.float32),
             synth.varcoef(9, 31, 26, seed=901), synth.varcoef(35, 12, 30, seed=902)]
    with s7.Server(storage="f16", three_pass=three_pass, residual_f64=f64) as srv:
        ids = []
        for p in cases:
            coef = p.coef
            if p.constant:
                coef = {k: np.array([v], dtype=np.float32) for k, v in p.coef.items()}
            ids.append(srv.submit(p.nx, p.ny, p.nz, coef, p.b.astype(np.float64),
                                  np.zeros(p.n, np.float64), 1e-8))
        for rid, p in zip(ids, cases):
            r = srv.wait(rid, timeout=120)
            assert r["status"] == 0, r
            x = srv.result(rid)
            b = p.b.astype(np.float64)
            assert ob.true_residual(p.nx, p.ny, p.nz, p.coef, b, x) <= 1.01e-8
            ref = ob.bicgstab(p.nx, p.ny, p.nz, p.coef, b, tol=1e-12, maxit=3000)
            assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) < 1e-5
