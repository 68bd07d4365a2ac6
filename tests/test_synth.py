"""The seeded input generator: reproducibility, sampled access and the
value distributions the workloads ask for (CPU only)."""

import numpy as np

import synth


def test_splitmix64_reference_values():
    # SplitMix64 started from state 0: the first outputs of the published
    # generator (state += GAMMA; then the mix64 finaliser)
    key0 = np.uint64(0)
    with np.errstate(over="ignore"):
        w = synth._mix(key0 + np.arange(1, 4, dtype=np.uint64) * synth.GAMMA)
    assert [int(v) for v in w] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_counter_access_matches_sequential():
    a = synth.uniform(5, 1, 1000, 300000)
    b = synth.uniform_at(5, 1, np.arange(1000, 301000))
    assert np.array_equal(a, b)
    assert 0.0 <= a.min() and a.max() < 1.0
    assert abs(a.mean() - 0.5) < 0.003


def test_varcoef_distribution_and_dominance():
    p = synth.varcoef(17, 9, 33, seed=0)
    offs = np.stack([p.coef[d].astype(np.float64) for d in synth.DIRS])
    assert offs.min() >= -1.5 and offs.max() <= -0.5
    margin = p.coef["diag"].astype(np.float64) - np.abs(offs).sum(0)
    assert margin.min() > 0.0099 and margin.max() < 0.1001
    assert abs(p.b.mean()) < 0.08 and abs(p.b.std() - 1) < 0.05   # 5 sigma at n = 5049


def test_varcoef_at_matches_full():
    p = synth.varcoef(31, 7, 5, seed=4)
    idx = np.array([0, 1, 100, 999, p.n - 1])
    c, b = synth.varcoef_at(31, 7, 5, idx, seed=4)
    for d in synth.DIRS + ("diag",):
        assert np.array_equal(c[d], p.coef[d][idx])
    assert np.array_equal(b, p.b[idx])


def test_convdiff_constant_recipe():
    p = synth.convdiff_constant(32, 32, 32, seed=0)
    assert p.coef["diag"] == 6.1
    for a in "xyz":
        m, q = p.coef[a + "m"], p.coef[a + "p"]
        assert -1.3 <= m <= -1.0 and -1.0 <= q <= -0.7
        assert abs((m + q) + 2.0) < 1e-12
    assert -1 <= p.b.min() and p.b.max() < 1


def test_batched_and_request_streams():
    e = synth.batched_edges()
    assert len(e) == 512 and min(e) >= 16 and max(e) <= 128
    reqs = synth.request_stream(200, rate=50.0)
    assert all(32 <= r.nx <= 384 for r in reqs)
    assert all(r.tol in (1e-4, 1e-6, 1e-8) for r in reqs)
    t = [r.arrival for r in reqs]
    assert all(b > a for a, b in zip(t, t[1:]))
    assert len({r.seed for r in reqs}) == 200
