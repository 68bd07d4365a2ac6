"""The device-side generator draws the host generator's systems: coefficients
bit for bit, b to one unit in the last place of float32 in rare cells
(device libm)."""

import numpy as np
import pytest

import synth
from synth import device as sd

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,seed", [((37, 29, 23), 5), ((64, 1, 1), 0), ((3, 5, 7), 123456789)])
def test_device_generator_matches_host(shape, seed):
    import torch
    nx, ny, nz = shape
    p = synth.varcoef(nx, ny, nz, seed=seed)
    coef, b = sd.varcoef(nx, ny, nz, seed, torch.device("cuda:0"))
    for k in synth.DIRS + ("diag",):
        assert np.array_equal(coef[k].cpu().numpy().view(np.uint32), p.coef[k].view(np.uint32)), k
    bd = b.cpu().numpy()
    assert np.array_equal(bd.astype(np.float32).astype(np.float64), bd)   # float32 values
    ulp = np.abs(bd.astype(np.float32).view(np.int32).astype(np.int64) -
                 p.b.view(np.int32).astype(np.int64))
    assert ulp.max() <= 1 and np.mean(ulp) <= 1e-3


def test_device_generator_large_sampled():
    """A 512 x 512 x 64 mesh, checked at sampled cells against varcoef_at."""
    import torch
    nx, ny, nz = 512, 512, 64
    coef, b = sd.varcoef(nx, ny, nz, 2, torch.device("cuda:0"), b_dtype="f32")
    idx = np.random.default_rng(0).integers(0, nx * ny * nz, 20000)
    c_at, b_at = synth.varcoef_at(nx, ny, nz, idx, seed=2)
    it = torch.from_numpy(idx).cuda()
    for k in synth.DIRS + ("diag",):
        assert np.array_equal(coef[k][it].cpu().numpy(), c_at[k]), k
    ulp = np.abs(b[it].cpu().numpy().view(np.int32).astype(np.int64) -
                 b_at.view(np.int32).astype(np.int64))
    assert ulp.max() <= 1
