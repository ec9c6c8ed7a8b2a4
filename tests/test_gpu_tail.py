"""GPU soft-binarisation iterations (Alg. 1 step 3, Sec. 4.1) against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_08058_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5   # FP32 storage, on values in (0, 1)


@pytest.fixture(scope="module")
def sf():
    from paper_2212_08058_gb300 import build, sfseg
    build.build()
    oracle.build()
    return sfseg


def _check(x, mask, xo, margin):
    """x within TOL of the oracle; the mask is x > 1/2 of the GPU's own x, bit for bit, and
    equals the oracle's mask wherever the oracle's x is farther than `margin` from 1/2."""
    err = np.abs(x - xo).max()
    assert err < TOL, err
    np.testing.assert_array_equal(mask, (x > 0.5).astype(np.uint8))
    clear = np.abs(xo - 0.5) > margin
    np.testing.assert_array_equal(mask[clear], (xo[clear] > 0.5).astype(np.uint8))


@pytest.mark.parametrize("shape,radius,iters,gain,center", [
    ((8, 64, 64), (1, 3, 3), 3, 10.0, 0.5),     # TMA kernel
    ((5, 37, 70), (2, 7, 7), 2, 6.0, 0.35),     # TMA kernel, ragged tiles
    ((4, 20, 33), (1, 2, 3), 3, 12.0, 0.5),     # radius without a TMA kernel: generic stencil
    ((1, 1, 1), (1, 3, 3), 2, 4.0, 0.5),        # one voxel
])
def test_soft_binarize_matches_oracle(sf, shape, radius, iters, gain, center):
    T, H, W = shape
    if shape == (1, 1, 1):
        V = np.full((1, 1, 1, 1), 0.7, np.float32)
    else:
        V = synth.drifting_blob(T, H, W, seed=7100 + T)
    f = V[0].astype(np.float64)
    # the continuous solution both sides start from: 10 oracle iterations, rounded to float32
    xc, _ = oracle.power_filter(f, f, 0.3, 1.0, radius, np.ones(f.shape), 10)
    x0 = xc.astype(np.float32)
    with sf.PowerIteration(1, T, H, W, p=0.3) as h:
        h.set_features(torch.from_numpy(V).cuda())
        x, mask = h.soft_binarize(torch.from_numpy(x0).cuda(), radius, iters=iters, gain=gain, center=center)
        x, mask = x.cpu().numpy().astype(np.float64), mask.cpu().numpy()
    xo, _ = oracle.soft_binarize(f, f, 0.3, 1.0, radius, x0.astype(np.float64), iters, gain, center)
    _check(x, mask, xo, margin=1e-4)


def test_segment_end_to_end(sf):
    """Alg. 1 with C = 8 channels: 40 continuous iterations, then 4 soft-binarisation steps;
    against the oracle run from the oracle's own continuous solution."""
    V, gt, w = synth.multichannel(8, 48, 64, C=8, seed=7200)
    radius = (1, 3, 3)
    with sf.PowerIteration(8, 8, 48, 64) as h:
        x, mask = h.segment(torch.from_numpy(V).cuda(), w, 0.0, radius, n_iter=44, n_cont=40, gain=8.0)
        x, mask = x.cpu().numpy().astype(np.float64), mask.cpu().numpy()
    f = oracle.combine(V.astype(np.float64), w, 0.0)
    xc, _ = oracle.power_filter(f, f, 0.1, 1.0, radius, np.ones(f.shape), 40)
    xo, mo = oracle.soft_binarize(f, f, 0.1, 1.0, radius, xc, 4, 8.0, 0.5)
    _check(x, mask, xo, margin=1e-4)
    assert 0 < mask.sum() < mask.size


def test_soft_binarize_errors(sf):
    with sf.PowerIteration(1, 2, 8, 8) as h:
        x = torch.ones((2, 8, 8), device="cuda")
        with pytest.raises(sf.SFSegError) as e:
            h.soft_binarize(x, (1, 3, 3))
        assert e.value.status == "STATE"
        h.set_features(torch.rand((1, 2, 8, 8), device="cuda") + 0.1)
        for kw in ({"iters": 0}, {"gain": -1.0}, {"gain": float("inf")}, {"center": float("nan")}):
            with pytest.raises(sf.SFSegError):
                h.soft_binarize(x, (1, 3, 3), **kw)
        # features all zero: A x = 0, max(A x) = 0 -> ZERO_NORM, reported not hidden
        h.set_features(torch.zeros((1, 2, 8, 8), device="cuda"))
        with pytest.raises(sf.SFSegError) as e:
            h.soft_binarize(x, (1, 3, 3))
        assert e.value.status == "ZERO_NORM"
        # the handle stays usable
        h.set_features(torch.rand((1, 2, 8, 8), device="cuda") + 0.1)
        xs, m = h.soft_binarize(x, (1, 3, 3), iters=2)
        assert bool(((xs > 0) & (xs < 1)).all())
