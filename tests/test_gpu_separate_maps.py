"""GPU power iteration with separate unary and pairwise maps (Eq. 9 with its two channel sets,
Alg. 1 lines 1-2) against the FP64 oracle, whose Eq. 2 / Eq. 7 forms take s and f separately."""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_08058_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def sf():
    from paper_2212_08058_gb300 import build, sfseg
    build.build()
    oracle.build()
    return sfseg


def _maps(T, H, W, Cs, Cf, seed):
    Vs, _, ws = synth.multichannel(T, H, W, C=Cs, seed=seed)
    Vf, _, wf = synth.multichannel(T, H, W, C=Cf, seed=seed + 1)
    if Cs == 1:
        ws = None
    return Vs, ws, Vf, wf


@pytest.mark.parametrize("T,H,W,Cs,Cf,radius,iters,init", [
    (6, 40, 70, 3, 5, (1, 3, 3), 12, "uniform"),    # TMA kernel, separate-map variant
    (5, 37, 70, 1, 4, (2, 7, 7), 8, "smap"),        # single unary channel (no sigmoid); S_m start
    (4, 20, 33, 2, 2, (1, 2, 3), 10, "uniform"),    # generic stencil
])
def test_separate_maps_match_oracle(sf, T, H, W, Cs, Cf, radius, iters, init):
    Vs, ws, Vf, wf = _maps(T, H, W, Cs, Cf, 7400 + T)
    s = oracle.combine(Vs.astype(np.float64), ws, 0.3)
    f = oracle.combine(Vf.astype(np.float64), wf, -0.2)
    x0 = s if init == "smap" else np.ones(s.shape)
    xo, nuo = oracle.power_filter(s, f, 0.2, 1.0, radius, x0, iters)
    with sf.PowerIteration(Cf, T, H, W, p=0.2) as h:
        h.set_features_sf(torch.from_numpy(Vs).cuda(), ws, 0.3, torch.from_numpy(Vf).cuda(), wf, -0.2)
        x, nu = h.power_iterate(None, radius=radius, iters=iters, init=init, return_norms=True)
        x = x.cpu().numpy().astype(np.float64)
        assert np.abs(x - xo).max() < TOL
        np.testing.assert_allclose(nu, nuo, rtol=1e-5)
        # y = A x and the Eq. 3 residual use the same separate maps
        y = h.apply(torch.from_numpy(xo.astype(np.float32)).cuda(), radius).cpu().numpy()
        yo = oracle.filter_apply(s, f, 0.2, 1.0, radius, xo.astype(np.float32).astype(np.float64))
        assert np.abs(y - yo).max() < 1e-5 * np.abs(yo).max()
        # shared maps again after set_features: back to s = f
        h.set_features(torch.from_numpy(Vf).cuda(), wf, -0.2)
        x2 = h.power_iterate(None, radius=radius, iters=iters).cpu().numpy().astype(np.float64)
        x2o, _ = oracle.power_filter(f, f, 0.2, 1.0, radius, np.ones(f.shape), iters)
        assert np.abs(x2 - x2o).max() < TOL


def test_separate_maps_soft_binarize(sf):
    T, H, W = 5, 30, 64
    Vs, ws, Vf, wf = _maps(T, H, W, 2, 3, 7450)
    s = oracle.combine(Vs.astype(np.float64), ws, 0.0)
    f = oracle.combine(Vf.astype(np.float64), wf, 0.0)
    xc, _ = oracle.power_filter(s, f, 0.1, 1.0, (1, 3, 3), np.ones(s.shape), 15)
    x0 = xc.astype(np.float32)
    xo, _ = oracle.soft_binarize(s, f, 0.1, 1.0, (1, 3, 3), x0.astype(np.float64), 3, 8.0, 0.5)
    with sf.PowerIteration(3, T, H, W) as h:
        h.set_features_sf(torch.from_numpy(Vs).cuda(), ws, 0.0, torch.from_numpy(Vf).cuda(), wf, 0.0)
        x, mask = h.soft_binarize(torch.from_numpy(x0).cuda(), (1, 3, 3), iters=3, gain=8.0)
    assert np.abs(x.cpu().numpy() - xo).max() < TOL


def test_separate_maps_unsupported_paths(sf):
    T, H, W = 4, 16, 16
    Vs, ws, Vf, wf = _maps(T, H, W, 2, 2, 7460)
    with sf.PowerIteration(2, T, H, W) as h:
        h.set_features_sf(torch.from_numpy(Vs).cuda(), ws, 0.0, torch.from_numpy(Vf).cuda(), wf, 0.0)
        with pytest.raises(sf.SFSegError) as e:
            h.coarse_start((1, 3, 3))
        assert e.value.status == "UNSUPPORTED"
        with pytest.raises(sf.SFSegError) as e:
            h.power_iterate(None, radius=(1, 3, 3), iters=4, record_every=2)
        assert e.value.status == "UNSUPPORTED"
