"""A seeded sweep of small random problems against the FP64 oracle: volume shapes from one voxel
up to several tiles with ragged edges, the eight radii of the TMA kernel and others served by the
generic stencil, one or several channels (Eq. 9), float32 or bf16 features, a bf16 storage
phase, uniform and S_m starts, per-axis Gaussian widths and alpha, p away from the defaults.
Each case compares the unit-norm iterate (1e-5 with float32 storage, 2e-3 with a bf16 phase)
and the norms after a few iterations, and checks which kernel ran the steps."""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_08058_gb300 import synth

pytestmark = pytest.mark.gpu

TMA_RADII = [(1, 3, 3), (2, 7, 7), (1, 4, 4), (1, 2, 2), (1, 5, 5), (2, 3, 3), (2, 5, 5), (1, 7, 7)]
OTHER_RADII = [(0, 1, 1), (2, 2, 5), (3, 1, 0), (1, 8, 8), (4, 3, 2)]


@pytest.fixture(scope="module")
def sf():
    from paper_2212_08058_gb300 import build, sfseg
    build.build()
    oracle.build()
    return sfseg


def _case(i):
    rng = np.random.default_rng(9000 + i)
    T = int(rng.integers(1, 14))
    H = int(rng.choice([1, 2, 15, 16, 31, 47]))
    W = int(rng.choice([1, 7, 63, 64, 65, 130, 200]))
    radius = TMA_RADII[i % len(TMA_RADII)] if i % 3 else OTHER_RADII[(i // 3) % len(OTHER_RADII)]
    C = int(rng.choice([1, 1, 3]))
    V = rng.uniform(0.0, 1.0, size=(C, T, H, W)).astype(np.float32)
    w = rng.normal(size=C).astype(np.float32) * 2.0 if C > 1 else None
    sigma = None if i % 2 else tuple(float(s) for s in rng.uniform(0.6, 3.0, size=3))
    alpha = float(rng.choice([1.0, 0.5]))
    p = float(rng.choice([0.1, 0.3]))
    iters = int(rng.integers(1, 7))
    bf16_feats = bool(i % 5 == 1)
    iters_bf16 = int(rng.integers(1, iters + 1)) if i % 4 == 2 else 0
    init = "smap" if i % 3 == 1 else "uniform"
    return dict(V=V, w=w, radius=radius, sigma=sigma, alpha=alpha, p=p, iters=iters, bf16_feats=bf16_feats,
                iters_bf16=iters_bf16, init=init)


@pytest.mark.parametrize("i", range(30))
def test_random_case(sf, i):
    c = _case(i)
    V, w, radius, iters = c["V"], c["w"], c["radius"], c["iters"]
    C, T, H, W = V.shape
    Vr = synth.to_bf16_round(V) if c["bf16_feats"] else V
    feats = torch.from_numpy(V).cuda()
    if c["bf16_feats"]:
        feats = feats.to(torch.bfloat16)
    sigma = c["sigma"] if c["sigma"] is not None else sf.default_sigma(radius)
    tma0, gen0, _ = sf.iterate_kernel_stats()
    with sf.PowerIteration(C, T, H, W, alpha=c["alpha"], p=c["p"]) as h:
        x, nu = h.power_iterate(feats, w, 0.0, radius, sigma, iters, c["iters_bf16"], init=c["init"],
                                return_norms=True)
        x = x.cpu().numpy().astype(np.float64)
    tma1, gen1, name = sf.iterate_kernel_stats()
    f = oracle.combine(Vr.astype(np.float64), w, 0.0)
    start = f if c["init"] == "smap" else np.ones(f.shape)
    xo, nuo = oracle.power_filter(f, f, c["p"], c["alpha"], radius, start, iters, sigma=sigma)
    tol = 2e-3 if c["iters_bf16"] else 1e-5
    assert np.abs(x - xo).max() <= tol, (c["radius"], (C, T, H, W), float(np.abs(x - xo).max()))
    np.testing.assert_allclose(nu, nuo, rtol=2e-3 if c["iters_bf16"] else 1e-5)
    if radius in TMA_RADII:
        assert gen1 == gen0 and tma1 - tma0 == iters and name.startswith("iter_fast"), (name, tma1 - tma0)
    else:
        assert gen1 - gen0 == iters and name.startswith("stream_stencil")
