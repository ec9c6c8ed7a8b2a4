"""GPU online form (Sec. 4.5 partial iterations on a frame stream) against the FP64 oracle."""
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


def _unit(a):
    return a / np.linalg.norm(a)


@pytest.mark.parametrize("C,T,H,W,q,radius,iters", [
    (1, 9, 40, 70, 4, (1, 3, 3), 6),      # TMA kernel, ragged tiles; window fills after 4 frames
    (8, 7, 24, 33, 3, (2, 7, 7), 4),      # C = 8 (Eq. 9 sigmoid), radius wider than the window's frames
    (1, 5, 20, 20, 1, (1, 2, 2), 5),      # q = 1: every frame alone; generic stencil
    (1, 4, 16, 16, 3, (1, 3, 3), 0),      # no iterations: the start vectors themselves
])
def test_online_matches_oracle(sf, C, T, H, W, q, radius, iters):
    if C == 1:
        V = synth.drifting_blob(T, H, W, seed=7300 + T)
        w = None
    else:
        V, _, w = synth.multichannel(T, H, W, C=C, seed=7301)
    ref = oracle.online(V.astype(np.float64), w, 0.0, 0.1, 1.0, radius, q, iters)
    with sf.OnlineStream(C, q, H, W) as st:
        Vd = torch.from_numpy(np.ascontiguousarray(V)).cuda()
        for k in range(T):
            lag = min(k, q - 1)
            out = st.push(Vd[:, k].contiguous(), w, 0.0, radius, iters=iters, lag=lag).cpu().numpy()
            win = st.window().cpu().numpy().astype(np.float64)
            # the whole window (unit norm on both sides) and the returned slice
            assert np.abs(win - ref[k]).max() < TOL, (k, np.abs(win - ref[k]).max())
            np.testing.assert_array_equal(out, win[q - 1 - lag].astype(np.float32))


def test_online_full_window_matches_offline(sf):
    """When the window spans the whole video (q = T), the last push runs the offline method on
    the whole volume from the stream's start vector: many iterations reach the offline
    eigenvector of the same volume (sfseg_power_iterate from the uniform start)."""
    T, H, W = 6, 32, 48
    V = synth.drifting_blob(T, H, W, seed=7310)
    Vd = torch.from_numpy(V).cuda()
    with sf.OnlineStream(1, T, H, W) as st:
        for k in range(T):
            st.push(Vd[:, k].contiguous(), radius=(1, 3, 3), iters=1500 if k == T - 1 else 3)
        win = st.window()
    with sf.PowerIteration(1, T, H, W) as h:
        x = h.power_iterate(Vd, radius=(1, 3, 3), iters=1500)
    assert float((win - x).abs().max()) < 1e-5


def test_online_errors(sf):
    with pytest.raises(sf.SFSegError):
        sf.OnlineStream(1, 0, 8, 8)
    with sf.OnlineStream(1, 3, 8, 8) as st:
        fr = torch.rand((1, 8, 8), device="cuda")
        with pytest.raises(sf.SFSegError):
            st.push(fr, radius=(1, 3, 3), lag=3)
        with pytest.raises(sf.SFSegError):
            st.push(fr, radius=(1, 3, 3), iters=-1)
        out = st.push(fr, radius=(1, 3, 3), iters=2)
        assert bool(torch.isfinite(out).all())
