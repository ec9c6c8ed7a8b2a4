"""The package's usage example, run as written on a small volume: every entry point it shows
returns what its description says (shapes, unit norm, the residual, the autograd path, the online
stream), and the first call agrees with the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sf():
    from paper_2212_08058_gb300 import build, sfseg
    build.build()
    oracle.build()
    return sfseg


def test_usage_example(sf):
    C, T, H, W = 8, 8, 48, 96
    gen = torch.Generator(device="cuda").manual_seed(21)
    feats = torch.rand((C, T, H, W), device="cuda", generator=gen)      # soft masks / features in [0, 1]
    w = [0.125] * C                                                   # Eq. 9 channel weights

    with sf.PowerIteration(C, T, H, W, alpha=1.0, p=0.1) as h:
        x = h.power_iterate(feats, w, 0.0, radius=(2, 7, 7), iters=50)
        rho, residual = h.rayleigh(x, (2, 7, 7))
        soft, mask = h.segment(feats, w, 0.0, radius=(2, 7, 7), n_iter=60, n_cont=50)
        x0, _ = h.coarse_start((2, 7, 7))
        x1 = h.power_iterate(None, radius=(2, 7, 7), iters=100, x=x0, init="user")
        xe = h.power_iterate_exact((2, 7, 7), iters=100)
        rho1, _ = h.rayleigh(x1, (2, 7, 7))
        torch.cuda.synchronize()

    assert x.shape == (T, H, W) and abs(float(x.double().norm()) - 1.0) < 1e-5 and bool((x >= 0).all())
    f = oracle.combine(feats.double().cpu().numpy(), np.array(w, dtype=np.float64), 0.0)
    ref, _ = oracle.power_filter(f, f, 0.1, 1.0, (2, 7, 7), np.ones((T, H, W)), 50)
    assert float(np.abs(x.double().cpu().numpy() - ref).max()) <= 1e-5
    assert rho > 0 and 0 <= residual < 1
    assert soft.shape == (T, H, W) and mask.shape == (T, H, W)
    assert bool(((soft > 0) & (soft < 1)).all())
    assert x0.shape == (T, H, W) and bool(torch.isfinite(x0).all())
    assert abs(float(x1.double().norm()) - 1.0) < 1e-5
    assert abs(float(xe.double().norm()) - 1.0) < 1e-5
    # the same operator's Rayleigh quotient (Eq. 3) from two starts agrees
    assert abs(rho1 - rho) <= 1e-2 * rho

    # learning the channel weights through the hand-written adjoint
    weights = torch.tensor(w, device="cuda", requires_grad=True)
    bias = torch.zeros((), device="cuda", requires_grad=True)
    with sf.PowerIteration(C, T, H, W) as h:
        xl = sf.sfseg_pp(weights, bias, feats, h, radius=(1, 3, 3), iters=30, record_every=5)
        xl.sum().backward()
    assert weights.grad is not None and weights.grad.shape == (C,) and bool(torch.isfinite(weights.grad).all())
    assert bias.grad is not None and bool(torch.isfinite(bias.grad))

    # online form: a sub-window of the 13 most recent frames
    with sf.OnlineStream(1, 13, H, W) as stream:
        for k in range(T):
            frame_solution = stream.push(feats[:1, k].contiguous(), radius=(2, 7, 7), iters=10)
            assert frame_solution.shape == (H, W) and bool(torch.isfinite(frame_solution).all())
