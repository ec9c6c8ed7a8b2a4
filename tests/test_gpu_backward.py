"""GPU adjoint of the unrolled power iteration (learning the Eq. 9 weights, Sec. 3.4) against
the FP64 oracle: its reverse-mode gradient on small volumes, and FP64 finite differences of the
oracle's forward pass at the sizes of the learning workload."""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_08058_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2212_08058_gb300 import build
    build.build()
    oracle.build()


def _sf():
    from paper_2212_08058_gb300 import sfseg
    return sfseg


def _gpu_grad(V, w, b, radius, K, every, grad_fn, p=0.1, alpha=1.0):
    """Forward with checkpoints, dL/dx_K from grad_fn(x_K), then the library's adjoint."""
    sf = _sf()
    C, T, H, W = V.shape
    with sf.PowerIteration(C, T, H, W, alpha=alpha, p=p) as h:
        feats = torch.from_numpy(np.ascontiguousarray(V)).cuda()
        x = h.power_iterate(feats, w, b, radius, iters=K, record_every=every)
        g = grad_fn(h, x)
        gw, gb = h.backward(g, radius)
        return x.cpu().numpy().astype(np.float64), gw.astype(np.float64), gb


@pytest.mark.parametrize("K,every,r", [(6, 2, (1, 2, 2)), (6, 4, (1, 2, 2)), (5, 5, (1, 2, 2)), (1, 3, (1, 2, 2)),
                                        (6, 2, (1, 3, 3)), (5, 5, (2, 7, 7)), (4, 2, (2, 3, 3)), (3, 3, (1, 5, 5)),
                                        (3, 2, (1, 1, 2))])
def test_adjoint_matches_oracle_gradient(K, every, r):
    """Linear loss <c, x_K>: the GPU adjoint equals the oracle's reverse pass on the explicit
    Eq. 2 matrix (4 x 12 x 12, C = 2), for several checkpoint spacings (K a multiple of the
    spacing, not one, and below it); radii with a TMA kernel ((1,2,2), (1,3,3), (2,7,7), (2,3,3),
    (1,5,5): the reverse pass in the stencil's state form) and without ((1,1,2): the six-signal
    stencil)."""
    V, _, _ = synth.multichannel(4, 12, 12, C=2, seed=4001)
    w = np.array([1.4, -0.7], dtype=np.float32)
    b = 0.1
    rng = np.random.default_rng(11)
    c = rng.normal(size=V.shape[1:]).astype(np.float32)
    _, gw, gb = _gpu_grad(V, w, b, r, K, every, lambda h, x: torch.from_numpy(c).cuda())
    gwo, gbo = oracle.grad_csr(V.astype(np.float64), w.astype(np.float64), b, 0.1, 1.0, r,
                               np.ones(V[0].size), K, c.astype(np.float64))
    scale = max(np.abs(gwo).max(), abs(gbo))
    assert np.abs(gw - gwo).max() <= 2e-4 * scale
    assert abs(gb - gbo) <= 2e-4 * scale


def test_soft_iou_loss_matches_oracle():
    sf = _sf()
    V = synth.drifting_blob(6, 40, 52, seed=1003)
    tgt = (synth.drifting_blob_mask(6, 40, 52) > 0.5).astype(np.float32)
    with sf.PowerIteration(1, 6, 40, 52) as h:
        x = h.power_iterate(torch.from_numpy(V).cuda(), radius=(1, 3, 3), iters=8)
        loss, g = h.soft_iou_loss(x, torch.from_numpy(tgt).cuda())
        xr = x.cpu().numpy().astype(np.float64)
        g = g.cpu().numpy()
    lo, go = oracle.soft_iou_loss(xr, tgt.astype(np.float64))
    assert abs(loss - lo) <= 1e-6
    assert np.abs(g.reshape(-1) - go).max() <= 1e-5 * np.abs(go).max()


def _fd_loss(V, w, b, radius, K, tgt):
    f = oracle.combine(V.astype(np.float64), w, b)
    x, _ = oracle.power_filter(f, f, 0.1, 1.0, radius, np.ones(f.shape), K)
    return oracle.soft_iou_loss(x, tgt)[0]


def test_adjoint_matches_finite_differences_fd_size():
    """C = 2, 8 x 32 x 32, radius (1, 3, 3), 30 iterations, checkpoint every 5, soft-IoU loss:
    GPU gradient vs FP64 central differences of the oracle's forward pass."""
    V, m, _ = synth.multichannel(8, 32, 32, C=2, seed=4002)
    w = np.array([2.0, 1.0])
    b = -1.0
    tgt = (m > 0.5).astype(np.float64)
    r, K = (1, 3, 3), 30

    def grad_fn(h, x):
        _, g = h.soft_iou_loss(x, torch.from_numpy(tgt.astype(np.float32)).cuda())
        return g

    _, gw, gb = _gpu_grad(V, w.astype(np.float32), b, r, K, 5, grad_fn)
    eps = 1e-5
    fd = []
    for c in range(2):
        wp, wm = w.copy(), w.copy()
        wp[c] += eps
        wm[c] -= eps
        fd.append((_fd_loss(V, wp, b, r, K, tgt) - _fd_loss(V, wm, b, r, K, tgt)) / (2 * eps))
    fdb = (_fd_loss(V, w, b + eps, r, K, tgt) - _fd_loss(V, w, b - eps, r, K, tgt)) / (2 * eps)
    scale = max(np.abs(fd).max(), abs(fdb))
    assert np.abs(gw - np.array(fd)).max() <= 1e-3 * scale, (gw, fd)
    assert abs(gb - fdb) <= 1e-3 * scale, (gb, fdb)


def test_adjoint_directional_derivative_full_size():
    """The differentiation workload: C = 8 float32, 32 x 240 x 427, 30 unrolled iterations,
    checkpoint every 5, loss 1 - soft-IoU against the noiseless blob mask.  The GPU gradient,
    projected on a random direction of (w, b), equals the FP64 central difference of the
    oracle's forward pass along that direction."""
    T, H, W = 32, 240, 427
    V, m, w = synth.multichannel(T, H, W, C=8, seed=4003)
    w = (w * 8.0).astype(np.float64)
    b = -2.0
    tgt = (m > 0.5).astype(np.float64)
    r, K = (1, 3, 3), 30

    def grad_fn(h, x):
        _, g = h.soft_iou_loss(x, torch.from_numpy(tgt.astype(np.float32)).cuda())
        return g

    _, gw, gb = _gpu_grad(V, w.astype(np.float32), b, r, K, 5, grad_fn)
    rng = np.random.default_rng(12)
    d = rng.normal(size=9)
    d /= np.linalg.norm(d)
    eps = 1e-4
    lp = _fd_loss(V, w + eps * d[:8], b + eps * d[8], r, K, tgt)
    lm = _fd_loss(V, w - eps * d[:8], b - eps * d[8], r, K, tgt)
    fd = (lp - lm) / (2 * eps)
    ana = float(np.dot(np.append(gw, gb), d))
    assert abs(ana - fd) <= 2e-3 * max(abs(fd), np.abs(np.append(gw, gb)).max()), (ana, fd)


def test_autograd_function():
    """torch.autograd through SFSegFunction gives the same weight gradient as the direct call."""
    sf = _sf()
    V, m, w0 = synth.multichannel(6, 24, 40, C=3, seed=4004)
    tgt = torch.from_numpy((m > 0.5).astype(np.float32)).cuda()
    feats = torch.from_numpy(V).cuda()
    with sf.PowerIteration(3, 6, 24, 40) as h:
        w = torch.tensor(w0 * 3.0, requires_grad=True)
        b = torch.tensor(-1.0, requires_grad=True)
        x = sf.sfseg_pp(w, b, feats, h, radius=(1, 3, 3), iters=10, record_every=5)
        xs = x / x.max()
        inter = (xs * tgt).sum()
        loss = 1.0 - inter / (xs + tgt - xs * tgt).sum()
        loss.backward()
        x2 = h.power_iterate(feats, w.detach().numpy(), -1.0, (1, 3, 3), iters=10, record_every=5)
        _, g = h.soft_iou_loss(x2, tgt)
        gw, gb = h.backward(g, (1, 3, 3))
    np.testing.assert_allclose(w.grad.numpy(), gw, rtol=1e-3, atol=1e-6)
    assert abs(b.grad.item() - gb) <= 1e-3 * max(1.0, abs(gb))


def test_adjoint_with_the_maximum_channel_count():
    """C = 64 (the largest the handle takes): every weight's gradient against the oracle's
    reverse pass (each channel's gradient lands in its own slot of the handle's scratch)."""
    rng = np.random.default_rng(13)
    C, T, H, W = 64, 2, 8, 9
    V = rng.uniform(0.0, 1.0, size=(C, T, H, W)).astype(np.float32)
    w = (rng.normal(size=C) * 0.3).astype(np.float32)
    c = rng.normal(size=(T, H, W)).astype(np.float32)
    r = (1, 1, 2)
    _, gw, gb = _gpu_grad(V, w, -0.2, r, 4, 2, lambda h, x: torch.from_numpy(c).cuda())
    gwo, gbo = oracle.grad_csr(V.astype(np.float64), w.astype(np.float64), -0.2, 0.1, 1.0, r,
                               np.ones(V[0].size), 4, c.astype(np.float64))
    scale = max(np.abs(gwo).max(), abs(gbo))
    assert np.abs(gw - gwo).max() <= 2e-4 * scale
    assert abs(gb - gbo) <= 2e-4 * scale


def test_adjoint_graph_replay_is_identical():
    """sfseg_backward replayed from a captured CUDA graph (sfseg_enable_graphs) gives the same
    weight gradients as direct launches (to the order of the FP64 atomic sums), over repeated forward/backward calls with new loss
    gradients under the same pointers."""
    sf = _sf()
    V, _, w = synth.multichannel(6, 40, 70, C=4, seed=4010)
    feats = torch.from_numpy(V).cuda()
    rng = np.random.default_rng(21)
    outs = {}
    for on in (False, True):
        with sf.PowerIteration(4, 6, 40, 70) as h:
            h.enable_graphs(on)
            g = torch.empty((6, 40, 70), device="cuda")
            res = []
            for rep in range(3):
                x = h.power_iterate(feats, w, 0.2, (1, 3, 3), iters=12, record_every=4)
                g.copy_(torch.from_numpy(rng.normal(size=(6, 40, 70)).astype(np.float32) if not on else
                                         outs["g"][rep]))
                if not on:
                    outs.setdefault("g", []).append(g.cpu().numpy().copy())
                gw, gb = h.backward(g, (1, 3, 3))
                res.append((gw.copy(), gb))
            outs[on] = res
    # the FP64 sums are accumulated with atomics, so their order (not the arithmetic) may differ
    for (a, ab), (b, bb) in zip(outs[False], outs[True]):
        np.testing.assert_allclose(a, b, rtol=1e-6, atol=1e-9 * np.abs(a).max())
        assert abs(ab - bb) <= 1e-6 * max(abs(ab), np.abs(a).max())
