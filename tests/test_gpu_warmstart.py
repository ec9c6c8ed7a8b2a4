"""GPU warm-start network (tensor-core convolutions) against the FP64 oracle's plain loops."""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_08058_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sf():
    from paper_2212_08058_gb300 import build, sfseg
    build.build()
    oracle.build()
    return sfseg


def _bf16(a):
    return synth.to_bf16_round(np.asarray(a, dtype=np.float32)).astype(np.float64)


def _case(seed, C=8, T=3, H=37, W=140):
    rng = np.random.default_rng(seed)
    feats = rng.uniform(0.0, 1.0, size=(C, T, H, W)).astype(np.float32)
    return feats


def test_net_forward_matches_oracle(sf):
    """x0 of the 4-layer network (bf16 activations, fp32 accumulation on the tensor cores) equals
    the FP64 plain-loop network on the same bf16-rounded inputs and weights, within bf16
    rounding of the three hidden activations.  W = 140 spans two 128-voxel tiles, H = 37 two
    row ranges of 32."""
    feats = _case(1)
    net = sf.WarmStartNet(8, seed=3)
    p = net.get_params()
    x0 = net.forward(torch.from_numpy(feats).cuda()).cpu().numpy().astype(np.float64)
    params = [(_bf16(w), b.astype(np.float64)) for w, b in net.unflatten(p)]
    ref, _ = oracle.warmstart_forward(_bf16(feats), params)
    assert np.all(x0 > 0)
    err = np.abs(x0 - ref).max() / np.abs(ref).max()
    assert err < 3e-2, err
    # one voxel's value depends on its 9x9x9 neighbourhood only: check the corner explicitly
    assert abs(x0[0, 0, 0] - ref[0, 0, 0]) <= 3e-2 * np.abs(ref).max()
    net.close()


@pytest.mark.parametrize("T", [1, 2])
def test_net_forward_few_frames(sf, T):
    """One and two frames: the convolution's two-frame CTAs (one output frame at T = 1) and the
    last layer's frame groups with their zero-padded frames outside the volume."""
    feats = _case(10 + T, T=T, H=20, W=40)
    net = sf.WarmStartNet(8, seed=5)
    p = net.get_params()
    x0 = net.forward(torch.from_numpy(feats).cuda()).cpu().numpy().astype(np.float64)
    params = [(_bf16(w), b.astype(np.float64)) for w, b in net.unflatten(p)]
    ref, _ = oracle.warmstart_forward(_bf16(feats), params)
    assert x0.shape == (T, 20, 40) and np.all(x0 > 0)
    err = np.abs(x0 - ref).max() / np.abs(ref).max()
    assert err < 3e-2, err
    net.close()


def test_net_gradients_match_oracle(sf):
    """Parameter gradients of the cosine loss (tensor-core data gradients + weight-gradient
    reduction) against the FP64 reverse pass of the plain loops."""
    feats = _case(2, T=3, H=20, W=40)
    rng = np.random.default_rng(5)
    target = rng.uniform(0.1, 1.0, size=feats.shape[1:]).astype(np.float32)
    net = sf.WarmStartNet(8, seed=4)
    p = net.get_params()
    loss, g = net.backward(torch.from_numpy(feats).cuda(), torch.from_numpy(target).cuda(), want_grads=True)
    params = [(_bf16(w), b.astype(np.float64)) for w, b in net.unflatten(p)]
    lo, grads = oracle.warmstart_backward(_bf16(feats), params, target.astype(np.float64))
    assert abs(loss - lo) <= 1e-2 * max(lo, 1e-3)
    gl = net.unflatten(g)
    for li in range(4):
        for gi in range(2):
            ref = grads[li][gi]
            got = gl[li][gi].astype(np.float64)
            rel = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-12)
            assert rel < 5e-2, (li, gi, rel)
    net.close()


def test_net_training_reduces_loss(sf):
    """A few AdamW steps on one volume lower the cosine loss against its eigenvector."""
    V, _, w = synth.multichannel(8, 32, 48, C=8, seed=5001)
    feats = torch.from_numpy(V).cuda()
    with sf.PowerIteration(8, 8, 32, 48) as h:
        target = h.power_iterate(feats, w, 0.0, (2, 7, 7), iters=200)
    net = sf.WarmStartNet(8, seed=5)
    first = net.backward(feats, target)
    for _ in range(60):
        net.backward(feats, target)
        net.adamw(lr=3e-3)
    last = net.backward(feats, target)
    assert last < 0.7 * first, (first, last)
    net.close()


def test_warmstart_entry_point(sf):
    V, _, w = synth.multichannel(5, 24, 70, C=8, seed=5002)
    feats = torch.from_numpy(V).cuda().to(torch.bfloat16)
    net = sf.WarmStartNet(8, seed=6)
    with sf.PowerIteration(8, 5, 24, 70) as h:
        x0 = h.warmstart(net, feats)
        x1 = net.forward(feats)
        torch.cuda.synchronize()
        assert torch.equal(x0, x1)
        x = h.power_iterate(feats, w, 0.0, (1, 3, 3), iters=5, x=x0.clone(), init="user")
        assert torch.isfinite(x).all()
    net.close()


def test_trained_network_gain(sf):
    """What the trained network adds to the method without it, on generated volumes outside its
    training and hold-out sets (volume indices 4000+): its refinement of the coarse-to-fine start
    is closer to the eigenvector (cosine loss) than the coarse start alone, and from it the plain
    iteration reaches residual 1e-4 in no more steps.  Both beat the uniform start."""
    from paper_2212_08058_gb300 import warmstart
    C, T, H, W = 8, 16, 128, 128
    radius = (2, 7, 7)
    net = sf.WarmStartNet(C + 1)
    assert warmstart.load(net), "trained weights missing"
    w = synth.fixed_weights(C)

    def cos_loss(a, b):
        return float(1.0 - (a * b).sum() / (a.norm() * b.norm()))

    losses = {"coarse": [], "net": []}
    its = {"uniform": [], "coarse": [], "net": []}
    with sf.PowerIteration(C, T, H, W) as h:
        for i in range(4000, 4006):
            V = synth.training_volume_torch(i, T, H, W, C).to(torch.bfloat16)
            label = warmstart.make_label(h, V, w, radius)
            xc, _ = h.coarse_start(radius, levels=warmstart.COARSE_LEVELS_TRAIN, tol=warmstart.COARSE_TOL)
            xn = h.warmstart(net, V, xc)
            losses["coarse"].append(cos_loss(xc, label))
            losses["net"].append(cos_loss(xn, label))
            for name, x0, init in (("uniform", torch.empty_like(xc), "uniform"), ("coarse", xc, "user"),
                                   ("net", xn, "user")):
                _, n, res, _ = warmstart.iterate_to_residual(h, radius, x0.clone(), 1e-4, chunk=10, init=init)
                assert res <= 1e-4
                its[name].append(n)
    net.close()
    assert np.mean(losses["net"]) < 0.5 * np.mean(losses["coarse"]), losses
    assert sum(its["net"]) <= sum(its["coarse"]) < sum(its["uniform"]), its
