"""GPU coarse-to-fine start (sfseg_coarse_start) against a plain restatement built on the FP64
oracle: block means of f, the Eq. 7 + Eq. 8 iteration on the coarse volume (oracle), trilinear
upsampling with half-pixel centres.  Iteration counts are fixed (tol tiny, check_every =
max_iters) so both sides run the same number of steps."""
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


def _pool(f):
    """Mean of f over the in-volume part of each 2x2x2 block (factor 1 on axes of extent 1)."""
    T, H, W = f.shape
    p = [2 if n > 1 else 1 for n in (T, H, W)]
    Tc, Hc, Wc = [(n + q - 1) // q for n, q in zip((T, H, W), p)]
    s = np.zeros((Tc, Hc, Wc))
    n = np.zeros((Tc, Hc, Wc))
    for a in range(p[0]):
        for b in range(p[1]):
            for c in range(p[2]):
                blk = f[a::p[0], b::p[1], c::p[2]]
                s[:blk.shape[0], :blk.shape[1], :blk.shape[2]] += blk
                n[:blk.shape[0], :blk.shape[1], :blk.shape[2]] += 1
    return s / n, p


def _upsample(xc, p, shape):
    """Trilinear interpolation, source coordinate (d + 0.5)/p - 0.5 clamped to [0, n_c - 1]."""
    out = xc
    for ax, (q, n) in enumerate(zip(p, shape)):
        nc = out.shape[ax]
        if q == 1:
            idx = np.minimum(np.arange(n), nc - 1)
            out = np.take(out, idx, axis=ax)
            continue
        src = np.clip((np.arange(n) + 0.5) / q - 0.5, 0.0, nc - 1)
        i0 = np.floor(src).astype(int)
        i1 = np.minimum(i0 + 1, nc - 1)
        wgt = (src - i0).reshape([-1 if a == ax else 1 for a in range(3)])
        out = np.take(out, i0, axis=ax) * (1 - wgt) + np.take(out, i1, axis=ax) * wgt
    return out


def _coarse_nb(radius, sigma, scale):
    r = [0 if ri == 0 else max(1, int(np.floor(ri / s + 0.5))) for ri, s in zip(radius, scale)]
    return tuple(r), tuple(si / s for si, s in zip(sigma, scale))


def _reference(f, p, radius, sigma, levels, K):
    """x0 the coarse-to-fine start computes, levels coarser by 2 each, K steps per level."""
    fs, facs = [f], []
    for _ in range(levels):
        fc, q = _pool(fs[-1])
        fs.append(fc)
        facs.append(q)
    scale = [1.0, 1.0, 1.0]
    nbs = []
    for q in facs:
        scale = [s * qi for s, qi in zip(scale, q)]
        nbs.append(_coarse_nb(radius, sigma, scale))
    x = None
    for l in range(levels - 1, -1, -1):
        fl = fs[l + 1]
        start = np.ones_like(fl) if x is None else _upsample(x, facs[l + 1], fl.shape)
        r, sg = nbs[l]
        x, _ = oracle.power_filter(fl, fl, p, 1.0, r, start, K, sigma=sg)
    return _upsample(x, facs[0], f.shape)


@pytest.mark.parametrize("shape,radius,levels", [
    ((6, 40, 70), (2, 7, 7), 1),      # ragged W, several (fine) tiles
    ((5, 37, 70), (1, 3, 3), 2),      # odd T, H and W on both levels
    ((1, 33, 65), (0, 4, 4), 2),      # single frame: no pooling along t
    ((8, 64, 64), (2, 7, 7), 3),
])
def test_coarse_start_matches_reference(sf, shape, radius, levels):
    T, H, W = shape
    rng = np.random.default_rng(sum(shape) + levels)
    f = rng.uniform(0.05, 1.0, size=shape).astype(np.float32)
    K = 12
    sigma = oracle.default_sigma(radius)
    with sf.PowerIteration(1, T, H, W, p=0.5) as h:
        h.set_features(torch.from_numpy(f[None]).cuda())
        x0, its = h.coarse_start(radius, levels=levels, tol=1e-30, max_iters=K, check_every=K)
        x0 = x0.cpu().numpy().astype(np.float64)
    assert its == [K] * levels
    ref = _reference(f.astype(np.float64), 0.5, radius, sigma, levels, K)
    a = x0 / np.linalg.norm(x0)
    b = ref / np.linalg.norm(ref)
    err = np.abs(a - b).max() / np.abs(b).max()
    assert err < 1e-5, err


def test_coarse_start_cuts_fine_iterations(sf):
    """From the coarse start, the fine iteration reaches residual 1e-4 in fewer steps than from
    the uniform start, and the two converge to the same eigenvector."""
    V, _, w = synth.multichannel(16, 128, 128, C=8, seed=5003)
    feats = torch.from_numpy(V).cuda()
    radius = (2, 7, 7)
    with sf.PowerIteration(8, 16, 128, 128) as h:
        h.set_features(feats, w, 0.0)

        def to_tol(x, init):
            its, res = 0, 1.0
            while res > 1e-4 and its < 4000:
                x = h.power_iterate(None, radius=radius, iters=20, x=x, init=init)
                init = "user"
                its += 20
                res = h.rayleigh(x, radius)[1]
            return x, its

        xu, its_u = to_tol(torch.empty((16, 128, 128), device="cuda"), "uniform")
        x0, lvl_its = h.coarse_start(radius, levels=1, tol=1e-4)
        xc, its_c = to_tol(x0, "user")
    assert its_c < its_u, (its_c, its_u, lvl_its)
    cos = float((xu * xc).sum() / (xu.norm() * xc.norm()))
    assert cos > 1 - 1e-4, cos


def test_coarse_start_errors(sf):
    with sf.PowerIteration(1, 4, 16, 16) as h:
        with pytest.raises(sf.SFSegError) as e:
            h.coarse_start((1, 3, 3))
        assert e.value.status == "STATE"
        h.set_features(torch.rand((1, 4, 16, 16), device="cuda"))
        for bad in (0, 5):
            with pytest.raises(sf.SFSegError):
                h.coarse_start((1, 3, 3), levels=bad)
        with pytest.raises(sf.SFSegError):
            h.coarse_start((1, 3, 3), tol=0.0)
        # levels deeper than the volume: extents clamp at 1
        x0, its = h.coarse_start((1, 3, 3), levels=4, tol=1e-3)
        assert torch.isfinite(x0).all() and bool((x0 > 0).all())


def test_net_extra_channel_matches_oracle(sf):
    """The coarse solution enters the network as input channel C: forward against the FP64
    plain-loop network on the 9-channel stack."""
    rng = np.random.default_rng(11)
    C, T, H, W = 8, 3, 21, 140
    feats = rng.uniform(0.0, 1.0, size=(C, T, H, W)).astype(np.float32)
    extra = rng.uniform(0.0, 1.0, size=(T, H, W)).astype(np.float32)
    net = sf.WarmStartNet(9, seed=7)
    x0 = net.forward(torch.from_numpy(feats).cuda(), torch.from_numpy(extra).cuda()).cpu().numpy()
    bf = lambda a: synth.to_bf16_round(np.asarray(a, dtype=np.float32)).astype(np.float64)
    params = [(bf(wt), b.astype(np.float64)) for wt, b in net.unflatten(net.get_params())]
    ref, _ = oracle.warmstart_forward(bf(np.concatenate([feats, extra[None]], 0)), params)
    err = np.abs(x0 - ref).max() / np.abs(ref).max()
    assert err < 3e-2, err
    with sf.PowerIteration(C, T, H, W) as h:
        xw = h.warmstart(net, torch.from_numpy(feats).cuda(), torch.from_numpy(extra).cuda())
        torch.cuda.synchronize()
        assert np.array_equal(xw.cpu().numpy(), x0)
    net.close()
