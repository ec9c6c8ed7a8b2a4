"""The warm-start network at the tile heights and frame groups its production launches use.

Each hidden-layer convolution launch takes three output frames per CTA when that grid still
gives four waves at some tile height, else two, else one, and then the tallest of 64, 32 or 16
output rows per CTA that gives four waves; the last layer's kernel takes four frames or one.
The small network tests select one frame and 16 rows; the volumes here select three frames and
64 rows (as the 120 x 1080 x 1920 inference does), three frames and 32 rows, three frames and
16 rows (32 x 256 x 512, the profiled case), two frames and one frame per CTA, and frame counts
that leave the last group of a layer short.  Each case checks the shape that the library
reports for its launches.  Every layer alone is compared with the FP64 oracle's plain
convolution loops on the GPU layer's own bf16 input, so that only the fp32 accumulation and the
final bf16 rounding differ: |gpu - ref| <= 2^-8 |ref| + 1e-5 sum|w x| (bf16's unit roundoff on
the stored output, and an fp32-accumulation bound relative to the sum of the absolute
products).  The sampled voxels include the tile seams along h and w, rows around the wraps of
the accumulator ring in tensor memory (5, 8 or 16 row blocks per output frame for three, two or
one frames per CTA; 8 or 16 in the last layer), every frame position inside a CTA's group, and
the volume's faces.  The data gradient (flipped taps, ReLU mask) is checked the same way, the
weight gradient over a whole smaller volume, and the whole network at sampled voxels on the
9 x 9 x 9 crop around each (one voxel's output depends on nothing else).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_08058_gb300 import synth

pytestmark = pytest.mark.gpu

C_IN = 9          # 8 feature channels and the coarse start, as the trained network
EPS_ACC = 1e-5    # fp32 accumulation, relative to sum |w x|
U_BF16 = 2.0 ** -8


@pytest.fixture(scope="module")
def sf():
    from paper_2212_08058_gb300 import build, sfseg
    build.build()
    oracle.build()
    return sfseg


def _ctas(T, H, W, frames, rows, tile_w):
    return -(-T // frames) * -(-W // tile_w) * -(-H // rows)


def _check_launch(sf, kernel, T, H, W, frames, rows):
    """The library's report of its most recent launch of a convolution kernel (0: hidden layers,
    128-voxel tiles; 1: the last layer, 126-voxel tiles) has the frames and rows per CTA that the
    test case is meant to exercise, and one CTA per (frame group, tile column, row tile)."""
    tile_w = 128 if kernel == 0 else 126
    assert sf.net_launch_shape(kernel) == (frames, rows, _ctas(T, H, W, frames, rows, tile_w))


def _points(T, H, W, HR, seed, n_random=40):
    hs = {0, 1, H - 2, H - 1}
    for base in (HR, 2 * HR, (H // HR - 1) * HR):      # tile seams along h
        hs.update({base - 1, base, base + 1})
    for j in (1, 2, 4, 5, 6, 7, 8, 9, 10, 11, 15, 16, 17, 31, 32, 33):   # ring wraps (5, 8, 16 blocks)
        hs.add(HR + j)
    # 128-voxel tiles of the hidden layers, 126-voxel tiles of the last layer
    ws = {0, 1, 125, 126, 127, 128, 129, 251, 252, 255, 256, W - 129, W - 128, W - 2, W - 1}
    pts = set()
    # frames 0..3 take every position inside a CTA's group of frames (up to three per CTA in the
    # hidden layers, four in the last layer)
    for h in hs:
        for t in (0, 1, 2, 3, T // 2, T - 1):
            for w in (0, 125, 126, 127, 128, W - 1):
                pts.add((t, h, w))
    for w in ws:
        for t in (0, 1, 3, T - 1):
            for h in (0, HR - 1, HR, H - 1):
                pts.add((t, h, w))
    rng = np.random.default_rng(seed)
    for _ in range(n_random):
        pts.add(tuple(int(v) for v in rng.integers((0, 0, 0), (T, H, W))))
    return sorted(p for p in pts if 0 <= p[0] < T and 0 <= p[1] < H and 0 <= p[2] < W)


def _crop(a, p, r, shape):
    """a[t-r..t+r, h-r..h+r, w-r..w+r] clipped to the volume (zero padding is the oracle's) as
    float64, and the index of p inside it."""
    sl = tuple(slice(max(c - r, 0), min(c + r + 1, n)) for c, n in zip(p, shape))
    return a[sl].float().cpu().numpy().astype(np.float64), tuple(c - s.start for c, s in zip(p, sl))


def _bf16(a):
    return synth.to_bf16_round(np.asarray(a, dtype=np.float32)).astype(np.float64)


def _layer_params(net):
    return [(_bf16(w), b.astype(np.float64)) for w, b in net.unflatten(net.get_params())]


def _check_fwd(layer, x_in, out, params, pts, shape):
    wt, b = params[layer]
    cin = wt.shape[-1]
    worst = 0.0
    for p in pts:
        xc, ci = _crop(x_in, p, 1, shape)
        xc = xc[..., :cin]
        ref = oracle.conv3d_fwd(xc, wt, b)[ci]
        S = oracle.conv3d_fwd(np.abs(xc), np.abs(wt), np.abs(b))[ci]
        if layer < 3:
            ref = np.maximum(ref, 0.0)
            got = out[p].float().cpu().numpy().astype(np.float64)
        else:
            ref = ref[:1]
            got = np.array([float(out[p])])
            S = S[:1]
        err = np.abs(got - ref)
        tol = U_BF16 * np.abs(ref) + EPS_ACC * S if layer < 3 else EPS_ACC * S
        assert np.all(err <= tol), (layer, p, float((err / np.maximum(tol, 1e-30)).max()))
        worst = max(worst, float((err / np.maximum(S, 1e-30)).max()))
    return worst


def _forward_layers(net, x16):
    a1 = net.layer_forward(0, x16)
    a2 = net.layer_forward(1, a1)
    a3 = net.layer_forward(2, a2)
    z, x0 = net.layer_forward(3, a3)
    net.check()
    return [x16, a1, a2, a3], z, x0


def _input16(T, H, W, seed):
    gen = torch.Generator(device="cuda").manual_seed(seed)
    x = torch.zeros((T, H, W, 16), device="cuda", dtype=torch.bfloat16)
    x[..., :C_IN] = torch.rand((T, H, W, C_IN), device="cuda", generator=gen).to(torch.bfloat16)
    return x


@pytest.mark.parametrize("shape,fr,hr,last", [((35, 1024, 640), 3, 64, (4, 64)), ((17, 1024, 640), 3, 32, (4, 32)),
                                             ((32, 256, 512), 3, 16, (4, 16)), ((5, 1024, 512), 2, 16, (4, 16)),
                                             ((2, 1024, 640), 1, 16, (1, 16))],
                         ids=["rows64_partial_groups", "rows32", "rows16", "two_frames_per_cta", "one_frame_per_cta"])
def test_layers_at_production_tile_heights(sf, shape, fr, hr, last):
    """Each layer's output at sampled voxels against the oracle's convolution of the GPU layer's
    own input, at the frames and tile height per CTA the launch picks for this volume (the last
    layer's kernel picks its own: four frames and 64 rows as at 1080p for the first volume).
    Frame counts that the groups do not divide leave the last CTA of a layer with fewer output
    frames (35 = 11 x 3 + 2 and 8 x 4 + 3; 17 = 5 x 3 + 2; 5 = 2 x 2 + 1); the 2-frame volume
    runs one output frame per CTA in both kernels."""
    T, H, W = shape
    net = sf.WarmStartNet(C_IN, seed=11)
    params = _layer_params(net)
    x16 = _input16(T, H, W, 900 + hr)
    ins, z, x0 = _forward_layers(net, x16)
    _check_launch(sf, 0, T, H, W, fr, hr)
    _check_launch(sf, 1, T, H, W, *last)
    pts = sorted(set(_points(T, H, W, hr, seed=hr)) | set(_points(T, H, W, last[1], seed=hr + 1, n_random=0)))
    outs = [ins[1], ins[2], ins[3], z]
    for layer in range(4):
        _check_fwd(layer, ins[layer], outs[layer], params, pts, shape)
    # the softplus epilogue of the last layer
    zz = z.double()
    sp = torch.where(zz > 20, zz, torch.log1p(torch.exp(zz)))
    assert float(((x0.double() - sp).abs() / sp).max()) <= 1e-5
    net.close()


@pytest.mark.parametrize("shape,fr,hr", [((35, 1024, 640), 3, 64), ((17, 1024, 640), 3, 32), ((5, 1024, 512), 2, 16)],
                         ids=["rows64_partial_groups", "rows32", "two_frames_per_cta"])
def test_data_gradient_at_production_tile_heights(sf, shape, fr, hr):
    """dx = conv^T(dz) * [x > 0] of layers 1..3 (the data-gradient convolution on the tensor
    cores) at sampled voxels against the oracle's reverse loops on the same bf16 inputs."""
    T, H, W = shape
    net = sf.WarmStartNet(C_IN, seed=12)
    params = _layer_params(net)
    ins, _, _ = _forward_layers(net, _input16(T, H, W, 910 + hr))
    gen = torch.Generator(device="cuda").manual_seed(920 + hr)
    pts = _points(T, H, W, hr, seed=100 + hr, n_random=25)
    for layer in (1, 2, 3):
        x = ins[layer]
        if layer == 3:
            dz = torch.zeros((T, H, W, 16), device="cuda", dtype=torch.bfloat16)
            dz[..., 0] = torch.randn((T, H, W), device="cuda", generator=gen).to(torch.bfloat16)
        else:
            dz = torch.randn((T, H, W, 32), device="cuda", generator=gen).to(torch.bfloat16)
        dx, _, _ = net.layer_backward(layer, x, dz)
        net.check()
        _check_launch(sf, 0, T, H, W, fr, hr)
        wt, _ = params[layer]
        cout = wt.shape[0]
        for p in pts:
            xc, ci = _crop(x, p, 1, shape)
            dzc, _ = _crop(dz, p, 1, shape)
            dzc = dzc[..., :cout]
            dxr, _, _ = oracle.conv3d_bwd(xc, wt, dzc)
            Sx, _, _ = oracle.conv3d_bwd(np.abs(xc), np.abs(wt), np.abs(dzc))
            ref = dxr[ci] * (xc[ci] > 0)
            S = Sx[ci]
            got = dx[p].float().cpu().numpy().astype(np.float64)
            err = np.abs(got - ref)
            tol = U_BF16 * np.abs(ref) + EPS_ACC * S
            assert np.all(err <= tol), (layer, p, float((err / np.maximum(tol, 1e-30)).max()))
    net.close()


def test_weight_gradient_whole_volume(sf):
    """dW and db of every layer over a whole 4 x 64 x 200 volume (two 128-voxel tiles along w,
    a ragged second one) against the oracle's reverse loops, relative to the sum of the
    absolute products of each entry."""
    T, H, W = 4, 64, 200
    net = sf.WarmStartNet(C_IN, seed=13)
    params = _layer_params(net)
    ins, _, _ = _forward_layers(net, _input16(T, H, W, 930))
    gen = torch.Generator(device="cuda").manual_seed(931)
    for layer in range(4):
        x = ins[layer]
        if layer == 3:
            dz = torch.zeros((T, H, W, 16), device="cuda", dtype=torch.bfloat16)
            dz[..., 0] = torch.randn((T, H, W), device="cuda", generator=gen).to(torch.bfloat16)
        else:
            dz = torch.randn((T, H, W, 32), device="cuda", generator=gen).to(torch.bfloat16)
        _, dW, db = net.layer_backward(layer, x, dz, want_dx=False)
        net.check()
        wt, _ = params[layer]
        cout, cin = wt.shape[0], wt.shape[-1]
        xa = x.float().cpu().numpy().astype(np.float64)[..., :cin]
        dza = dz.float().cpu().numpy().astype(np.float64)[..., :cout]
        _, dwr, dbr = oracle.conv3d_bwd(xa, wt, dza, need_dx=False)
        _, dws, dbs = oracle.conv3d_bwd(np.abs(xa), np.abs(wt), np.abs(dza), need_dx=False)
        gw = dW.cpu().numpy().astype(np.float64)
        gb = db.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(gw - dwr) <= 4 * EPS_ACC * dws + 1e-30), (layer, float(np.abs(gw - dwr).max()))
        assert np.all(np.abs(gb - dbr) <= 4 * EPS_ACC * dbs + 1e-30), (layer, float(np.abs(gb - dbr).max()))
    net.close()


def test_weight_gradient_training_volume(sf):
    """The weight gradient of a 32 -> 32 layer over a whole 16 x 128 x 128 training volume (the
    volumes the network is trained on: 2048 work units spread over every SM) against the
    oracle's reverse loops."""
    T, H, W = 16, 128, 128
    net = sf.WarmStartNet(C_IN, seed=15)
    params = _layer_params(net)
    gen = torch.Generator(device="cuda").manual_seed(950)
    x = torch.relu(torch.randn((T, H, W, 32), device="cuda", generator=gen)).to(torch.bfloat16)
    dz = torch.randn((T, H, W, 32), device="cuda", generator=gen).to(torch.bfloat16)
    _, dW, db = net.layer_backward(2, x, dz, want_dx=False)
    net.check()
    wt, _ = params[2]
    xa = x.float().cpu().numpy().astype(np.float64)
    dza = dz.float().cpu().numpy().astype(np.float64)
    _, dwr, dbr = oracle.conv3d_bwd(xa, wt, dza, need_dx=False)
    _, dws, dbs = oracle.conv3d_bwd(np.abs(xa), np.abs(wt), np.abs(dza), need_dx=False)
    assert np.all(np.abs(dW.cpu().numpy() - dwr) <= 4 * EPS_ACC * dws), float(np.abs(dW.cpu().numpy() - dwr).max())
    assert np.all(np.abs(db.cpu().numpy() - dbr) <= 4 * EPS_ACC * dbs), float(np.abs(db.cpu().numpy() - dbr).max())
    net.close()


@pytest.mark.parametrize("shape,fr,hr", [((35, 1024, 640), 3, 64), ((17, 1024, 640), 3, 32)],
                         ids=["rows64_partial_groups", "rows32"])
def test_network_sampled_at_production_tile_heights(sf, shape, fr, hr):
    """sfseg_net_forward (8 bf16 channels + the extra channel) at sampled voxels against the
    oracle's FP64 network on the 9 x 9 x 9 crop around each voxel, within the end-to-end bf16
    tolerance of the small network test (three hidden activations rounded to bf16)."""
    T, H, W = shape
    gen = torch.Generator(device="cuda").manual_seed(940 + hr)
    feats = torch.rand((8, T, H, W), device="cuda", generator=gen).to(torch.bfloat16)
    extra = torch.rand((T, H, W), device="cuda", generator=gen)
    net = sf.WarmStartNet(C_IN, seed=14)
    params = _layer_params(net)
    x0 = net.forward(feats, extra)
    net.check()
    _check_launch(sf, 0, T, H, W, fr, hr)
    extra_b = extra.to(torch.bfloat16)
    pts = _points(T, H, W, hr, seed=200 + hr, n_random=10)[::3]
    refs, gots = [], []
    for p in pts:
        sl = tuple(slice(max(c - 4, 0), min(c + 5, n)) for c, n in zip(p, shape))
        fc = feats[(slice(None),) + sl].float().cpu().numpy().astype(np.float64)
        ec = extra_b[sl].float().cpu().numpy().astype(np.float64)
        crop = np.concatenate([fc, ec[None]], axis=0)
        ref, _ = oracle.warmstart_forward(crop, params)
        ci = tuple(c - s.start for c, s in zip(p, sl))
        refs.append(ref[ci])
        gots.append(float(x0[p]))
    refs, gots = np.array(refs), np.array(gots)
    assert np.all(gots > 0)
    assert np.abs(gots - refs).max() <= 3e-2 * np.abs(refs).max(), float(np.abs(gots - refs).max())
    net.close()
