"""GPU parity of the forward power iteration (Eq. 7 + Eq. 8) against the FP64 CPU oracle.

Bar (from the method's tolerance): max |x_gpu - x_oracle| <= 1e-5 on the unit-norm iterate with
float32 storage, <= 2e-3 with bf16 storage, at equal iteration count from the same start.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_08058_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5
TOL_BF16 = 2e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2212_08058_gb300 import build
    build.build()
    oracle.build()


def _sf():
    from paper_2212_08058_gb300 import sfseg
    return sfseg


def _run(V, radius, iters, sigma=None, alpha=1.0, p=0.1, weights=None, bias=0.0, init="uniform", x0=None,
         iters_bf16=0, dtype=torch.float32):
    sf = _sf()
    C, T, H, W = V.shape
    with sf.PowerIteration(C, T, H, W, alpha=alpha, p=p) as h:
        feats = torch.from_numpy(np.ascontiguousarray(V)).cuda().to(dtype)
        x = None if x0 is None else torch.from_numpy(np.ascontiguousarray(x0, dtype=np.float32)).cuda()
        x, nu = h.power_iterate(feats, weights, bias, radius, sigma, iters, iters_bf16, x=x, init=init,
                                return_norms=True)
        torch.cuda.synchronize()
        return x.cpu().numpy().astype(np.float64), nu


def _oracle(V, radius, iters, sigma=None, alpha=1.0, p=0.1, weights=None, bias=0.0, x0=None):
    f = oracle.combine(V.astype(np.float64), weights, bias)
    start = np.ones(f.shape) if x0 is None else x0
    return oracle.power_filter(f, f, p, alpha, radius, start, iters, sigma=sigma)


def test_config1_blob_parity():
    """8 x 64 x 64 drifting blob, radius (1, 3, 3), 20 iterations from the uniform start."""
    V = synth.drifting_blob(8, 64, 64, seed=1000)
    xg, nug = _run(V, (1, 3, 3), 20)
    xo, nuo = _oracle(V, (1, 3, 3), 20)
    assert np.abs(xg - xo).max() <= TOL_F32
    np.testing.assert_allclose(nug, nuo, rtol=1e-5)
    # the explicit-matrix oracle (Eq. 2, Eq. 4): same iterate, nu_M = alpha nu_A
    f = V[0].astype(np.float64)
    xc, nuc = oracle.power_csr(oracle.affinity(f, f, 0.1, 1.0, (1, 3, 3)), np.ones(f.size), 20)
    assert np.abs(xg.reshape(-1) - xc).max() <= TOL_F32
    assert xg.min() >= -1e-7


@pytest.mark.parametrize("shape,radius,sigma,alpha,p,K", [
    ((5, 37, 70), (2, 3, 5), (1.1, 1.7, 2.3), 0.7, 0.25, 7),     # ragged tiles, anisotropic
    ((3, 5, 6), (4, 8, 8), None, 1.0, 0.1, 5),                   # radius beyond the volume
    ((1, 1, 1), (1, 1, 1), None, 1.0, 0.1, 3),                   # a single voxel
    ((9, 16, 129), (1, 3, 3), None, 1.0, 0.2, 11),               # width one past a tile
    ((4, 20, 64), (0, 2, 8), None, 1.0, 0.1, 6),                 # no temporal coupling
])
def test_ragged_and_degenerate_shapes(shape, radius, sigma, alpha, p, K):
    rng = np.random.default_rng(sum(shape))
    V = rng.uniform(0.0, 1.0, size=(1, *shape)).astype(np.float32)
    V[0].reshape(-1)[5::11] = 0.0                     # u = 0 nodes (0^p := 0), never all of them
    xg, nug = _run(V, radius, K, sigma=sigma, alpha=alpha, p=p)
    xo, nuo = _oracle(V, radius, K, sigma=sigma, alpha=alpha, p=p)
    assert np.abs(xg - xo).max() <= TOL_F32
    np.testing.assert_allclose(nug, nuo, rtol=1e-5)


@pytest.mark.parametrize("shape,radius", [
    ((1, 5, 7), (2, 7, 7)),          # one frame, tile larger than the volume
    ((3, 17, 65), (2, 7, 7)),        # one row and one column past a tile
    ((4, 40, 72), (2, 7, 7)),
    ((2, 9, 130), (1, 3, 3)),
    ((6, 31, 200), (1, 3, 3)),
    ((2, 16, 64), (1, 3, 3)),        # exactly one tile
])
def test_fast_kernel_shapes(shape, radius):
    """The TMA kernel used for the method's radii: parity with the oracle, and with the generic
    streaming kernel (which the library uses when checkpoints are recorded every step)."""
    sf = _sf()
    rng = np.random.default_rng(sum(shape) + 7)
    V = rng.uniform(0.0, 1.0, size=(1, *shape)).astype(np.float32)
    K = 9
    xg, nug = _run(V, radius, K)
    xo, nuo = _oracle(V, radius, K)
    assert np.abs(xg - xo).max() <= TOL_F32
    np.testing.assert_allclose(nug, nuo, rtol=1e-5)
    with sf.PowerIteration(1, *shape) as h:
        xr = h.power_iterate(torch.from_numpy(V).cuda(), radius=radius, iters=K, record_every=1)
        torch.cuda.synchronize()
        xr = xr.cpu().numpy().astype(np.float64)
    assert np.abs(xg - xr).max() <= 1e-6


def test_radius_zero_is_diagonal():
    """Radius (0, 0, 0): K steps from uniform give u^(2K)/||u^(2K)|| exactly."""
    rng = np.random.default_rng(5)
    V = rng.uniform(0.3, 1.0, size=(1, 3, 10, 17)).astype(np.float32)
    p, K = 0.35, 6
    xg, _ = _run(V, (0, 0, 0), K, p=p)
    ref = V[0].astype(np.float64) ** (2 * p * K)
    assert np.abs(xg - ref / np.linalg.norm(ref)).max() <= TOL_F32


def test_start_vectors_and_zero_iterations():
    rng = np.random.default_rng(6)
    V = synth.drifting_blob(6, 40, 48, seed=1001)
    x0 = rng.uniform(0.1, 1.0, size=V.shape[1:])
    xg, _ = _run(V, (1, 3, 3), 9, init="user", x0=x0)
    xo, _ = _oracle(V, (1, 3, 3), 9, x0=x0)
    assert np.abs(xg - xo).max() <= TOL_F32
    xg, _ = _run(V, (1, 3, 3), 9, init="smap")
    xo, _ = _oracle(V, (1, 3, 3), 9, x0=V[0].astype(np.float64))
    assert np.abs(xg - xo).max() <= TOL_F32
    xg, nu = _run(V, (1, 3, 3), 0, init="user", x0=x0)
    assert len(nu) == 0
    assert np.abs(xg - x0 / np.linalg.norm(x0)).max() <= 1e-7


def test_multichannel_sigmoid_float32():
    """Eq. 9 + Eq. 10: C = 3 float32 channels combined by the sigmoid, then iterated."""
    V, _, w = synth.multichannel(6, 48, 80, C=3, seed=3001)
    xg, nug = _run(V, (1, 3, 3), 12, weights=w, bias=-0.2)
    xo, nuo = _oracle(V, (1, 3, 3), 12, weights=w, bias=-0.2)
    assert np.abs(xg - xo).max() <= TOL_F32
    np.testing.assert_allclose(nug, nuo, rtol=1e-5)


@pytest.mark.parametrize("bf16_iters", [16, 11, 0])
def test_bf16_storage(bf16_iters):
    """SFSeg++ with C = 8 bf16 channels (Sec. 5.1.2 setting): bf16 storage of f and the iterate
    for the first iterations, float32 afterwards; error against the FP64 oracle run on the
    float32 originals of the channels."""
    V, _, w = synth.multichannel(8, 64, 96, C=8, seed=3002)
    K = 16
    xg, _ = _run(V, (2, 7, 7), K, weights=w, iters_bf16=bf16_iters, dtype=torch.bfloat16)
    xo, _ = _oracle(V, (2, 7, 7), K, weights=w)
    err = np.abs(xg - xo).max()
    assert err <= TOL_BF16
    if bf16_iters == 0:   # bf16 inputs, float32 storage: only the input rounding remains
        Vb = synth.to_bf16_round(V)
        xb, _ = _oracle(Vb, (2, 7, 7), K, weights=w)
        assert np.abs(xg - xb).max() <= TOL_F32


def test_apply_and_symmetry():
    """One A application equals the oracle's Eq. 7; <Ay, z> = <y, Az> on the GPU operator."""
    sf = _sf()
    rng = np.random.default_rng(7)
    V = synth.drifting_blob(7, 33, 90, seed=1002)
    y = rng.normal(size=V.shape[1:]).astype(np.float32)
    z = rng.normal(size=V.shape[1:]).astype(np.float32)
    with sf.PowerIteration(1, *V.shape[1:]) as h:
        h.set_features(torch.from_numpy(V).cuda())
        Ay = h.apply(torch.from_numpy(y).cuda(), (2, 3, 4)).cpu().numpy().astype(np.float64)
        Az = h.apply(torch.from_numpy(z).cuda(), (2, 3, 4)).cpu().numpy().astype(np.float64)
    f = V[0].astype(np.float64)
    ref = oracle.filter_apply(f, f, 0.1, 1.0, (2, 3, 4), y.astype(np.float64))
    assert np.abs(Ay - ref).max() <= 1e-5 * np.abs(ref).max()
    lhs, rhs = np.sum(Ay * z), np.sum(y * Az)
    assert abs(lhs - rhs) <= 1e-5 * np.sqrt(np.sum(Ay ** 2) * np.sum(z ** 2))


def test_rayleigh_and_residual():
    """Eq. 3 quantities on the GPU against the oracle's operator, for a non-converged and a
    nearly converged x."""
    sf = _sf()
    V = synth.drifting_blob(8, 64, 64, seed=1000)
    f = V[0].astype(np.float64)
    with sf.PowerIteration(1, 8, 64, 64) as h:
        feats = torch.from_numpy(V).cuda()
        for K in (3, 300):
            x = h.power_iterate(feats, radius=(1, 3, 3), iters=K)
            rho, res = h.rayleigh(x, (1, 3, 3))
            xr = x.cpu().numpy().astype(np.float64)
            rho_o, res_o = oracle.rayleigh(lambda v: oracle.filter_apply(f, f, 0.1, 1.0, (1, 3, 3), v), xr)
            assert abs(rho - rho_o) <= 1e-6 * rho_o
            assert abs(res - res_o) <= 1e-4 * res_o + 1e-6


def test_error_statuses():
    sf = _sf()
    with sf.PowerIteration(1, 2, 8, 8) as h:
        bad = torch.full((1, 2, 8, 8), 0.5, device="cuda")
        bad[0, 1, 3, 3] = -1.0
        with pytest.raises(sf.SFSegError) as e:
            h.power_iterate(bad, radius=(1, 1, 1), iters=2, return_norms=True)
        assert e.value.status == "NONFINITE"
        with pytest.raises(sf.SFSegError) as e:
            h.power_iterate(torch.zeros((1, 2, 8, 8), device="cuda"), radius=(1, 1, 1), iters=2,
                            return_norms=True)
        assert e.value.status == "ZERO_NORM"
        with pytest.raises(sf.SFSegError) as e:
            h.power_iterate(torch.full((1, 2, 8, 8), 0.5, device="cuda"), radius=(5, 1, 1), iters=2)
        assert e.value.status == "SHAPE"
        with pytest.raises(sf.SFSegError) as e:
            h.rayleigh(torch.zeros((2, 8, 8), device="cuda"), (1, 1, 1))
        assert e.value.status == "ZERO_NORM"
        x = h.power_iterate(torch.full((1, 2, 8, 8), 0.5, device="cuda"), radius=(1, 1, 1), iters=2)
        assert torch.isfinite(x).all()          # the handle is still usable after the errors


def test_full_size_480p_parity():
    """Config of the benchmark: C = 1 float32, 64 x 480 x 854, three crossing blobs, radius
    (2, 7, 7), 50 iterations, in the launch configuration the benchmark times; compared
    element by element with the FP64 filter-form oracle."""
    V = synth.crossing_blobs(64, 480, 854, seed=2000)
    xg, nug = _run(V, (2, 7, 7), 50)
    xo, nuo = _oracle(V, (2, 7, 7), 50)
    assert np.abs(xg - xo).max() <= TOL_F32
    np.testing.assert_allclose(nug, nuo, rtol=1e-5)


def test_kronecker_eigenpair_full_size():
    """Constant features: the closed-form top eigenpair (u^2/alpha) l_t l_h l_w,
    v_t (x) v_h (x) v_w satisfies A v = lambda v on the GPU at 64 x 480 x 854, borders included."""
    sf = _sf()
    T, H, W = 64, 480, 854
    r = (2, 7, 7)
    sig = sf.default_sigma(r)
    fval, p = 0.6, 0.1

    def band(n, ra, sa):
        d = np.arange(n)[:, None] - np.arange(n)[None, :]
        return np.where(np.abs(d) <= ra, np.exp(-d * d / (2 * sa * sa)), 0.0)

    vals, vecs = [], []
    for n, ra, sa in zip((T, H, W), r, sig):
        e, Vv = np.linalg.eigh(band(n, ra, sa))
        vals.append(e[-1])
        vecs.append(Vv[:, -1] * np.sign(Vv[:, -1].sum()))
    lam = fval ** (2 * p) * vals[0] * vals[1] * vals[2]
    v = np.einsum("a,b,c->abc", *vecs).astype(np.float32)
    with sf.PowerIteration(1, T, H, W, p=p) as h:
        h.set_features(torch.full((1, T, H, W), fval, device="cuda"))
        Av = h.apply(torch.from_numpy(v).cuda(), r).cpu().numpy().astype(np.float64)
        rho, res = h.rayleigh(torch.from_numpy(v).cuda(), r)
    assert np.abs(Av - lam * v).max() <= 2e-6 * lam * np.abs(v).max()
    assert abs(rho - lam) <= 1e-5 * lam
    assert res < 1e-5


def test_invariants_480p():
    """The invariants that hold on every run, on the benchmark's workload (three crossing blobs,
    64 x 480 x 854, radius (2,7,7), 50 iterations from the uniform start; alpha = 1 and f in
    [0, 1], so M >= 0): x >= 0; the norms nu_k = ||A x_{k-1}|| do not decrease (for symmetric A,
    ||A^k x0|| is log-convex in k); the Eq. 3 quotient is at most the largest row sum max(A 1);
    and a slab of rt frames with f = 0 (u = 0) decouples the frames before it from the frames
    after it: A maps a vector supported before the slab to one that is exactly 0 after it."""
    sf = _sf()
    T, H, W = 64, 480, 854
    r = (2, 7, 7)
    V = synth.crossing_blobs(T, H, W, seed=2000)
    with sf.PowerIteration(1, T, H, W) as h:
        feats = torch.from_numpy(np.ascontiguousarray(V)).cuda()
        x, nu = h.power_iterate(feats, radius=r, iters=50, return_norms=True)
        assert float(x.min()) >= 0.0
        nu = np.asarray(nu)
        assert np.all(nu[1:] >= nu[:-1] * (1 - 1e-6)), np.min(nu[1:] / nu[:-1])
        rho, _ = h.rayleigh(x, r)
        rowsum = float(h.apply(torch.ones((T, H, W), device="cuda"), r).max())
        assert rho <= rowsum * (1 + 1e-6)
        # decoupling: zero f on frames [30, 30 + rt)
        Vz = V.copy()
        Vz[:, 30:30 + r[0]] = 0.0
        h.set_features(torch.from_numpy(np.ascontiguousarray(Vz)).cuda())
        y = torch.zeros((T, H, W), device="cuda")
        y[:30] = torch.rand((30, H, W), device="cuda")
        Ay = h.apply(y, r)
        assert float(Ay[30:].abs().max()) == 0.0
        assert float(Ay[:30].abs().max()) > 0.0


def test_kronecker_eigenpair_1080p():
    """The same closed form at the warm-start volume's shape, 120 x 1080 x 1920 (2.49e8 voxels,
    the outer product built on the device): A v = lambda v, the Eq. 3 quotient and residual."""
    sf = _sf()
    T, H, W = 120, 1080, 1920
    r = (2, 7, 7)
    sig = sf.default_sigma(r)
    fval, p = 0.35, 0.1

    def band(n, ra, sa):
        d = np.arange(n)[:, None] - np.arange(n)[None, :]
        return np.where(np.abs(d) <= ra, np.exp(-d * d / (2 * sa * sa)), 0.0)

    vals, vecs = [], []
    for n, ra, sa in zip((T, H, W), r, sig):
        e, Vv = np.linalg.eigh(band(n, ra, sa))
        vals.append(e[-1])
        vecs.append(torch.from_numpy(Vv[:, -1] * np.sign(Vv[:, -1].sum())).float().cuda())
    lam = fval ** (2 * p) * vals[0] * vals[1] * vals[2]
    v = torch.einsum("a,b,c->abc", *vecs).contiguous()
    with sf.PowerIteration(1, T, H, W, p=p) as h:
        h.set_features(torch.full((1, T, H, W), fval, device="cuda"))
        Av = h.apply(v, r)
        rho, res = h.rayleigh(v, r)
    err = float((Av - lam * v).abs().max())
    assert err <= 2e-6 * lam * float(v.abs().max())
    assert abs(rho - lam) <= 1e-5 * lam
    assert res < 1e-5


def test_full_size_sfsegpp_bf16_parity():
    """SFSeg++ at the 480p shape: C = 8 channels of 64 x 480 x 854 in bf16 (multichannel recipe),
    radius (2,7,7), every iteration in bf16 storage, in the launch configuration the benchmark's
    bf16 line times, for the workload's 50 iterations; element by element against the FP64 oracle
    run on the float32 originals of the channels (about half a second per oracle iteration on
    the host cores)."""
    V, _, w = synth.multichannel(64, 480, 854, C=8, seed=3000)
    K = 50
    xg, nug = _run(V, (2, 7, 7), K, weights=w, iters_bf16=K, dtype=torch.bfloat16)
    xo, nuo = _oracle(V, (2, 7, 7), K, weights=w)
    assert np.abs(xg - xo).max() <= TOL_BF16
    np.testing.assert_allclose(nug, nuo, rtol=2e-3)


def test_bounded_wait_reports_timeout():
    """The failure path of the kernels' bounded waits, run on purpose without a GPU fault: a
    wait on a barrier nothing completes gives up, the call returns TIMEOUT, and the handle and
    the context keep working (the next power iteration matches the oracle)."""
    sf = _sf()
    V = synth.drifting_blob(4, 32, 40, seed=7500)
    with sf.PowerIteration(1, 4, 32, 40) as h:
        for _ in range(2):
            with pytest.raises(sf.SFSegError) as e:
                h.selftest_wait(200)
            assert e.value.status == "TIMEOUT"
        x = h.power_iterate(torch.from_numpy(V).cuda(), radius=(1, 3, 3), iters=8).cpu().numpy()
    xo, _ = _oracle(V, (1, 3, 3), 8)
    assert np.abs(x - xo).max() <= TOL_F32


def test_cuda_graph_replay_is_identical():
    """sfseg_enable_graphs: calls replayed from captured CUDA graphs give the same results as
    direct launches (the kernels are the same; only the order of the FP64 atomic norm sums may
    differ, so the comparison allows a few float32 ulps) -- with new feature values under the
    same pointers, new x buffers (new captures), more keys than the cache holds, a bf16 phase
    and the S_m start."""
    sf = _sf()
    T, H, W = 8, 64, 64
    V1 = torch.from_numpy(synth.drifting_blob(T, H, W, seed=7600)).cuda()
    V2 = torch.from_numpy(synth.drifting_blob(T, H, W, seed=7601)).cuda()
    with sf.PowerIteration(1, T, H, W) as ref, sf.PowerIteration(1, T, H, W) as gr:
        gr.enable_graphs(True)
        xs = [torch.empty((T, H, W), device="cuda") for _ in range(10)]
        for V in (V1, V2, V1):
            ref.set_features(V)
            gr.set_features(V)
            for i, (radius, iters, nb, init) in enumerate([((1, 3, 3), 20, 0, "uniform"), ((2, 7, 7), 7, 3, "uniform"),
                                                           ((1, 3, 3), 5, 0, "smap"), ((1, 2, 3), 4, 0, "uniform")]):
                a = ref.power_iterate(None, radius=radius, iters=iters, iters_bf16=nb, init=init)
                b = gr.power_iterate(None, radius=radius, iters=iters, iters_bf16=nb, init=init, x=xs[i])
                torch.cuda.synchronize()
                assert torch.allclose(a, b, rtol=1e-6, atol=1e-9), (radius, iters, nb, init)
        # more distinct keys than the cache keeps (x buffers), each replayed twice
        for rep in range(2):
            for i in range(10):
                b = gr.power_iterate(None, radius=(1, 3, 3), iters=3 + i % 3, x=xs[i])
                a = ref.power_iterate(None, radius=(1, 3, 3), iters=3 + i % 3)
                torch.cuda.synchronize()
                assert torch.allclose(a, b, rtol=1e-6, atol=1e-9)


def test_near_maximum_volume_sampled():
    """Close to the largest volume a handle takes (T H W < 2^31; here 996 x 1080 x 1990 = 2.14e9
    voxels, whose pitched layout, 2.17e9 elements, passes 2^31): y = A x at radius (2,7,7)
    through the TMA kernel, checked at sampled voxels (corners, borders, interior) against the
    FP64 oracle evaluated on the crop that holds each voxel's whole neighbourhood.  Inputs are
    drawn on the device from a seeded generator."""
    sf = _sf()
    T, H, W = 996, 1080, 1990
    r = (2, 7, 7)
    gen = torch.Generator(device="cuda").manual_seed(7700)
    feats = torch.rand((1, T, H, W), device="cuda", generator=gen)
    x = torch.rand((T, H, W), device="cuda", generator=gen) + 0.5
    with sf.PowerIteration(1, T, H, W) as h:
        h.set_features(feats)
        y = h.apply(x, r)
        torch.cuda.synchronize()
        rng = np.random.default_rng(17)
        pts = [(0, 0, 0), (T - 1, H - 1, W - 1), (0, H - 1, 0), (T - 1, 0, W - 1), (T // 2, 7, W - 8)]
        pts += [tuple(int(v) for v in rng.integers((0, 0, 0), (T, H, W))) for _ in range(11)]
        scale = float(y.abs().max())
        for (t, hh, w) in pts:
            sl = tuple(slice(max(c - rr, 0), min(c + rr + 1, n)) for c, rr, n in zip((t, hh, w), r, (T, H, W)))
            fc = feats[0][sl].cpu().numpy().astype(np.float64)
            xc = x[sl].cpu().numpy().astype(np.float64)
            yo = oracle.filter_apply(fc, fc, 0.1, 1.0, r, xc)
            ci = tuple(c - s.start for c, s in zip((t, hh, w), sl))
            assert abs(float(y[t, hh, w]) - yo[ci]) <= 1e-5 * scale, ((t, hh, w), float(y[t, hh, w]), yo[ci])
        # one power iteration at this size runs and stays finite
        xs = h.power_iterate(None, radius=r, iters=2)
        assert bool(torch.isfinite(xs[::97, ::101, ::103]).all())
    del feats, x, y, xs
    torch.cuda.empty_cache()
