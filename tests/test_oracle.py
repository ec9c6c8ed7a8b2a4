"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Each test names the passage it pins and the mistake it would catch.
"""
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.ndimage
import scipy.special

import oracle
from paper_2212_08058_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_counts.txt")


def _golden():
    rows = {}
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            rows[key] = [int(v) for v in vals]
    return rows


def _rand_volume(rng, T, H, W, lo=0.0, hi=1.0):
    return rng.uniform(lo, hi, size=(T, H, W))


# --------------------------------------------------------------------------- Eq. 9
def test_combine_single_channel_passes_through():
    """Alg. 1 initialisation note: one channel is assigned directly, without the sigmoid."""
    rng = np.random.default_rng(0)
    V = rng.uniform(size=(1, 3, 4, 5))
    np.testing.assert_array_equal(oracle.combine(V, [2.0], 1.0), V[0])


def test_combine_sigmoid_is_logistic():
    """Eq. 9 with the standard logistic (reading of the printed 1/(1+e^x)): compare with
    scipy's expit; a sign error in the exponent or a dropped bias fails."""
    rng = np.random.default_rng(1)
    V = rng.uniform(size=(3, 2, 4, 5))
    w = np.array([0.7, -1.2, 2.5])
    b = -0.3
    z = np.tensordot(w, V, axes=1) + b
    np.testing.assert_allclose(oracle.combine(V, w, b), scipy.special.expit(z), rtol=1e-15, atol=0)
    assert np.all(oracle.combine(V, 10 * np.abs(w), 0.0) > 0.5)  # larger weights raise S_m


# --------------------------------------------------------------------- paper counts
def test_paper_tap_counts():
    """Sec. 4.2: a 3x7x7 kernel means 147 neighbours per node (interior row of M), and 17 taps
    in the separable filter form; the 10x20x20 video has 4000 nodes."""
    g = _golden()
    kt, kh, kw, dense, sep = g["kernel"]
    r = ((kt - 1) // 2, (kh - 1) // 2, (kw - 1) // 2)
    T, H, W = 5, 12, 12
    f = np.full((T, H, W), 0.5)
    M = oracle.affinity(f, f, 0.1, 1.0, r)
    row = (2 * H + 6) * W + 6  # t=2, h=6, w=6: an interior node
    assert M.indptr[row + 1] - M.indptr[row] == dense
    assert sum(len(oracle.taps(ri, 1.0)) for ri in r) == sep
    fr, hh, ww, nodes = g["graph"]
    M2 = oracle.affinity(np.full((fr, hh, ww), 0.3), np.full((fr, hh, ww), 0.3), 0.1, 1.0, (1, 1, 1))
    assert M2.shape == (nodes, nodes)
    fr, hh, ww, approx = g["graph_approx"]
    assert abs(fr * hh * ww - approx) / approx < 0.03


# ------------------------------------------------------------------------- Eq. 2
def test_affinity_symmetric_nonnegative():
    """Sec. 3: M must be symmetric and non-negative (alpha <= 1, features in [0, 1])."""
    rng = np.random.default_rng(2)
    f = _rand_volume(rng, 3, 5, 7)
    M = oracle.affinity(f, f, 0.2, 1.0, (1, 2, 2), sigma=(1.0, 1.3, 0.8))
    D = M.toarray()
    assert np.array_equal(D, D.T)        # bitwise symmetric
    assert D.min() >= 0.0
    np.testing.assert_allclose(np.diag(D), np.power(f.reshape(-1), 0.4), rtol=1e-15)  # u_i^2, G_ii = 1


def test_two_node_closed_form():
    """Eq. 2 on a 1x1x2 volume, worked by hand: with s = f = (0.2, 0.6), p = 0.5, alpha = 1 and
    sigma_w = 1, M = [[0.2, b], [b, 0.6]] with b = sqrt(0.12) (1 - 0.16) e^{-1/2}; its top
    eigenpair has the textbook 2x2 closed form."""
    f = np.array([0.2, 0.6]).reshape(1, 1, 2)
    M = oracle.affinity(f, f, 0.5, 1.0, (0, 0, 1), sigma=(1.0, 1.0, 1.0)).toarray()
    b = np.sqrt(0.12) * 0.84 * np.exp(-0.5)
    np.testing.assert_allclose(M, [[0.2, b], [b, 0.6]], rtol=1e-15, atol=1e-16)
    lam = 0.4 + np.sqrt(0.2 ** 2 + b * b)
    v = np.array([b, lam - 0.2])
    v /= np.linalg.norm(v)
    x, nu = oracle.power_csr(oracle.affinity(f, f, 0.5, 1.0, (0, 0, 1), sigma=(1.0, 1.0, 1.0)),
                             np.ones(2), 200)
    np.testing.assert_allclose(x, v, rtol=0, atol=1e-13)
    np.testing.assert_allclose(nu[-1], lam, rtol=1e-13)


def test_exact_kernel_approaches_taylor():
    """Eq. 1 vs Eq. 2: the first-order expansion differs by O(alpha^2 d^4), so the angle between
    the two principal eigenvectors shrinks like alpha^2 (Sec. 4.3 quantitative analysis)."""
    rng = np.random.default_rng(3)
    f = synth.drifting_blob(4, 10, 12, seed=7)[0].astype(np.float64)
    angles = []
    for alpha in (0.4, 0.2, 0.1):
        Mt = oracle.affinity(f, f, 0.1, alpha, (1, 2, 2))
        Me = oracle.affinity(f, f, 0.1, alpha, (1, 2, 2), exact=True)
        xt = np.linalg.eigh(Mt.toarray())[1][:, -1]
        xe = np.linalg.eigh(Me.toarray())[1][:, -1]
        xe *= np.sign(xe @ xt)
        angles.append(2 * np.arcsin(np.linalg.norm(xt - xe) / 2))
    assert angles[0] > angles[1] > angles[2]
    assert angles[1] / angles[2] > 3.0   # close to the factor 4 of a quadratic error


# --------------------------------------------------------------------- Eq. 7 vs Eq. 2
@pytest.mark.parametrize("shape,radius,sigma,alpha,p", [
    ((3, 5, 7), (1, 2, 2), None, 1.0, 0.1),
    ((4, 9, 6), (1, 3, 3), (0.9, 1.7, 2.1), 0.5, 0.2),
    ((2, 3, 11), (2, 1, 4), (1.2, 0.6, 3.0), 2.0, 0.35),
    ((5, 4, 4), (0, 0, 0), None, 1.0, 0.1),
    ((1, 17, 3), (0, 7, 7), None, 1.0, 0.1),     # radius larger than the volume
])
def test_filter_form_equals_explicit_matrix(shape, radius, sigma, alpha, p):
    """Eq. 6 -> Eq. 7 is an identity up to the factor alpha: A x = M x / alpha for any x.
    Catches a dropped term, a wrong sign in Eq. 6, a transposed axis or wrong padding."""
    rng = np.random.default_rng(sum(shape) + sum(radius))
    s = _rand_volume(rng, *shape)
    f = _rand_volume(rng, *shape)
    s.reshape(-1)[::7] = 0.0                  # 0^p := 0 nodes
    x = rng.uniform(-1, 1, size=shape)
    M = oracle.affinity(s, f, p, alpha, radius, sigma=sigma)
    y_mat = (M @ x.reshape(-1)) / alpha
    y_fil = oracle.filter_apply(s, f, p, alpha, radius, x, sigma=sigma).reshape(-1)
    scale = np.abs(M @ x.reshape(-1)).max()
    assert np.abs(y_mat - y_fil).max() <= 1e-13 * scale


def test_filter_form_symmetric_operator():
    """<A y, z> = <y, A z> (M symmetric); boundary or index mistakes break this."""
    rng = np.random.default_rng(4)
    f = _rand_volume(rng, 4, 7, 9)
    y = rng.normal(size=f.shape)
    z = rng.normal(size=f.shape)
    Ay = oracle.filter_apply(f, f, 0.1, 1.0, (1, 3, 2), y)
    Az = oracle.filter_apply(f, f, 0.1, 1.0, (1, 3, 2), z)
    assert abs(np.sum(Ay * z) - np.sum(y * Az)) <= 1e-12 * np.abs(Ay).sum()


# ------------------------------------------------------------------- Eq. 3, 4, 8
def test_power_iteration_matches_dense_eigensolver():
    """Eq. 3: the limit of Eq. 4 + Eq. 8 is the principal eigenvector of M (Perron vector,
    non-negative) and nu -> lambda_max.  Brute force with LAPACK on a 960-node volume."""
    f = synth.drifting_blob(5, 12, 16, seed=11)[0].astype(np.float64)
    M = oracle.affinity(f, f, 0.1, 1.0, (1, 2, 2))
    evals, evecs = np.linalg.eigh(M.toarray())
    v = evecs[:, -1] * np.sign(evecs[:, -1].sum())
    ratio = evals[-2] / evals[-1]
    K = int(np.ceil(np.log(1e-12) / np.log(ratio))) + 20
    x, nu = oracle.power_csr(M, synth.uniform_start(M.shape[0]), K)
    assert 2 * np.arcsin(np.linalg.norm(x - v) / 2) < 1e-8    # angle, well conditioned
    np.testing.assert_allclose(nu[-1], evals[-1], rtol=1e-12)
    assert x.min() >= 0.0
    rho, res = oracle.rayleigh(lambda z: M @ z, x)
    np.testing.assert_allclose(rho, evals[-1], rtol=1e-12)
    assert res < 1e-9


def test_kronecker_closed_form():
    """Constant s = f: Eq. 2 reduces to M = u^2 G_t (x) G_h (x) G_w with each G_a the 1D
    zero-padded Gaussian band matrix, so A = M/alpha has the top eigenpair
    (u^2/alpha) l_t l_h l_w, v_t (x) v_h (x) v_w, each factor from a 1D dense eigensolver.
    Every term of Eq. 7 matters here: 1/alpha - f^2 - f^2 + 2 f^2 = 1/alpha."""
    T, H, W = 5, 9, 13
    r = (1, 3, 2)
    sig = (0.8, 1.6, 1.1)
    fval, p, alpha = 0.7, 0.3, 0.8
    f = np.full((T, H, W), fval)

    def band(n, ra, sa):
        d = np.arange(n)[:, None] - np.arange(n)[None, :]
        return np.where(np.abs(d) <= ra, np.exp(-d * d / (2 * sa * sa)), 0.0)

    vals, vecs = [], []
    for n, ra, sa in zip((T, H, W), r, sig):
        e, V = np.linalg.eigh(band(n, ra, sa))
        vals.append(e[-1])
        vecs.append(V[:, -1] * np.sign(V[:, -1].sum()))
    u2 = fval ** (2 * p)
    lam = u2 / alpha * vals[0] * vals[1] * vals[2]
    v = np.einsum("a,b,c->abc", *vecs)
    Av = oracle.filter_apply(f, f, p, alpha, r, v, sigma=sig)
    np.testing.assert_allclose(Av, lam * v, rtol=0, atol=1e-13 * lam)
    x, nu = oracle.power_filter(f, f, p, alpha, r, np.ones((T, H, W)), 400, sigma=sig)
    np.testing.assert_allclose(x, v, atol=1e-10)
    np.testing.assert_allclose(nu[-1], lam, rtol=1e-12)


def test_exact_kernel_kronecker_closed_form():
    """Eq. 1 with constant f: the pair term is exp(0) = 1 for every alpha, so M = u^2 G_t (x)
    G_h (x) G_w with the top eigenpair u^2 l_t l_h l_w, v_t (x) v_h (x) v_w (1D dense
    eigensolvers); and at two voxels with known features one entry is
    u_i u_j exp(-alpha (f_i - f_j)^2) exp(-d^2 / (2 sigma^2)) per axis."""
    T, H, W = 4, 7, 9
    r = (1, 2, 3)
    sig = (0.9, 1.3, 1.7)
    fval, p, alpha = 0.55, 0.2, 1.7
    f = np.full((T, H, W), fval)

    def band(n, ra, sa):
        d = np.arange(n)[:, None] - np.arange(n)[None, :]
        return np.where(np.abs(d) <= ra, np.exp(-d * d / (2 * sa * sa)), 0.0)

    vals, vecs = [], []
    for n, ra, sa in zip((T, H, W), r, sig):
        e, V = np.linalg.eigh(band(n, ra, sa))
        vals.append(e[-1])
        vecs.append(V[:, -1] * np.sign(V[:, -1].sum()))
    lam = fval ** (2 * p) * vals[0] * vals[1] * vals[2]
    v = np.einsum("a,b,c->abc", *vecs).ravel()
    Me = oracle.affinity(f, f, p, alpha, r, sigma=sig, exact=True)
    np.testing.assert_allclose(Me @ v, lam * v, rtol=0, atol=1e-13 * lam)
    # one entry with distinct features: voxel (1, 3, 4) and its neighbour (2, 2, 6)
    g = np.linspace(0.1, 0.9, T * H * W).reshape(T, H, W)
    Mg = oracle.affinity(g, g, p, alpha, r, sigma=sig, exact=True)
    i = np.ravel_multi_index((1, 3, 4), (T, H, W))
    j = np.ravel_multi_index((2, 2, 6), (T, H, W))
    want = (g.flat[i] * g.flat[j]) ** p * np.exp(-alpha * (g.flat[i] - g.flat[j]) ** 2) * \
        np.exp(-1 / (2 * sig[0] ** 2) - 1 / (2 * sig[1] ** 2) - 4 / (2 * sig[2] ** 2))
    assert abs(Mg[i, j] - want) <= 1e-14 * want
    assert Mg[i, j] == Mg[j, i]


def test_diagonal_special_case():
    """Radius (0, 0, 0): M = diag(u_i^2), so K steps from the uniform start give exactly
    u^(2K) / ||u^(2K)|| (catches a wrong exponent p, e.g. s^(2p) for the unary term)."""
    rng = np.random.default_rng(5)
    f = _rand_volume(rng, 2, 3, 4, lo=0.2)
    p, K = 0.35, 7
    M = oracle.affinity(f, f, p, 1.0, (0, 0, 0))
    x, nu = oracle.power_csr(M, np.ones(f.size), K)
    ref = f.reshape(-1) ** (2 * p * K)
    np.testing.assert_allclose(x, ref / np.linalg.norm(ref), rtol=1e-13)
    xf, _ = oracle.power_filter(f, f, p, 1.0, (0, 0, 0), np.ones(f.shape), K)
    np.testing.assert_allclose(xf.reshape(-1), ref / np.linalg.norm(ref), rtol=1e-13)


def test_invariants_on_blob_volume():
    """Perron-Frobenius and power-iteration invariants: x >= 0; nu_k non-decreasing
    (log-convexity of ||A^k x|| for symmetric A); rho <= max row sum; zero-u slab decouples."""
    V = synth.drifting_blob(6, 14, 15, seed=12)[0].astype(np.float64)
    M = oracle.affinity(V, V, 0.1, 1.0, (1, 2, 2))
    x, nu = oracle.power_csr(M, synth.uniform_start(V.size), 60)
    assert x.min() >= 0.0
    assert np.all(np.diff(nu) >= -1e-14 * nu[1:])
    rho, _ = oracle.rayleigh(lambda z: M @ z, x)
    assert rho <= np.abs(M).sum(axis=1).max() * (1 + 1e-14)
    s = V.copy()
    s[2:4] = 0.0                                   # two empty frames, r_t = 1
    Ms = oracle.affinity(s, V, 0.1, 1.0, (1, 2, 2)).tocoo()
    HW = 14 * 15
    ti, tj = Ms.row // HW, Ms.col // HW
    nz = Ms.data != 0
    assert not np.any(((ti[nz] < 2) & (tj[nz] >= 4)) | ((ti[nz] >= 4) & (tj[nz] < 2)))


# ---------------------------------------------------------------------- Sec. 3.4
def _forward_loss(V, w, b, p, alpha, r, K, lossfn):
    f = oracle.combine(V, w, b)
    M = oracle.affinity(f, f, p, alpha, r)
    x, _ = oracle.power_csr(M, synth.uniform_start(f.size), K)
    return lossfn(x)


@pytest.mark.parametrize("which", ["linear", "soft_iou"])
def test_grad_matches_finite_differences(which):
    """The reverse pass through K normalised steps equals central finite differences of the
    forward pass (dL/dw_c and dL/db), C = 2."""
    rng = np.random.default_rng(6)
    V, m, _ = synth.multichannel(3, 6, 7, C=2, seed=21)
    V = V.astype(np.float64)
    w = np.array([1.3, -0.6])
    b = 0.2
    p, alpha, r, K = 0.2, 1.0, (1, 1, 2), 5
    if which == "linear":
        cvec = rng.normal(size=V[0].size)
        lossfn = lambda x: float(cvec @ x)
        gK = cvec
        f = oracle.combine(V, w, b)
        M = oracle.affinity(f, f, p, alpha, r)
    else:
        tgt = (m > 0.5).astype(np.float64).reshape(-1)
        lossfn = lambda x: oracle.soft_iou_loss(x, tgt)[0]
        f = oracle.combine(V, w, b)
        M = oracle.affinity(f, f, p, alpha, r)
        xK, _ = oracle.power_csr(M, synth.uniform_start(f.size), K)
        gK = oracle.soft_iou_loss(xK, tgt)[1]
    gw, gb = oracle.grad_csr(V, w, b, p, alpha, r, synth.uniform_start(V[0].size), K, gK)
    h = 1e-6
    for c in range(2):
        wp, wm = w.copy(), w.copy()
        wp[c] += h
        wm[c] -= h
        fd = (_forward_loss(V, wp, b, p, alpha, r, K, lossfn)
              - _forward_loss(V, wm, b, p, alpha, r, K, lossfn)) / (2 * h)
        assert abs(fd - gw[c]) <= 1e-6 * max(1.0, abs(fd)), (c, fd, gw[c])
    fd = (_forward_loss(V, w, b + h, p, alpha, r, K, lossfn)
          - _forward_loss(V, w, b - h, p, alpha, r, K, lossfn)) / (2 * h)
    assert abs(fd - gb) <= 1e-6 * max(1.0, abs(fd))


def test_soft_iou_loss_values_and_gradient():
    """1 - soft-IoU: zero when the max-normalised x equals a binary target; 1 for disjoint
    support; gradient equal to central differences."""
    g = np.array([0.0, 1.0, 1.0, 0.0, 1.0])
    assert oracle.soft_iou_loss(3.0 * g, g)[0] == pytest.approx(0.0, abs=1e-15)
    assert oracle.soft_iou_loss(np.array([1.0, 0, 0, 1.0, 0]), g)[0] == pytest.approx(1.0)
    rng = np.random.default_rng(7)
    x = rng.uniform(0.1, 1.0, size=5)
    _, dx = oracle.soft_iou_loss(x, g)
    h = 1e-7
    for i in range(5):
        e = np.zeros(5)
        e[i] = h
        fd = (oracle.soft_iou_loss(x + e, g)[0] - oracle.soft_iou_loss(x - e, g)[0]) / (2 * h)
        assert abs(fd - dx[i]) < 1e-7


# ------------------------------------------------------------- warm-start network
def test_conv3d_matches_scipy_correlate():
    """The plain convolution loops equal scipy.ndimage.correlate (zero padding) summed over
    input channels; catches a flipped kernel or a transposed tap index."""
    rng = np.random.default_rng(8)
    T, H, W, Cin, Cout = 3, 5, 6, 2, 3
    x = rng.normal(size=(T, H, W, Cin))
    wt = rng.normal(size=(Cout, 3, 3, 3, Cin))
    b = rng.normal(size=Cout)
    y = oracle.conv3d_fwd(x, wt, b)
    for co in range(Cout):
        ref = np.full((T, H, W), b[co])
        for ci in range(Cin):
            ref += scipy.ndimage.correlate(x[..., ci], wt[co, ..., ci], mode="constant", cval=0.0)
        np.testing.assert_allclose(y[..., co], ref, rtol=1e-12, atol=1e-12)


def test_conv3d_backward_matches_finite_differences():
    rng = np.random.default_rng(9)
    T, H, W, Cin, Cout = 2, 4, 3, 2, 2
    x = rng.normal(size=(T, H, W, Cin))
    wt = rng.normal(size=(Cout, 3, 3, 3, Cin))
    b = rng.normal(size=Cout)
    c = rng.normal(size=(T, H, W, Cout))
    L = lambda xx, ww, bb: float(np.sum(c * oracle.conv3d_fwd(xx, ww, bb)))
    dx, dw, db = oracle.conv3d_bwd(x, wt, c)
    h = 1e-6
    for idx in [(0, 1, 2, 1), (1, 3, 0, 0)]:
        e = np.zeros_like(x)
        e[idx] = h
        assert abs((L(x + e, wt, b) - L(x - e, wt, b)) / (2 * h) - dx[idx]) < 1e-6
    for idx in [(0, 1, 1, 1, 0), (1, 0, 2, 1, 1), (1, 2, 0, 0, 1)]:
        e = np.zeros_like(wt)
        e[idx] = h
        assert abs((L(x, wt + e, b) - L(x, wt - e, b)) / (2 * h) - dw[idx]) < 1e-6
    np.testing.assert_allclose(db, c.sum(axis=(0, 1, 2)), rtol=1e-12)


def test_cosine_loss_closed_forms():
    """The warm-start training loss 1 - cos(x0, target): 0 for any positive multiple of the
    target, 1 for orthogonal vectors, 1 - 1/sqrt(2) at 45 degrees, invariant to scaling either
    argument; its gradient is orthogonal to x0 (the loss does not change along x0) and equals
    central differences."""
    t = np.array([0.0, 3.0, 4.0])
    assert oracle.cosine_loss(2.5 * t, t)[0] == pytest.approx(0.0, abs=1e-15)
    assert oracle.cosine_loss(np.array([1.0, 0.0, 0.0]), t)[0] == pytest.approx(1.0)
    a, b = np.array([1.0, 0.0]), np.array([1.0, 1.0])
    assert oracle.cosine_loss(a, b)[0] == pytest.approx(1.0 - 1.0 / np.sqrt(2.0))
    rng = np.random.default_rng(12)
    x, g = rng.uniform(0.1, 1.0, 7), rng.uniform(0.1, 1.0, 7)
    l0, dx = oracle.cosine_loss(x, g)
    assert oracle.cosine_loss(4.0 * x, 0.5 * g)[0] == pytest.approx(l0, rel=1e-13)
    assert abs(np.dot(dx, x)) < 1e-13
    h = 1e-7
    for i in range(7):
        e = np.zeros(7)
        e[i] = h
        fd = (oracle.cosine_loss(x + e, g)[0] - oracle.cosine_loss(x - e, g)[0]) / (2 * h)
        assert abs(fd - dx[i]) < 1e-7


def test_warmstart_network_gradient_matches_finite_differences():
    rng = np.random.default_rng(10)
    C, T, H, W = 3, 3, 4, 5
    feats = rng.uniform(size=(C, T, H, W))
    target = rng.uniform(size=(T, H, W))
    dims = [C, 4, 4, 1]
    params = [(rng.normal(scale=0.3, size=(dims[i + 1], 3, 3, 3, dims[i])),
               rng.normal(scale=0.1, size=dims[i + 1])) for i in range(3)]
    loss, grads = oracle.warmstart_backward(feats, params, target)
    h = 1e-6
    for li, idx in [(0, (1, 0, 1, 2, 2)), (1, (3, 2, 2, 0, 1)), (2, (0, 1, 1, 1, 3))]:
        pp = [(w.copy(), b.copy()) for w, b in params]
        pm = [(w.copy(), b.copy()) for w, b in params]
        pp[li][0][idx] += h
        pm[li][0][idx] -= h
        fd = (oracle.warmstart_backward(feats, pp, target)[0]
              - oracle.warmstart_backward(feats, pm, target)[0]) / (2 * h)
        assert abs(fd - grads[li][0][idx]) < 1e-7 * max(1.0, abs(fd))


# ------------------------------------------------------------ Alg. 1 step 3, Sec. 4.1
def test_soft_binarize_kronecker_closed_form():
    """Constant f and x0 = the top eigenvector v of A (the Kronecker product of 1D dense
    eigenvectors, as above): y = lambda v, so one step gives sigmoid(gain (v / max v - c)) for any
    positive scale of x0.  Catches a dropped max scaling, a flipped sigmoid and a lost centre."""
    T, H, W = 4, 9, 11
    r = (1, 3, 2)
    sig = (0.8, 1.6, 1.1)
    f = np.full((T, H, W), 0.6)

    def band(n, ra, sa):
        d = np.arange(n)[:, None] - np.arange(n)[None, :]
        return np.where(np.abs(d) <= ra, np.exp(-d * d / (2 * sa * sa)), 0.0)

    vecs = []
    for n, ra, sa in zip((T, H, W), r, sig):
        _, V = np.linalg.eigh(band(n, ra, sa))
        vecs.append(np.abs(V[:, -1]))
    v = np.einsum("a,b,c->abc", *vecs)
    gain, c = 7.0, 0.55
    want = scipy.special.expit(gain * (v / v.max() - c))
    for scale in (1.0, 3.7e-4):
        x, mask = oracle.soft_binarize(f, f, 0.4, 0.9, r, scale * v, 1, gain, c, sigma=sig)
        np.testing.assert_allclose(x, want, rtol=1e-12, atol=1e-14)
        np.testing.assert_array_equal(mask, (want > 0.5).astype(np.uint8))


def test_soft_binarize_diagonal_two_steps():
    """Radius (0, 0, 0): A = diag(u^2 / alpha), so y = u^2 x / alpha and two steps from the
    uniform start are a closed form in u (catches steps applied in the wrong order, e.g. the
    sigmoid before the operator)."""
    rng = np.random.default_rng(17)
    f = _rand_volume(rng, 2, 5, 6, lo=0.1)
    p, alpha, gain, c = 0.45, 0.7, 5.0, 0.4
    u2 = f ** (2 * p)
    y1 = u2 / alpha
    x1 = scipy.special.expit(gain * (y1 / y1.max() - c))
    y2 = u2 * x1 / alpha
    x2 = scipy.special.expit(gain * (y2 / y2.max() - c))
    x, _ = oracle.soft_binarize(f, f, p, alpha, (0, 0, 0), np.ones(f.shape), 2, gain, c)
    np.testing.assert_allclose(x, x2, rtol=1e-13)


def test_soft_binarize_gain_limits():
    """gain 0: every voxel is sigmoid(0) = 1/2 exactly.  Large gain: x approaches the indicator
    of y / max y > c, and the hard mask equals it wherever y / max y is not within 1/gain of c."""
    rng = np.random.default_rng(3)
    f = _rand_volume(rng, 3, 12, 10, lo=0.05)
    x0 = rng.uniform(0.2, 1.0, size=f.shape)
    x, mask = oracle.soft_binarize(f, f, 0.5, 1.0, (1, 2, 2), x0, 1, 0.0, 0.5)
    assert np.all(x == 0.5) and not mask.any()
    y = oracle.filter_apply(f, f, 0.5, 1.0, (1, 2, 2), x0)
    q = y / y.max()
    gain = 1e4
    x, mask = oracle.soft_binarize(f, f, 0.5, 1.0, (1, 2, 2), x0, 1, gain, 0.5)
    clear = np.abs(q - 0.5) > 10.0 / gain
    assert clear.mean() > 0.9
    np.testing.assert_array_equal(mask[clear], (q[clear] > 0.5).astype(np.uint8))
    assert np.all(np.abs(x[clear] - (q[clear] > 0.5)) < 1e-4)


# ------------------------------------------------------------------------ Sec. 4.5
def _dense_top(f, p, alpha, radius, sigma=None):
    M = oracle.affinity(f, f, p, alpha, radius, sigma).toarray()
    e, V = scipy.linalg.eigh(M)
    v = V[:, -1]
    return (v * np.sign(v.sum())).reshape(f.shape)


def test_online_full_window_is_full_video_eigenvector():
    """q = T: after the last frame the sub-window is the whole video, so enough iterations give
    the principal eigenvector of the whole video's Eq. 2 matrix (dense LAPACK solver)."""
    rng = np.random.default_rng(21)
    V = rng.uniform(0.1, 1.0, size=(1, 4, 5, 6))
    out = oracle.online(V, None, 0.0, 0.3, 1.0, (1, 2, 2), q=4, iters=600)
    np.testing.assert_allclose(out[-1], _dense_top(V[0], 0.3, 1.0, (1, 2, 2)), atol=1e-9)


def test_online_single_frame_window():
    """q = 1: each frame is solved alone, so every output is the principal eigenvector of that
    frame's own 2D matrix."""
    rng = np.random.default_rng(22)
    V = rng.uniform(0.1, 1.0, size=(1, 3, 6, 7))
    out = oracle.online(V, None, 0.0, 0.2, 1.0, (1, 2, 2), q=1, iters=800)
    for k in range(3):
        np.testing.assert_allclose(out[k, 0], _dense_top(V[0, k:k + 1], 0.2, 1.0, (1, 2, 2))[0], atol=1e-9)


def test_online_start_vectors():
    """iters = 0 exposes the start vectors: the window holds the previous solution shifted by
    one frame and the new frame copies the previous newest one, uniform at the first frame, so
    from an all-uniform history each window is uniform on its min(k+1, q) real frames, zero on
    the frames before frame 0, normalised to 1."""
    rng = np.random.default_rng(23)
    T, q, H, W = 6, 4, 3, 5
    V = rng.uniform(0.1, 1.0, size=(2, T, H, W))
    out = oracle.online(V, np.array([0.5, -1.0]), 0.2, 0.3, 1.0, (1, 1, 1), q=q, iters=0)
    for k in range(T):
        n = min(k + 1, q)
        want = np.zeros((q, H, W))
        want[q - n:] = 1.0 / np.sqrt(n * H * W)
        np.testing.assert_allclose(out[k], want, rtol=1e-14, atol=0)


def test_online_diagonal_closed_form():
    """Radius (0, 0, 0): A = diag(u^2 / alpha), so K steps multiply the start by u^(2K) and the
    window solutions are closed forms in u.  With q = 2 the second window starts from
    (x_0, x_0) -- the first window's solution and its copy for the new frame -- and ends at
    (u_0^(2K) x_0, u_1^(2K) x_0) normalised, x_0 = u_0^(2K) / ||u_0^(2K)||.  Catches a new frame
    started from the uniform vector instead of the previous newest frame, and a shift in the
    wrong direction."""
    rng = np.random.default_rng(24)
    T, H, W, K, p = 3, 4, 5, 3, 0.4
    V = rng.uniform(0.2, 1.0, size=(1, T, H, W))
    out = oracle.online(V, None, 0.0, p, 1.0, (0, 0, 0), q=2, iters=K)
    u2k = V[0] ** (2 * p * K)
    x0 = u2k[0] / np.linalg.norm(u2k[0])
    np.testing.assert_allclose(out[0, 1], x0, rtol=1e-13)
    np.testing.assert_allclose(out[0, 0], 0.0, atol=0)
    w1 = np.stack([u2k[0] * x0, u2k[1] * x0])
    w1 /= np.linalg.norm(w1)
    np.testing.assert_allclose(out[1], w1, rtol=1e-13)
    w2 = np.stack([u2k[1] * w1[1], u2k[2] * w1[1]])
    w2 /= np.linalg.norm(w2)
    np.testing.assert_allclose(out[2], w2, rtol=1e-13)
