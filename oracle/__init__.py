"""Plain FP64 CPU oracle for the SFSeg / SFSeg++ power iteration (arXiv 2212.08058).

TEST INFRASTRUCTURE ONLY.  Only the test suite (with ``tests/golden/make_golden.py``),
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg and ``--impl reference`` arm may
import this package.  It shares no code with the CUDA library
(``paper_2212_08058_gb300``) and never imports it; both sides receive the same seeded inputs
from ``paper_2212_08058_gb300.synth``, which holds no arithmetic of the method.

What each function computes, and the passage it follows:

============================  ===============================================================
``combine``                   Eq. 9 channel combination (sigmoid), single channel passes through
                              unchanged (Alg. 1, initialisation note)
``affinity``                  Eq. 2 first-order Taylor affinity (Eq. 1 with ``exact=True``) as
                              an explicit sparse matrix
``power_csr``                 Eq. 4 power iteration + Eq. 8 renormalisation on that matrix
``filter_apply``              Eq. 7 three-Gaussian-filter form (returns M x / alpha)
``power_filter``              Eq. 7 + Eq. 8 iterated (for volumes too large for a matrix)
``soft_binarize``             Alg. 1 step 3 / Sec. 4.1 soft-binarisation iterations and the
                              final hard threshold
``online``                    Sec. 4.5 partial iterations on sub-windows of a frame stream
``rayleigh``                  Eq. 3 Rayleigh quotient and the eigen-residual ||Mx - rho x|| / rho
``grad_csr``                  derivative of a loss of x_K w.r.t. the Eq. 9 weights (Sec. 3.4)
``soft_iou_loss``             1 - soft-IoU of the max-normalised x against a target mask
``conv3d_fwd`` / ``_bwd``     plain 3x3x3 convolution loops (warm-start network)
``warmstart_forward``         the 4-layer warm-start network, FP64, from those loops
============================  ===============================================================

Readings of the paper that these functions take (the paper is silent or garbled there):
the sigmoid is the standard logistic 1/(1+e^-z); the operator between the second and third
lines of Eq. 6 is "+"; the Eq. 7 filter operator is A = M/alpha; the Gaussian is
exp(-0.5 sum_a d_a^2 / sigma_a^2), unnormalised, truncated to the box of radii (rt, rh, rw);
the border is zero padding; every frame is updated each iteration; the soft-binarisation
sigmoid acts on the new vector scaled to maximum 1, x <- sigmoid(gain (y / max y - center)),
and the hard segmentation is x > 1/2; the online sub-window of q frames ends at the newest frame,
its overlap starts from the previous window's final solution and the new frame from the previous
newest frame's (uniform for the first frame).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sfseg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP) into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_build_affinity.restype = ctypes.c_int64
            lib.orc_sumsq.restype = ctypes.c_double
            lib.orc_dot.restype = ctypes.c_double
            lib.orc_power_csr.restype = ctypes.c_int
            lib.orc_power_filter.restype = ctypes.c_int
            lib.orc_grad_csr.restype = ctypes.c_int
            lib.orc_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _d(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _c64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    """OpenMP threads the C oracle uses."""
    return int(_load().orc_num_threads())


def set_num_threads(n: int) -> None:
    _load().orc_set_num_threads(ctypes.c_int(int(n)))


def default_sigma(radius) -> tuple:
    """Default Gaussian widths: isotropic sigma = max(radius)/2 (1.0 when every radius is 0)."""
    rt, rh, rw = radius
    s = max(rt, rh, rw) / 2.0 or 1.0
    return (s, s, s)


# ----------------------------------------------------------------------------------- Eq. 9
def combine(V: np.ndarray, w=None, b: float = 0.0) -> np.ndarray:
    """Eq. 9: f = sigmoid(sum_c w_c V_c + b); for one channel f = V_0 (no sigmoid).

    V has shape [C, T, H, W]; returns [T, H, W] float64."""
    V = _c64(V)
    C = V.shape[0]
    N = int(np.prod(V.shape[1:]))
    f = np.empty(V.shape[1:], dtype=np.float64)
    wv = _c64(np.zeros(C) if w is None else w)
    _load().orc_combine(ctypes.c_int64(C), ctypes.c_int64(N), _d(V), _d(wv), ctypes.c_double(b), _d(f))
    return f


def taps(r: int, sigma: float) -> np.ndarray:
    g = np.empty(2 * r + 1)
    _load().orc_taps(ctypes.c_int(r), ctypes.c_double(sigma), _d(g))
    return g


# ----------------------------------------------------------------------------------- Eq. 2
def affinity(s: np.ndarray, f: np.ndarray, p: float, alpha: float, radius, sigma=None,
             exact: bool = False):
    """Eq. 2 (or Eq. 1 if ``exact``) as a scipy CSR matrix of shape [N, N].

    ``s`` (unary map) and ``f`` (pairwise map) have shape [T, H, W]."""
    import scipy.sparse as sp
    s = _c64(s)
    f = _c64(f)
    T, H, W = s.shape
    rt, rh, rw = radius
    st, sh, sw = default_sigma(radius) if sigma is None else sigma
    N = T * H * W
    cap = N * (2 * rt + 1) * (2 * rh + 1) * (2 * rw + 1)
    rowptr = np.empty(N + 1, dtype=np.int64)
    col = np.empty(cap, dtype=np.int64)
    val = np.empty(cap, dtype=np.float64)
    nnz = _load().orc_build_affinity(
        T, H, W, _d(s), _d(f), ctypes.c_double(p), ctypes.c_double(alpha), rt, rh, rw,
        ctypes.c_double(st), ctypes.c_double(sh), ctypes.c_double(sw), int(bool(exact)),
        rowptr.ctypes.data_as(_i64p), col.ctypes.data_as(_i64p), _d(val))
    return sp.csr_matrix((val[:nnz].copy(), col[:nnz].copy(), rowptr), shape=(N, N))


# ------------------------------------------------------------------------------- Eq. 4, 8
def power_csr(M, x0: np.ndarray, K: int):
    """Eq. 4 + Eq. 8: K normalised steps x <- Mx/||Mx|| from x0/||x0||.

    Returns (x_K, nu) with nu[k] = ||M x_k||."""
    N = M.shape[0]
    x0 = _c64(x0).reshape(-1)
    indptr = np.ascontiguousarray(M.indptr, dtype=np.int64)
    indices = np.ascontiguousarray(M.indices, dtype=np.int64)
    data = _c64(M.data)
    x = np.empty(N)
    nu = np.empty(max(K, 1))
    rc = _load().orc_power_csr(ctypes.c_int64(N), indptr.ctypes.data_as(_i64p),
                               indices.ctypes.data_as(_i64p), _d(data), _d(x0), int(K), _d(x), _d(nu))
    if rc != 0:
        raise FloatingPointError("zero norm in power iteration")
    return x, nu[:K]


# ----------------------------------------------------------------------------------- Eq. 7
def filter_apply(s, f, p: float, alpha: float, radius, x, sigma=None) -> np.ndarray:
    """Eq. 7: y = A x with A = M / alpha, computed with three separable Gaussian filterings."""
    s = _c64(s)
    f = _c64(f)
    T, H, W = s.shape
    rt, rh, rw = radius
    st, sh, sw = default_sigma(radius) if sigma is None else sigma
    x = _c64(x).reshape(T, H, W)
    y = np.empty_like(x)
    _load().orc_filter_apply(T, H, W, _d(s), _d(f), ctypes.c_double(p), ctypes.c_double(alpha),
                             rt, rh, rw, ctypes.c_double(st), ctypes.c_double(sh),
                             ctypes.c_double(sw), _d(x), _d(y))
    return y


def power_filter(s, f, p: float, alpha: float, radius, x0, K: int, sigma=None):
    """Eq. 7 + Eq. 8 iterated K times from x0/||x0||.  Returns (x_K, nu), nu[k] = ||A x_k||."""
    s = _c64(s)
    f = _c64(f)
    T, H, W = s.shape
    rt, rh, rw = radius
    st, sh, sw = default_sigma(radius) if sigma is None else sigma
    x0 = _c64(x0).reshape(T, H, W)
    x = np.empty_like(x0)
    nu = np.empty(max(K, 1))
    rc = _load().orc_power_filter(T, H, W, _d(s), _d(f), ctypes.c_double(p), ctypes.c_double(alpha),
                                  rt, rh, rw, ctypes.c_double(st), ctypes.c_double(sh),
                                  ctypes.c_double(sw), _d(x0), int(K), _d(x), _d(nu))
    if rc != 0:
        raise FloatingPointError("zero norm in power iteration")
    return x, nu[:K]


def soft_binarize(s, f, p: float, alpha: float, radius, x0, K: int, gain: float, center: float = 0.5,
                  sigma=None):
    """Alg. 1 step 3 (Sec. 4.1): K soft-binarisation steps x <- sigmoid(gain (y / max y - center)),
    y = A x (Eq. 7), from x0.  Returns (x_K, hard mask x_K > 1/2 as uint8)."""
    s = _c64(s)
    f = _c64(f)
    T, H, W = s.shape
    rt, rh, rw = radius
    st, sh, sw = default_sigma(radius) if sigma is None else sigma
    x0 = _c64(x0).reshape(T, H, W)
    x = np.empty_like(x0)
    rc = _load().orc_soft_binarize(T, H, W, _d(s), _d(f), ctypes.c_double(p), ctypes.c_double(alpha),
                                   rt, rh, rw, ctypes.c_double(st), ctypes.c_double(sh),
                                   ctypes.c_double(sw), _d(x0), int(K), ctypes.c_double(gain),
                                   ctypes.c_double(center), _d(x))
    if rc != 0:
        raise FloatingPointError("max(A x) <= 0 in a soft-binarisation step")
    return x, (x > 0.5).astype(np.uint8)


def online(V, w, b: float, p: float, alpha: float, radius, q: int, iters: int, sigma=None):
    """Sec. 4.5 partial iterations on a stream of frames V [C, T, H, W] (the online form of
    Alg. 1): when frame k arrives the sub-window is frames k-q+1 .. k (all-zero features before
    frame 0), started from the previous window's final solution shifted by one frame, with the
    new frame started from the previous newest frame's solution (uniform at k = 0); then `iters`
    steps of Eq. 7 + Eq. 8 on the window.  Returns the window solutions, shape [T, q, H, W]
    (index [k, q-1] is the newest frame's slice after frame k)."""
    V = _c64(V)
    C, T, H, W = V.shape
    f_all = combine(V, w, b)
    fw = np.zeros((q, H, W))
    xw = np.zeros((q, H, W))
    out = np.empty((T, q, H, W))
    for k in range(T):
        fw = np.concatenate([fw[1:], f_all[k:k + 1]])
        newest = xw[-1] if k > 0 else np.ones((H, W))
        xw = np.concatenate([xw[1:], newest[None]])
        xw, _ = power_filter(fw, fw, p, alpha, radius, xw, iters, sigma=sigma)
        out[k] = xw
    return out


def sumsq(x) -> float:
    x = _c64(x).reshape(-1)
    return float(_load().orc_sumsq(_d(x), ctypes.c_int64(x.size)))


def dot(x, y) -> float:
    x = _c64(x).reshape(-1)
    y = _c64(y).reshape(-1)
    return float(_load().orc_dot(_d(x), _d(y), ctypes.c_int64(x.size)))


# ----------------------------------------------------------------------------------- Eq. 3
def rayleigh(apply, x):
    """Eq. 3: rho = x'Ax / x'x and the residual ||Ax - rho x|| / rho for an operator ``apply``."""
    x = _c64(x).reshape(-1)
    y = _c64(apply(x)).reshape(-1)
    rho = dot(x, y) / sumsq(x)
    r = np.sqrt(sumsq(y - rho * x) / sumsq(x)) / rho
    return rho, float(r)


# ------------------------------------------------------------------------------- Sec. 3.4
def grad_csr(V, w, b: float, p: float, alpha: float, radius, x0, K: int, gK, sigma=None):
    """dL/dw, dL/db through K steps of Eq. 4 + Eq. 8 on the Eq. 2 matrix of f = Eq. 9(V; w, b).

    ``gK`` = dL/dx_K.  Tiny volumes only (explicit matrix, all iterates kept)."""
    V = _c64(V)
    C, T, H, W = V.shape
    rt, rh, rw = radius
    st, sh, sw = default_sigma(radius) if sigma is None else sigma
    wv = _c64(w)
    x0 = _c64(x0).reshape(-1)
    gK = _c64(gK).reshape(-1)
    gw = np.empty(C)
    gb = ctypes.c_double(0.0)
    rc = _load().orc_grad_csr(T, H, W, C, _d(V), _d(wv), ctypes.c_double(b), ctypes.c_double(p),
                              ctypes.c_double(alpha), rt, rh, rw, ctypes.c_double(st),
                              ctypes.c_double(sh), ctypes.c_double(sw), _d(x0), int(K), _d(gK),
                              _d(gw), ctypes.byref(gb))
    if rc != 0:
        raise ValueError("grad_csr needs C > 1")
    return gw, float(gb.value)


# ------------------------------------------------------------------------- learning loss
def soft_iou_loss(x, g):
    """1 - soft-IoU(xh, g) with xh = x / max(x):  soft-IoU = sum(xh g) / sum(xh + g - xh g).

    Returns (loss, dloss/dx).  The max is differentiated as a subgradient on its first
    (lowest linear index) argmax."""
    x = _c64(x).reshape(-1)
    g = _c64(g).reshape(-1)
    m_idx = int(np.argmax(x))
    m = x[m_idx]
    xh = x / m
    inter = float(np.sum(xh * g))
    union = float(np.sum(xh + g - xh * g))
    loss = 1.0 - inter / union
    # d loss / d xh_i = -(g_i * union - inter * (1 - g_i)) / union^2
    dxh = -(g * union - inter * (1.0 - g)) / (union * union)
    dx = dxh / m
    dx[m_idx] -= float(np.sum(dxh * x)) / (m * m)
    return loss, dx


# --------------------------------------------------------------------- warm-start network
def conv3d_fwd(x, wt, bias=None):
    """3x3x3 cross-correlation, zero padding 1.  x [T,H,W,Cin], wt [Cout,3,3,3,Cin]."""
    x = _c64(x)
    wt = _c64(wt)
    T, H, W, Cin = x.shape
    Cout = wt.shape[0]
    y = np.empty((T, H, W, Cout))
    bb = _c64(bias) if bias is not None else None
    _load().orc_conv3d_fwd(T, H, W, Cin, Cout, _d(x), _d(wt), _d(bb) if bb is not None else None, _d(y))
    return y


def conv3d_bwd(x, wt, dy, need_dx: bool = True):
    """Gradients of ``conv3d_fwd``: returns (dx or None, dw, db)."""
    x = _c64(x)
    wt = _c64(wt)
    dy = _c64(dy)
    T, H, W, Cin = x.shape
    Cout = wt.shape[0]
    dx = np.empty_like(x) if need_dx else None
    dw = np.empty_like(wt)
    db = np.empty(Cout)
    _load().orc_conv3d_bwd(T, H, W, Cin, Cout, _d(x), _d(wt), _d(dy),
                           _d(dx) if dx is not None else None, _d(dw), _d(db))
    return dx, dw, db


def softplus(z):
    return np.logaddexp(0.0, z)


def warmstart_forward(feats, params):
    """FP64 forward of the warm-start network: three 3x3x3 conv + ReLU layers and a 3x3x3 conv
    to one channel followed by softplus (a strictly positive start vector).

    ``feats`` [C, T, H, W]; ``params`` = [(w1, b1), ..., (w4, b4)] with w [Cout,3,3,3,Cin].
    Returns (x0 [T,H,W], activations) where activations are the per-layer (input, pre-act)."""
    a = np.moveaxis(_c64(feats), 0, -1)
    acts = []
    for li, (wt, b) in enumerate(params):
        z = conv3d_fwd(a, wt, b)
        acts.append((a, z))
        a = np.maximum(z, 0.0) if li < len(params) - 1 else softplus(z)
    return a[..., 0], acts


def cosine_loss(x0, target):
    """1 - <x0, t> / (||x0|| ||t||): the direction of the start vector is what matters."""
    x0 = _c64(x0).reshape(-1)
    t = _c64(target).reshape(-1)
    nx = np.sqrt(sumsq(x0))
    nt = np.sqrt(sumsq(t))
    c = dot(x0, t) / (nx * nt)
    grad = -(t / (nx * nt) - c * x0 / (nx * nx))
    return 1.0 - c, grad


def warmstart_backward(feats, params, target):
    """Loss (cosine_loss of the network output against ``target``) and its parameter gradients,
    FP64 reverse pass through the plain convolution loops."""
    x0, acts = warmstart_forward(feats, params)
    loss, g = cosine_loss(x0, target)
    grads = [None] * len(params)
    da = g.reshape(x0.shape)[..., None]
    for li in range(len(params) - 1, -1, -1):
        a_in, z = acts[li]
        if li == len(params) - 1:
            dz = da * (1.0 / (1.0 + np.exp(-z)))          # softplus' = logistic
        else:
            dz = da * (z > 0.0)
        dx, dw, db = conv3d_bwd(a_in, params[li][0], dz, need_dx=li > 0)
        grads[li] = (dw, db)
        da = dx
    return loss, grads
