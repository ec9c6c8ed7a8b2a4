"""Thin Python binding of libsfseg.so (include/sfseg.h): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; PyTorch provides device
memory and the current stream.  There is no CPU fallback: if the library is missing this module
raises instead of computing anything.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsfseg.so")

SFSEG_F32, SFSEG_BF16 = 0, 1
INIT = {"user": 0, "uniform": 1, "smap": 2}
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "SHAPE", 3: "DTYPE", 4: "CUDA", 5: "OOM", 6: "TIMEOUT",
          7: "NONFINITE", 8: "ZERO_NORM", 9: "STATE", 10: "UNSUPPORTED"}

_lib = None


class SFSegError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sfseg error {STATUS.get(code, code)}: {msg}")
        self.code = code
        self.status = STATUS.get(code, str(code))


class Params(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("p", ctypes.c_double)]


class Neighborhood(ctypes.Structure):
    _fields_ = [("rt", ctypes.c_int), ("rh", ctypes.c_int), ("rw", ctypes.c_int),
                ("sigma_t", ctypes.c_float), ("sigma_h", ctypes.c_float), ("sigma_w", ctypes.c_float)]


_vp = ctypes.c_void_p
_i = ctypes.c_int
_f = ctypes.c_float
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)

# (name, argtypes) of every entry point declared in include/sfseg.h
SIGNATURES = {
    "sfseg_version": [],
    "sfseg_last_error": [],
    "sfseg_create": [ctypes.POINTER(Params), _i, _i, _i, _i, ctypes.POINTER(_vp)],
    "sfseg_destroy": [_vp],
    "sfseg_set_features": [_vp, _vp, _i, _fp, _f, _vp],
    "sfseg_power_iterate": [_vp, _vp, _i, _fp, _f, ctypes.POINTER(Neighborhood), _i, _i, _vp, _i, _i,
                            _dp, _vp],
    "sfseg_apply": [_vp, ctypes.POINTER(Neighborhood), _vp, _vp, _vp],
    "sfseg_apply_exact": [_vp, ctypes.POINTER(Neighborhood), _i, _vp, _vp, _vp],
    "sfseg_power_iterate_exact": [_vp, ctypes.POINTER(Neighborhood), _i, _i, _i, _vp, _dp, _vp],
    "sfseg_rayleigh": [_vp, ctypes.POINTER(Neighborhood), _vp, _dp, _dp, _vp],
    "sfseg_backward": [_vp, ctypes.POINTER(Neighborhood), _vp, _fp, _fp, _vp],
    "sfseg_soft_iou_loss": [_vp, _vp, _vp, _dp, _vp, _vp],
    "sfseg_set_features_sf": [_vp, _vp, _i, _i, _fp, _f, _vp, _i, _fp, _f, _vp],
    "sfseg_soft_binarize": [_vp, ctypes.POINTER(Neighborhood), _i, _f, _f, _vp, _vp, _vp],
    "sfseg_online_create": [ctypes.POINTER(Params), _i, _i, _i, _i, ctypes.POINTER(_vp)],
    "sfseg_online_destroy": [_vp],
    "sfseg_online_push": [_vp, _vp, _i, _fp, _f, ctypes.POINTER(Neighborhood), _i, _i, _i, _vp, _vp],
    "sfseg_online_window": [_vp, _vp, _vp],
    "sfseg_coarse_start": [_vp, ctypes.POINTER(Neighborhood), _i, ctypes.c_double, _i, _i, _vp,
                           ctypes.POINTER(_i), _vp],
    "sfseg_selftest_wait": [_vp, ctypes.c_longlong, _vp],
    "sfseg_enable_graphs": [_vp, _i],
    "sfseg_enable_iter_timing": [_vp, _i],
    "sfseg_iter_timing": [_vp, _dp, ctypes.POINTER(ctypes.c_int64)],
    "sfseg_kernel_launches": [ctypes.POINTER(ctypes.c_int64)],
    "sfseg_sumsq": [_vp, _vp, ctypes.c_int64, _vp, _vp],
    "sfseg_normalize": [_vp, _vp, ctypes.c_int64, _vp, _vp],
    "sfseg_check": [_vp, _vp],
    "sfseg_iterate_kernel_stats": [ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                   ctypes.c_char_p, _i],
    "sfseg_net_create": [_i, ctypes.c_uint64, ctypes.POINTER(_vp)],
    "sfseg_net_destroy": [_vp],
    "sfseg_net_num_params": [_vp, ctypes.POINTER(ctypes.c_int64)],
    "sfseg_net_get_params": [_vp, _fp, ctypes.c_int64],
    "sfseg_net_set_params": [_vp, _fp, ctypes.c_int64],
    "sfseg_net_forward": [_vp, _vp, _i, _i, _vp, _i, _i, _i, _vp, _vp],
    "sfseg_net_backward": [_vp, _vp, _i, _i, _vp, _i, _i, _i, _vp, _dp, _fp, _vp],
    "sfseg_net_adamw": [_vp, _f, _f, _f, _f, _f, _vp],
    "sfseg_net_layer_forward": [_vp, _i, _vp, _i, _i, _i, _vp, _vp, _vp],
    "sfseg_net_layer_backward": [_vp, _i, _vp, _vp, _i, _i, _i, _vp, _vp, _vp, _vp],
    "sfseg_net_check": [_vp, _vp],
    "sfseg_net_launch_shape": [_i, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i)],
    "sfseg_warmstart": [_vp, _vp, _vp, _i, _vp, _vp, _vp],
    "sfseg_power_iterate_noalloc": [ctypes.POINTER(Params), _i, _i, _i, _i, _vp, _i, _fp, _f,
                                    ctypes.POINTER(Neighborhood), _i, _vp, _i, _dp, _vp],
}


def lib(path: str | None = None):
    """Load libsfseg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build it with paper_2212_08058_gb300.build.build() "
                               "(there is no fallback implementation)")
        L = ctypes.CDLL(p)
        for name, args in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.sfseg_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise SFSegError(rc, lib().sfseg_last_error().decode())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: torch.Tensor | None):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return SFSEG_F32
    if t.dtype == torch.bfloat16:
        return SFSEG_BF16
    raise TypeError(f"unsupported dtype {t.dtype}: float32 or bfloat16")


def default_sigma(radius) -> tuple:
    """Isotropic Gaussian width sigma = max(radius) / 2 (1.0 when every radius is 0)."""
    s = max(radius) / 2.0 or 1.0
    return (s, s, s)


def neighborhood(radius, sigma=None) -> Neighborhood:
    rt, rh, rw = (int(r) for r in radius)
    st, sh, sw = default_sigma(radius) if sigma is None else sigma
    return Neighborhood(rt, rh, rw, float(st), float(sh), float(sw))


def _host_floats(w, n: int):
    if w is None:
        return None, None
    a = np.ascontiguousarray(np.asarray(w.detach().cpu() if torch.is_tensor(w) else w, dtype=np.float32))
    if a.size != n:
        raise ValueError(f"expected {n} channel weights, got {a.size}")
    return a, a.ctypes.data_as(_fp)


class PowerIteration:
    """A handle of the library for C-channel volumes of T x H x W voxels (sfseg_create)."""

    def __init__(self, C: int, T: int, H: int, W: int, alpha: float = 1.0, p: float = 0.1):
        self.shape = (C, T, H, W)
        self.C, self.T, self.H, self.W = C, T, H, W
        self.alpha, self.p = alpha, p
        h = ctypes.c_void_p()
        _check(lib().sfseg_create(ctypes.byref(Params(alpha, p)), C, T, H, W, ctypes.byref(h)))
        self._h = h
        self._features = None

    def close(self):
        if getattr(self, "_h", None):
            lib().sfseg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ----------------------------------------------------------------------------------
    def _check_features(self, features: torch.Tensor):
        if not features.is_cuda or not features.is_contiguous():
            raise ValueError("features must be a contiguous CUDA tensor")
        if tuple(features.shape) != self.shape:
            raise ValueError(f"features shape {tuple(features.shape)} != {self.shape}")

    def _check_volume(self, x: torch.Tensor, name: str):
        if x.dtype != torch.float32 or not x.is_cuda or not x.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
        if x.numel() != self.T * self.H * self.W:
            raise ValueError(f"{name} has {x.numel()} elements, expected {self.T * self.H * self.W}")

    def set_features(self, features: torch.Tensor, weights=None, bias: float = 0.0):
        self._check_features(features)
        _, wp = _host_floats(weights, self.C)
        _check(lib().sfseg_set_features(self._h, _ptr(features), _dtype_code(features), wp, float(bias),
                                        _stream()))
        self._features = features

    def set_features_sf(self, s_features: torch.Tensor, s_weights, s_bias: float, f_features: torch.Tensor,
                        f_weights=None, f_bias: float = 0.0):
        """Separate unary and pairwise maps (sfseg_set_features_sf): s_features [Cs, T, H, W],
        f_features [C, T, H, W]."""
        self._check_features(f_features)
        if (not s_features.is_cuda or not s_features.is_contiguous() or s_features.dim() != 4
                or tuple(s_features.shape[1:]) != (self.T, self.H, self.W)):
            raise ValueError("s_features must be a contiguous CUDA tensor [Cs, T, H, W]")
        Cs = s_features.shape[0]
        _, swp = _host_floats(s_weights, Cs)
        _, fwp = _host_floats(f_weights, self.C)
        _check(lib().sfseg_set_features_sf(self._h, _ptr(s_features), _dtype_code(s_features), int(Cs), swp,
                                           float(s_bias), _ptr(f_features), _dtype_code(f_features), fwp,
                                           float(f_bias), _stream()))
        self._features = f_features

    def power_iterate(self, features: torch.Tensor | None = None, weights=None, bias: float = 0.0,
                      radius=(2, 7, 7), sigma=None, iters: int = 50, iters_bf16: int = 0,
                      x: torch.Tensor | None = None, init: str = "uniform", record_every: int = 0,
                      return_norms: bool = False):
        """Run ``iters`` power iterations; returns the unit-norm x [T, H, W] (and the norms
        nu_k = ||A x_{k-1}|| when ``return_norms``, which synchronises)."""
        if features is not None:
            self._check_features(features)
            self._features = features
        _, wp = _host_floats(weights, self.C) if features is not None else (None, None)
        if x is None:
            x = torch.empty((self.T, self.H, self.W), device="cuda", dtype=torch.float32)
            if init == "user":
                raise ValueError("init='user' needs x")
        else:
            self._check_volume(x, "x")
        nb = neighborhood(radius, sigma)
        norms = np.empty(max(iters, 1)) if return_norms else None
        _check(lib().sfseg_power_iterate(
            self._h, _ptr(features), _dtype_code(features) if features is not None else 0, wp, float(bias),
            ctypes.byref(nb), int(iters), int(iters_bf16), _ptr(x), INIT[init], int(record_every),
            norms.ctypes.data_as(_dp) if norms is not None else None, _stream()))
        return (x, norms[:iters]) if return_norms else x

    def apply(self, x: torch.Tensor, radius=(2, 7, 7), sigma=None, out: torch.Tensor | None = None) -> torch.Tensor:
        """y = A x (the Eq. 7 operator, FP32), into `out` when given."""
        self._check_volume(x, "x")
        y = torch.empty_like(x) if out is None else out
        self._check_volume(y, "out")
        _check(lib().sfseg_apply(self._h, ctypes.byref(neighborhood(radius, sigma)), _ptr(x), _ptr(y), _stream()))
        return y

    def apply_exact(self, x: torch.Tensor, radius=(2, 7, 7), sigma=None, n_terms: int = 0) -> torch.Tensor:
        """y = (1/alpha) M x for the exact (Eq. 1) kernel (sfseg_apply_exact; n_terms = 0 picks the
        series length from alpha and max f, which synchronises)."""
        self._check_volume(x, "x")
        y = torch.empty_like(x)
        _check(lib().sfseg_apply_exact(self._h, ctypes.byref(neighborhood(radius, sigma)), int(n_terms), _ptr(x),
                                       _ptr(y), _stream()))
        return y

    def power_iterate_exact(self, radius=(2, 7, 7), sigma=None, iters: int = 50, x: torch.Tensor | None = None,
                            init: str = "uniform", n_terms: int = 0, return_norms: bool = False):
        """Power iteration on the exact kernel's operator (sfseg_power_iterate_exact) with the
        features already set; returns the unit-norm x [T, H, W] (and the norms when asked)."""
        if init not in ("uniform", "user"):
            raise ValueError("init must be 'uniform' or 'user'")
        if x is None:
            if init == "user":
                raise ValueError("init='user' needs x")
            x = torch.empty((self.T, self.H, self.W), device="cuda", dtype=torch.float32)
        else:
            self._check_volume(x, "x")
        norms = np.empty(max(iters, 1)) if return_norms else None
        _check(lib().sfseg_power_iterate_exact(
            self._h, ctypes.byref(neighborhood(radius, sigma)), int(n_terms), int(iters), INIT[init], _ptr(x),
            norms.ctypes.data_as(_dp) if norms is not None else None, _stream()))
        return (x, norms[:iters]) if return_norms else x

    def rayleigh(self, x: torch.Tensor, radius=(2, 7, 7), sigma=None):
        """(rho, residual) of x for the FP32 operator; synchronises."""
        self._check_volume(x, "x")
        rho = ctypes.c_double()
        res = ctypes.c_double()
        _check(lib().sfseg_rayleigh(self._h, ctypes.byref(neighborhood(radius, sigma)), _ptr(x),
                                    ctypes.byref(rho), ctypes.byref(res), _stream()))
        return rho.value, res.value

    def backward(self, grad_x: torch.Tensor, radius=(2, 7, 7), sigma=None):
        """(dL/dw [C] numpy float32, dL/db float) for the last recorded power_iterate call."""
        self._check_volume(grad_x, "grad_x")
        gw = np.zeros(self.C, dtype=np.float32)
        gb = ctypes.c_float()
        _check(lib().sfseg_backward(self._h, ctypes.byref(neighborhood(radius, sigma)), _ptr(grad_x),
                                    gw.ctypes.data_as(_fp), ctypes.byref(gb), _stream()))
        return gw, gb.value

    def soft_iou_loss(self, x: torch.Tensor, target: torch.Tensor, grad: bool = True):
        """(1 - soft-IoU(x / max x, target), dL/dx or None); synchronises."""
        self._check_volume(x, "x")
        self._check_volume(target, "target")
        g = torch.empty_like(x) if grad else None
        loss = ctypes.c_double()
        _check(lib().sfseg_soft_iou_loss(self._h, _ptr(x), _ptr(target), ctypes.byref(loss), _ptr(g), _stream()))
        return loss.value, g


    def soft_binarize(self, x: torch.Tensor, radius=(2, 7, 7), sigma=None, iters: int = 5, gain: float = 10.0,
                      center: float = 0.5, inplace: bool = False):
        """Soft-binarisation steps (Alg. 1 step 3, sfseg_soft_binarize) from the continuous
        solution x; returns (soft segmentation in (0, 1), hard mask uint8).  Synchronises."""
        self._check_volume(x, "x")
        xo = x if inplace else x.clone()
        mask = torch.empty((self.T, self.H, self.W), device="cuda", dtype=torch.uint8)
        _check(lib().sfseg_soft_binarize(self._h, ctypes.byref(neighborhood(radius, sigma)), int(iters), float(gain),
                                         float(center), _ptr(xo), _ptr(mask), _stream()))
        return xo, mask

    def segment(self, features: torch.Tensor | None = None, weights=None, bias: float = 0.0, radius=(2, 7, 7),
                sigma=None, n_iter: int = 60, n_cont: int = 50, gain: float = 10.0, center: float = 0.5,
                init: str = "uniform", x: torch.Tensor | None = None):
        """Alg. 1 end to end: n_cont continuous power iterations, then n_iter - n_cont
        soft-binarisation steps.  Returns (soft segmentation, hard mask)."""
        if not 0 <= n_cont < n_iter:
            raise ValueError("need 0 <= n_cont < n_iter")
        xc = self.power_iterate(features, weights, bias, radius, sigma, n_cont, x=x, init=init)
        return self.soft_binarize(xc, radius, sigma, n_iter - n_cont, gain, center, inplace=True)

    def coarse_start(self, radius=(2, 7, 7), sigma=None, levels: int = 2, tol: float = 1e-4,
                     max_iters: int = 3000, check_every: int = 20):
        """Start vector from the coarse-to-fine solve (sfseg_coarse_start); returns (x0, iterations
        per level, finest first).  Needs the features set; synchronises."""
        x0 = torch.empty((self.T, self.H, self.W), device="cuda", dtype=torch.float32)
        its = (ctypes.c_int * levels)()
        _check(lib().sfseg_coarse_start(self._h, ctypes.byref(neighborhood(radius, sigma)), int(levels), float(tol),
                                        int(max_iters), int(check_every), _ptr(x0), its, _stream()))
        return x0, list(its)

    def warmstart(self, net: "WarmStartNet", features: torch.Tensor, x_coarse: torch.Tensor | None = None) -> torch.Tensor:
        """x0 = net(features[, x_coarse]) for this handle's volume (sfseg_warmstart)."""
        self._check_features(features)
        if x_coarse is not None:
            self._check_volume(x_coarse, "x_coarse")
        x0 = torch.empty((self.T, self.H, self.W), device="cuda", dtype=torch.float32)
        _check(lib().sfseg_warmstart(self._h, net._n, _ptr(features), _dtype_code(features), _ptr(x_coarse),
                                     _ptr(x0), _stream()))
        return x0

    def sumsq(self, x: torch.Tensor, acc: torch.Tensor):
        """acc[0] += sum(x^2) (FP64 on the device; x float32 contiguous, acc float64 on the device)."""
        assert x.dtype == torch.float32 and x.is_contiguous() and acc.dtype == torch.float64
        _check(lib().sfseg_sumsq(self._h, _ptr(x), x.numel(), _ptr(acc), _stream()))

    def normalize(self, x: torch.Tensor, acc: torch.Tensor):
        """x *= 1/sqrt(acc[0]) in place (Eq. 8)."""
        assert x.dtype == torch.float32 and x.is_contiguous() and acc.dtype == torch.float64
        _check(lib().sfseg_normalize(self._h, _ptr(x), x.numel(), _ptr(acc), _stream()))

    def check(self):
        """Synchronise and raise for device-side errors (TIMEOUT, NONFINITE, ZERO_NORM)."""
        _check(lib().sfseg_check(self._h, _stream()))

    def selftest_wait(self, spins: int = 1000):
        """Run the bounded-wait failure path on purpose (sfseg_selftest_wait); raises SFSegError
        with status TIMEOUT, which is the expected outcome."""
        _check(lib().sfseg_selftest_wait(self._h, int(spins), _stream()))

    def enable_graphs(self, on: bool = True):
        """Run feature-less power_iterate calls as replayed CUDA graphs (sfseg_enable_graphs)."""
        _check(lib().sfseg_enable_graphs(self._h, int(bool(on))))

    def enable_iter_timing(self, on: bool = True):
        _check(lib().sfseg_enable_iter_timing(self._h, int(bool(on))))

    def iter_timing(self):
        """(milliseconds, launches) of the iteration kernels since the last read (CUDA events)."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        _check(lib().sfseg_iter_timing(self._h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value


class OnlineStream:
    """Partial iterations on a stream of frames (Sec. 4.5; sfseg_online_*): a sub-window of the
    q most recent frames, re-solved with a few iterations whenever a frame arrives."""

    def __init__(self, C: int, q: int, H: int, W: int, alpha: float = 1.0, p: float = 0.1):
        self.C, self.q, self.H, self.W = C, q, H, W
        o = ctypes.c_void_p()
        _check(lib().sfseg_online_create(ctypes.byref(Params(alpha, p)), C, q, H, W, ctypes.byref(o)))
        self._o = o

    def close(self):
        if getattr(self, "_o", None):
            lib().sfseg_online_destroy(self._o)
            self._o = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def push(self, frame: torch.Tensor, weights=None, bias: float = 0.0, radius=(2, 7, 7), sigma=None,
             iters: int = 5, iters_bf16: int = 0, lag: int = 0) -> torch.Tensor:
        """Push frame [C, H, W]; returns the window solution's slice of frame k - lag [H, W]."""
        if not frame.is_cuda or not frame.is_contiguous() or tuple(frame.shape) != (self.C, self.H, self.W):
            raise ValueError(f"frame must be a contiguous CUDA tensor of shape {(self.C, self.H, self.W)}")
        _, wp = _host_floats(weights, self.C)
        out = torch.empty((self.H, self.W), device="cuda", dtype=torch.float32)
        _check(lib().sfseg_online_push(self._o, _ptr(frame), _dtype_code(frame), wp, float(bias),
                                       ctypes.byref(neighborhood(radius, sigma)), int(iters), int(iters_bf16),
                                       int(lag), _ptr(out), _stream()))
        return out

    def window(self) -> torch.Tensor:
        out = torch.empty((self.q, self.H, self.W), device="cuda", dtype=torch.float32)
        _check(lib().sfseg_online_window(self._o, _ptr(out), _stream()))
        return out


class WarmStartNet:
    """The learned warm-start network (sfseg_net_*): x0 = net(channels) on the tensor cores."""

    def __init__(self, c_in: int = 8, seed: int = 0):
        n = ctypes.c_void_p()
        _check(lib().sfseg_net_create(int(c_in), ctypes.c_uint64(seed), ctypes.byref(n)))
        self._n = n
        self.c_in = c_in
        cnt = ctypes.c_int64()
        _check(lib().sfseg_net_num_params(self._n, ctypes.byref(cnt)))
        self.num_params = cnt.value

    def close(self):
        if getattr(self, "_n", None):
            lib().sfseg_net_destroy(self._n)
            self._n = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        a = np.empty(self.num_params, dtype=np.float32)
        _check(lib().sfseg_net_get_params(self._n, a.ctypes.data_as(_fp), a.size))
        return a

    def set_params(self, a) -> None:
        a = np.ascontiguousarray(a, dtype=np.float32)
        _check(lib().sfseg_net_set_params(self._n, a.ctypes.data_as(_fp), a.size))

    def unflatten(self, flat: np.ndarray):
        """[(W1, b1), ..., (W4, b4)] with W as [out, 3, 3, 3, in] views of a flat vector."""
        dims = [(32, self.c_in), (32, 32), (32, 32), (1, 32)]
        out, o = [], 0
        for co, ci in dims:
            w = flat[o:o + co * 27 * ci].reshape(co, 3, 3, 3, ci)
            o += co * 27 * ci
            b = flat[o:o + co]
            o += co
            out.append((w, b))
        return out

    def forward(self, features: torch.Tensor, extra: torch.Tensor | None = None) -> torch.Tensor:
        C, T, H, W = features.shape
        x0 = torch.empty((T, H, W), device="cuda", dtype=torch.float32)
        _check(lib().sfseg_net_forward(self._n, _ptr(features), _dtype_code(features), C, _ptr(extra), T, H, W,
                                       _ptr(x0), _stream()))
        return x0

    def backward(self, features: torch.Tensor, target: torch.Tensor, want_grads: bool = False,
                 extra: torch.Tensor | None = None):
        C, T, H, W = features.shape
        loss = ctypes.c_double()
        g = np.empty(self.num_params, dtype=np.float32) if want_grads else None
        _check(lib().sfseg_net_backward(self._n, _ptr(features), _dtype_code(features), C, _ptr(extra), T, H, W,
                                        _ptr(target.contiguous()), ctypes.byref(loss),
                                        g.ctypes.data_as(_fp) if g is not None else None, _stream()))
        return (loss.value, g) if want_grads else loss.value

    def adamw(self, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
              weight_decay: float = 0.0):
        _check(lib().sfseg_net_adamw(self._n, lr, beta1, beta2, eps, weight_decay, _stream()))

    def layer_forward(self, layer: int, x: torch.Tensor):
        """One layer on a channels-last bf16 activation x [T, H, W, 16 or 32]: bf16 [T, H, W, 32]
        for layers 0..2, (z, softplus(z)) float32 [T, H, W] for layer 3."""
        assert x.dtype == torch.bfloat16 and x.is_contiguous() and x.dim() == 4
        T, H, W, _ = x.shape
        if layer < 3:
            out = torch.empty((T, H, W, 32), device=x.device, dtype=torch.bfloat16)
            _check(lib().sfseg_net_layer_forward(self._n, layer, _ptr(x), T, H, W, _ptr(out), None, _stream()))
            return out
        z = torch.empty((T, H, W), device=x.device, dtype=torch.float32)
        x0 = torch.empty_like(z)
        _check(lib().sfseg_net_layer_forward(self._n, layer, _ptr(x), T, H, W, _ptr(z), _ptr(x0), _stream()))
        return z, x0

    def layer_backward(self, layer: int, x: torch.Tensor, dz: torch.Tensor, want_dx: bool = True):
        """Gradients of one layer: (dx bf16 [T, H, W, 32] or None, dW float32 [COUT, 3, 3, 3, CIN],
        db float32 [COUT]) for its input x and the gradient dz at its pre-activation output."""
        assert x.dtype == torch.bfloat16 and dz.dtype == torch.bfloat16
        T, H, W, _ = x.shape
        cout, cin = (1, 32) if layer == 3 else (32, self.c_in if layer == 0 else 32)
        dW = torch.empty((cout, 3, 3, 3, cin), device=x.device, dtype=torch.float32)
        db = torch.empty((cout,), device=x.device, dtype=torch.float32)
        dx = torch.empty((T, H, W, 32), device=x.device, dtype=torch.bfloat16) if (want_dx and layer > 0) else None
        _check(lib().sfseg_net_layer_backward(self._n, layer, _ptr(x.contiguous()), _ptr(dz.contiguous()), T, H, W,
                                              _ptr(dx), _ptr(dW), _ptr(db), _stream()))
        return dx, dW, db

    def check(self):
        """Synchronise; raise TIMEOUT if a bounded wait in the network's kernels gave up."""
        _check(lib().sfseg_net_check(self._n, _stream()))


def kernel_launches() -> int:
    """Kernels launched by libsfseg.so in this process so far."""
    n = ctypes.c_int64()
    _check(lib().sfseg_kernel_launches(ctypes.byref(n)))
    return n.value


def net_launch_shape(kernel: int):
    """(output frames per CTA, output rows per CTA, CTAs) of this thread's most recent launch of
    the network's hidden-layer convolution kernel (kernel 0) or of its last layer's (kernel 1)."""
    f, r, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().sfseg_net_launch_shape(kernel, ctypes.byref(f), ctypes.byref(r), ctypes.byref(c)))
    return f.value, r.value, c.value


def iterate_kernel_stats():
    """(steps on the TMA kernel, steps on the generic stencil, name of the last step's kernel),
    process-wide."""
    a, b = ctypes.c_int64(), ctypes.c_int64()
    buf = ctypes.create_string_buffer(128)
    _check(lib().sfseg_iterate_kernel_stats(ctypes.byref(a), ctypes.byref(b), buf, len(buf)))
    return a.value, b.value, buf.value.decode()


class SFSegFunction(torch.autograd.Function):
    """x_K = SFSeg++(features; w, b) as a differentiable function of the channel weights and bias
    (Sec. 3.4): the forward records checkpoints, the backward runs the library's adjoint."""

    @staticmethod
    def forward(ctx, weights, bias, features, handle: PowerIteration, radius, sigma, iters, record_every):
        x = handle.power_iterate(features, weights.detach().cpu().numpy(), float(bias), radius, sigma, iters,
                                 record_every=record_every)
        ctx.handle, ctx.radius, ctx.sigma = handle, radius, sigma
        ctx.wdev, ctx.bdev = weights.device, bias.device if torch.is_tensor(bias) else None
        return x

    @staticmethod
    def backward(ctx, grad_x):
        gw, gb = ctx.handle.backward(grad_x.contiguous(), ctx.radius, ctx.sigma)
        gw_t = torch.from_numpy(gw).to(ctx.wdev)
        gb_t = torch.tensor(gb, dtype=torch.float32, device=ctx.bdev) if ctx.bdev is not None else None
        return gw_t, gb_t, None, None, None, None, None, None


def sfseg_pp(weights, bias, features, handle, radius=(1, 3, 3), sigma=None, iters=30, record_every=5):
    return SFSegFunction.apply(weights, bias, features, handle, radius, sigma, iters, record_every)
