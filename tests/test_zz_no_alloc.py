"""sfseg_power_iterate_noalloc -- the power iteration for callers that cannot allocate device
memory (a fixed memory budget reserved at start-up, latency-bound loops where cudaMalloc would
synchronise the device, plug-ins without a long-lived workspace).

Called through the C ABI several times in a row, it must give what the handle-based
sfseg_power_iterate gives (same kernels, tolerance of the forward parity tests), match the FP64
oracle directly (float32 and bf16 features), leave no stale state behind between calls that
share its scratch, and not change the device's free memory.
This file is collected last so that a failure here does not hide any other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2212_08058_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5


@pytest.fixture(scope="module")
def sf():
    from paper_2212_08058_gb300 import build, sfseg
    build.build()
    oracle.build()
    return sfseg


def _call(sf, feats, x, weights, radius, iters, init, norms, alpha=1.0, p=0.1):
    """One call of the entry point on tensors that already live on the device."""
    C, T, H, W = feats.shape
    nb = sf.neighborhood(radius)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float32)
    dtype = sf.SFSEG_BF16 if feats.dtype == torch.bfloat16 else sf.SFSEG_F32
    rc = sf.lib().sfseg_power_iterate_noalloc(
        ctypes.byref(sf.Params(alpha, p)), C, T, H, W, ctypes.c_void_p(feats.data_ptr()), dtype,
        w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if w is not None else None, 0.0, ctypes.byref(nb),
        iters, ctypes.c_void_p(x.data_ptr()), sf.INIT[init], norms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, sf.lib().sfseg_last_error().decode()


def _noalloc(sf, V, weights, radius, iters, init, bf16=False):
    C, T, H, W = V.shape
    feats = torch.from_numpy(np.ascontiguousarray(V)).cuda()
    if bf16:
        feats = feats.to(torch.bfloat16)
    x = torch.empty((T, H, W), device="cuda")
    norms = np.empty(max(iters, 1))
    _call(sf, feats, x, weights, radius, iters, init, norms)
    torch.cuda.synchronize()
    return x.cpu().numpy(), norms[:iters]


def _handle(sf, V, weights, radius, iters, init, x0=None, bf16=False):
    C, T, H, W = V.shape
    with sf.PowerIteration(C, T, H, W) as h:
        x = None if x0 is None else torch.from_numpy(np.ascontiguousarray(x0, dtype=np.float32)).cuda()
        feats = torch.from_numpy(np.ascontiguousarray(V)).cuda()
        if bf16:
            feats = feats.to(torch.bfloat16)
        x, nu = h.power_iterate(feats, weights, 0.0, radius, iters=iters, x=x, init=init, return_norms=True)
        torch.cuda.synchronize()
        return x.cpu().numpy(), nu


def test_noalloc_matches_handle_on_consecutive_calls(sf):
    A = synth.drifting_blob(8, 64, 64, seed=1000)
    B, _, wB = synth.multichannel(6, 48, 80, C=3, seed=3003)
    cases = [
        (A, None, (1, 3, 3), 20, "uniform"),
        (B, wB * 4.0, (2, 7, 7), 9, "smap"),      # different shape, channels, radius, start
        (A, None, (1, 3, 3), 20, "uniform"),      # back to the first: nothing left over
    ]
    for V, w, r, K, init in cases:
        xn, nun = _noalloc(sf, V, w, r, K, init)
        xh, nuh = _handle(sf, V, w, r, K, init)
        assert np.abs(xn.astype(np.float64) - xh.astype(np.float64)).max() <= TOL_F32
        np.testing.assert_allclose(nun, nuh, rtol=1e-5)


def _oracle(V, weights, radius, iters, init, p=0.1, alpha=1.0):
    """The FP64 oracle on the same (already rounded) features: Eq. 9, then Eq. 7 + Eq. 8."""
    V = np.asarray(V, dtype=np.float64)
    f = oracle.combine(V, weights) if V.shape[0] > 1 else V[0]
    x0 = f if init == "smap" else np.ones(f.shape)
    return oracle.power_filter(f, f, p, alpha, radius, x0, iters)


@pytest.mark.parametrize("bf16", [False, True], ids=["f32_features", "bf16_features"])
def test_noalloc_matches_oracle(sf, bf16):
    """One call per feature type against the FP64 oracle (iterate parity at equal iteration
    count, 1e-5 max-abs on the unit-norm x, the forward tests' tolerance), and against the handle
    path with the same features.  bf16 features are widened exactly on both sides; the iterate
    storage stays float32."""
    cases = [(synth.drifting_blob(8, 64, 64, seed=1000), None, (1, 3, 3), 20, "uniform")]
    V3, _, w3 = synth.multichannel(6, 48, 80, C=3, seed=3005)
    cases.append((V3, w3 * 4.0, (2, 7, 7), 12, "smap"))
    for V, w, r, K, init in cases:
        Vr = synth.to_bf16_round(V) if bf16 else V
        xn, nun = _noalloc(sf, V, w, r, K, init, bf16=bf16)
        xo, nuo = _oracle(Vr, w, r, K, init)
        assert np.abs(xn.astype(np.float64) - xo).max() <= TOL_F32
        np.testing.assert_allclose(nun, nuo, rtol=1e-5)
        xh, _ = _handle(sf, V, w, r, K, init, bf16=bf16)
        assert np.abs(xn.astype(np.float64) - xh.astype(np.float64)).max() <= TOL_F32


def test_noalloc_takes_no_device_memory(sf):
    """Free device memory is unchanged across calls (inputs and outputs made beforehand; the
    first call of the process may load the module, so it runs before the measurement)."""
    B, _, wB = synth.multichannel(6, 48, 80, C=3, seed=3004)
    feats = torch.from_numpy(B).cuda()
    x = torch.empty(B.shape[1:], device="cuda")
    norms = np.empty(4)
    _call(sf, feats, x, wB, (2, 7, 7), 4, "uniform", norms)
    first = x.clone()
    torch.cuda.synchronize()
    before = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        _call(sf, feats, x, wB, (2, 7, 7), 4, "uniform", norms)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == before
    assert (x - first).abs().max().item() <= TOL_F32


def test_noalloc_rejects_oversized_requests(sf):
    L = sf.lib()
    nb = sf.neighborhood((1, 3, 3))
    dummy = ctypes.c_void_p(16)   # never dereferenced: the size check fails first
    rc = L.sfseg_power_iterate_noalloc(ctypes.byref(sf.Params(1.0, 0.1)), 1, 64, 480, 854, dummy, 0, None, 0.0,
                                       ctypes.byref(nb), 5, dummy, 1, None, None)
    assert rc == 2 and b"too large" in L.sfseg_last_error()
    rc = L.sfseg_power_iterate_noalloc(ctypes.byref(sf.Params(1.0, 0.1)), 1, 4, 16, 16, dummy, 0, None, 0.0,
                                       ctypes.byref(nb), 5000, dummy, 1, None, None)
    assert rc == 1 and b"iters" in L.sfseg_last_error()
