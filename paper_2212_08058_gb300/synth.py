"""Seeded synthetic feature volumes shaped like the paper's video workloads.

This module only PRODUCES INPUTS: soft-mask volumes in [0, 1] of one or several channels, the
noiseless masks they come from, and channel weights.  It contains none of the method's
arithmetic, so both the CUDA path and the CPU oracle may be fed from it.

The paper's workloads are DAVIS-2016 videos (480 x 854 frames, about 50 to 70 frames each) whose
feature channels are soft segmentation masks of other methods (Sec. 5.1).  Those videos are not
available, so the volumes below stand in for them: Gaussian blobs moving on straight lines, with
the noise models of Sec. 5.1.3 (uniform noise added to the soft masks), per-channel Gaussian
noise, small spatial shifts and dropped frames.  Every draw comes from ``numpy`` PCG64 with an
explicit seed; large volumes can be produced frame by frame, or on a torch device.
"""
from __future__ import annotations

import numpy as np


def _blob(T, H, W, amp, sigma, hc, wc):
    """amp * exp(-((h - hc(t))^2 + (w - wc(t))^2) / (2 sigma^2)) as float64 [T, H, W]."""
    h = np.arange(H, dtype=np.float64)[None, :, None]
    w = np.arange(W, dtype=np.float64)[None, None, :]
    hc = np.asarray(hc, dtype=np.float64).reshape(T, 1, 1)
    wc = np.asarray(wc, dtype=np.float64).reshape(T, 1, 1)
    return amp * np.exp(-((h - hc) ** 2 + (w - wc) ** 2) / (2.0 * sigma * sigma))


def drifting_blob_mask(T: int, H: int, W: int, sigma_b: float | None = None,
                       drift: float | None = None) -> np.ndarray:
    """Noiseless soft mask of one blob (amplitude 1) drifting right along the middle row.

    Defaults reproduce the 8 x 64 x 64 scene (sigma 8 px, 2 px/frame) and scale it with the
    frame size: sigma = 8 H/64, drift = 2 (H/64)(8/T) px per frame, start at W/4."""
    sigma_b = 8.0 * H / 64.0 if sigma_b is None else sigma_b
    drift = 2.0 * (H / 64.0) * (8.0 / T) if drift is None else drift
    t = np.arange(T, dtype=np.float64)
    return _blob(T, H, W, 1.0, sigma_b, np.full(T, (H - 1) / 2.0), W / 4.0 + drift * t)


def drifting_blob(T: int = 8, H: int = 64, W: int = 64, noise: float = 0.1, seed: int = 1000,
                  sigma_b: float | None = None, drift: float | None = None) -> np.ndarray:
    """One-channel volume [1, T, H, W] float32: the drifting blob plus U(0, noise), clipped."""
    rng = np.random.default_rng(seed)
    m = drifting_blob_mask(T, H, W, sigma_b, drift)
    v = np.clip(m + rng.uniform(0.0, noise, size=m.shape), 0.0, 1.0)
    return v.astype(np.float32)[None]


def crossing_blobs_mask(T: int, H: int, W: int, sigma_b: float | None = None) -> np.ndarray:
    """Three blobs of amplitude 0.9 / 0.6 / 0.4 on straight lines that all cross the frame
    centre at t = (T-1)/2: top-left -> bottom-right corner, left -> right edge along the middle
    row, bottom-left -> top-right corner.  Painter's order (0.4 at the back, 0.9 in front):
    a nearer blob replaces what is behind it where its value exceeds half its amplitude, and
    elsewhere the brighter of the two is kept (mutual occlusion)."""
    sigma_b = H / 8.0 if sigma_b is None else sigma_b
    s = np.arange(T, dtype=np.float64) / max(T - 1, 1)
    tracks = [  # (amplitude, h(s), w(s)), back to front
        (0.4, (H - 1) * (1.0 - s), (W - 1) * s),
        (0.6, np.full(T, (H - 1) / 2.0), (W - 1) * s),
        (0.9, (H - 1) * s, (W - 1) * s),
    ]
    canvas = None
    for amp, hc, wc in tracks:
        m = np.empty((T, H, W))
        for t in range(T):  # frame by frame keeps the peak memory at a few frames
            m[t] = _blob(1, H, W, amp, sigma_b, hc[t:t + 1], wc[t:t + 1])[0]
        if canvas is None:
            canvas = m
        else:
            canvas = np.where(m > 0.5 * amp, m, np.maximum(canvas, m))
    return canvas


def crossing_blobs(T: int = 64, H: int = 480, W: int = 854, noise: float = 0.15,
                   seed: int = 2000) -> np.ndarray:
    """One-channel volume [1, T, H, W] float32: ``crossing_blobs_mask`` + U(0, noise), clipped."""
    rng = np.random.default_rng(seed)
    out = np.empty((1, T, H, W), dtype=np.float32)
    m = crossing_blobs_mask(T, H, W)
    for t in range(T):
        out[0, t] = np.clip(m[t] + rng.uniform(0.0, noise, size=(H, W)), 0.0, 1.0)
    return out


def _shift2d(a: np.ndarray, dy: int, dx: int) -> np.ndarray:
    """Shift the last two axes by (dy, dx) pixels, filling with zeros (no wrap-around)."""
    out = np.zeros_like(a)
    H, W = a.shape[-2:]
    ys, yd = (slice(0, H - dy), slice(dy, H)) if dy >= 0 else (slice(-dy, H), slice(0, H + dy))
    xs, xd = (slice(0, W - dx), slice(dx, W)) if dx >= 0 else (slice(-dx, W), slice(0, W + dx))
    out[..., yd, xd] = a[..., ys, xs]
    return out


def multichannel(T: int, H: int, W: int, C: int = 8, seed: int = 3000, mask: np.ndarray | None = None,
                 sigma_lo: float = 0.05, sigma_hi: float = 0.3, max_shift: int = 4,
                 drop_frac: float = 0.1):
    """C noisy soft-mask channels of one scene (the SFSeg++ setting of Sec. 5.1.2: every channel
    is another method's estimate of the same mask).

    Channel c is the noiseless mask shifted by an integer (dy, dx) in [-max_shift, max_shift]^2,
    plus N(0, sigma_c^2) with sigma_c = linspace(sigma_lo, sigma_hi, C), clipped to [0, 1], and
    round(drop_frac * T) whole frames set to zero (drawn independently per channel).
    Returns (V [C, T, H, W] float32, mask [T, H, W] float64, weights [C] float32 ~ Dirichlet(1))."""
    rng = np.random.default_rng(seed)
    m = drifting_blob_mask(T, H, W) if mask is None else np.asarray(mask, dtype=np.float64)
    sig = np.linspace(sigma_lo, sigma_hi, C)
    V = np.empty((C, T, H, W), dtype=np.float32)
    n_drop = int(round(drop_frac * T))
    for c in range(C):
        dy, dx = rng.integers(-max_shift, max_shift + 1, size=2)
        sh = _shift2d(m, int(dy), int(dx))
        for t in range(T):
            V[c, t] = np.clip(sh[t] + rng.normal(0.0, sig[c], size=(H, W)), 0.0, 1.0)
        if n_drop:
            V[c, rng.choice(T, size=n_drop, replace=False)] = 0.0
    g = rng.gamma(1.0, 1.0, size=C)
    w = (g / g.sum()).astype(np.float32)
    return V, m, w


def random_scene_mask(T: int, H: int, W: int, rng: np.random.Generator) -> np.ndarray:
    """A noiseless mask of 1 to 3 blobs with random amplitude (0.4..1), width (H/12..H/4),
    start point and velocity (up to H/16 px per frame), combined with ``np.maximum``.
    Used for the training volumes of the warm-start network."""
    k = int(rng.integers(1, 4))
    m = np.zeros((T, H, W))
    t = np.arange(T, dtype=np.float64)
    for _ in range(k):
        amp = rng.uniform(0.4, 1.0)
        sg = rng.uniform(H / 12.0, H / 4.0)
        h0, w0 = rng.uniform(0, H), rng.uniform(0, W)
        vh, vw = rng.uniform(-H / 16.0, H / 16.0, size=2)
        m = np.maximum(m, _blob(T, H, W, amp, sg, h0 + vh * t, w0 + vw * t))
    return m


def training_volume(index: int, T: int = 16, H: int = 128, W: int = 128, C: int = 8,
                    base_seed: int = 5000):
    """Training input number ``index`` for the warm-start network: ``multichannel`` channels of a
    ``random_scene_mask`` scene, seed base_seed + index.  Returns (V, mask, weights)."""
    rng = np.random.default_rng(base_seed + index)
    m = random_scene_mask(T, H, W, rng)
    return multichannel(T, H, W, C, seed=base_seed + 100000 + index, mask=m)


def uniform_start(N: int) -> np.ndarray:
    return np.full(N, 1.0 / np.sqrt(N))


def to_bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even) and return them as float32,
    i.e. exactly the values a bf16 tensor made from ``a`` holds."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    r = ((u + rounding) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).reshape(a.shape)


# ------------------------------------------------------------------- device-side generator
def multichannel_torch(T: int, H: int, W: int, C: int, seed: int, device, dtype=None):
    """``multichannel`` recipe drawn with torch on ``device`` (for volumes too large to build on
    the host quickly, e.g. 8 x 120 x 1080 x 1920).  Same recipe, different random stream.
    Returns (V [C, T, H, W] in ``dtype``, weights [C] float32 on the device)."""
    import torch
    dtype = torch.bfloat16 if dtype is None else dtype
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    sigma_b = 8.0 * H / 64.0
    drift = 2.0 * (H / 64.0) * (8.0 / T)
    hh = torch.arange(H, device=device, dtype=torch.float32)[:, None]
    ww = torch.arange(W, device=device, dtype=torch.float32)[None, :]
    V = torch.empty((C, T, H, W), device=device, dtype=dtype)
    sig = torch.linspace(0.05, 0.3, C).tolist()
    shifts = torch.randint(-4, 5, (C, 2), generator=g, device=device).tolist()
    n_drop = int(round(0.1 * T))
    for c in range(C):
        dy, dx = shifts[c]
        for t in range(T):
            wc = W / 4.0 + drift * t + dx
            hc = (H - 1) / 2.0 + dy
            m = torch.exp(-((hh - hc) ** 2 + (ww - wc) ** 2) / (2 * sigma_b * sigma_b))
            n = torch.randn((H, W), generator=g, device=device) * sig[c]
            V[c, t] = (m + n).clamp_(0.0, 1.0).to(dtype)
        if n_drop:
            idx = torch.randperm(T, generator=g, device=device)[:n_drop]
            V[c, idx] = 0
    gm = -torch.log(torch.rand(C, generator=g, device=device))   # Gamma(1) = Exp(1)
    w = (gm / gm.sum()).float()
    return V, w


def fixed_weights(C: int = 8, seed: int = 5999) -> np.ndarray:
    """One Dirichlet(1) draw of channel weights, shared by every warm-start training volume and the
    large inference volume (a deployed SFSeg++ has one learned weight vector)."""
    g = np.random.default_rng(seed).gamma(1.0, 1.0, size=C)
    return (g / g.sum()).astype(np.float32)


def training_volume_torch(index: int, T: int = 16, H: int = 128, W: int = 128, C: int = 8,
                          base_seed: int = 5000, device="cuda", scale_h: int = 1080):
    """Training input ``index`` for the warm-start network, drawn on ``device``: 1 to 3 Gaussian
    blobs whose width, speed and noise follow the statistics of a ``scale_h``-row video seen
    through a H x W window (sigma between scale_h/16 and scale_h/6 pixels, so that a crop often
    shows a blob edge rather than a whole blob), rendered as C noisy channels like
    ``multichannel`` (shift in [-4, 4]^2, N(0, sigma_c^2) noise with sigma_c in [0.05, 0.3],
    10 % dropped frames).  Returns V [C, T, H, W] float32 on the device."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(base_seed + index)

    def u(lo, hi):
        return lo + (hi - lo) * float(torch.rand(1, generator=g, device=device).item())

    hh = torch.arange(H, device=device, dtype=torch.float32)[:, None]
    ww = torch.arange(W, device=device, dtype=torch.float32)[None, :]
    k = 1 + int(torch.randint(0, 3, (1,), generator=g, device=device).item())
    blobs = []
    for _ in range(k):
        sg = u(scale_h / 16.0, scale_h / 6.0)
        blobs.append((u(0.4, 1.0), sg, u(-sg, H + sg), u(-sg, W + sg), u(-H / 32, H / 32), u(-W / 32, W / 32)))
    m = torch.zeros((T, H, W), device=device)
    for t in range(T):
        for amp, sg, h0, w0, vh, vw in blobs:
            b = amp * torch.exp(-((hh - h0 - vh * t) ** 2 + (ww - w0 - vw * t) ** 2) / (2 * sg * sg))
            m[t] = torch.maximum(m[t], b)
    V = torch.empty((C, T, H, W), device=device)
    sig = torch.linspace(0.05, 0.3, C).tolist()
    n_drop = int(round(0.1 * T))
    for c in range(C):
        dy, dx = (int(v) for v in torch.randint(-4, 5, (2,), generator=g, device=device).tolist())
        sh = torch.roll(m, shifts=(dy, dx), dims=(1, 2))
        V[c] = (sh + torch.randn((T, H, W), generator=g, device=device) * sig[c]).clamp_(0.0, 1.0)
        if n_drop:
            V[c, torch.randperm(T, generator=g, device=device)[:n_drop]] = 0.0
    return V
