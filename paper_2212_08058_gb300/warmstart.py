"""Warm start for the power iteration: training the network on eigenvectors the plain method
produces, and the time-to-residual comparison of start vectors.

Everything runs through the C ABI (libsfseg.so): labels come from sfseg_power_iterate with
residual checks (sfseg_rayleigh), the network trains with sfseg_net_backward/sfseg_net_adamw, and
the comparison times whole runs with CUDA events.
"""
from __future__ import annotations

import os
import time

import numpy as np
import torch

from . import sfseg, synth

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "data", "warmstart_c8_coarse.npy")
COARSE_LEVELS_TRAIN = 1      # 16x128x128 training volumes: one 2x coarser level
COARSE_TOL = 1e-4


def iterate_to_residual(h: sfseg.PowerIteration, radius, x: torch.Tensor, tol: float, chunk: int = 20,
                        max_iters: int = 4000, bf16_until: float | None = None, init: str = "user",
                        adaptive: bool = False):
    """Power-iterate from x until the Eq. 3 residual of the FP32 operator is <= tol, checking every
    ``chunk`` iterations.  With ``bf16_until`` set, iterations keep bf16 storage while the residual
    is above that value.  With ``adaptive``, once two checks have shown the geometric rate of the
    residual, the next check is placed where that rate predicts tol (rounded up to a multiple of
    10, between chunk and 8 chunk iterations away), which saves checks on slow tails.
    Returns (x, iterations, residual, residual trace)."""
    import math
    its, trace = 0, []
    rho, res = h.rayleigh(x, radius) if init == "user" else (None, float("inf"))
    if init == "user":
        trace.append((0, res))
    first = init
    step = chunk
    while res > tol and its < max_iters:
        step = min(step, max_iters - its)
        nb = step if (bf16_until is not None and res > bf16_until) else 0
        x = h.power_iterate(None, radius=radius, iters=step, iters_bf16=nb, x=x, init=first)
        first = "user"
        its += step
        rho, res = h.rayleigh(x, radius)
        trace.append((its, res))
        step = chunk
        if adaptive and len(trace) >= 2 and res > tol:
            (i0, r0), (i1, r1) = trace[-2], trace[-1]
            if 0.0 < r1 < r0 and i1 > i0 and math.isfinite(r0):
                rate = math.log(r1 / r0) / (i1 - i0)          # log of the per-iteration factor
                need = math.log(tol / r1) / rate
                step = int(min(max(math.ceil(need / 10.0) * 10, chunk), 8 * chunk))
    return x, its, res, trace


def make_label(h: sfseg.PowerIteration, feats: torch.Tensor, w, radius, tol: float = 1e-6,
               max_iters: int = 3000) -> torch.Tensor:
    """Eigenvector of the volume's operator from the plain method (uniform start)."""
    h.set_features(feats, w, 0.0)
    x = torch.empty((h.T, h.H, h.W), device="cuda")
    x, _, _, _ = iterate_to_residual(h, radius, x, tol, chunk=50, max_iters=max_iters, init="uniform")
    return x


def train(net: sfseg.WarmStartNet, n_train: int = 2000, n_holdout: int = 100, epochs: int = 3,
          lr: float = 1e-3, radius=(2, 7, 7), shape=(16, 128, 128), C: int = 8, log=print):
    """Train ``net`` (built with C + 1 input channels) on ``n_train`` generated volumes: its input
    is the C raw channels plus the upsampled coarse solution (sfseg_coarse_start), its target the
    eigenvector the plain method reaches (residual 1e-6).  Returns a dict with the loss trace, the
    mean hold-out cosine loss before and after training, and that of the coarse start alone."""
    T, H, W = shape
    w = synth.fixed_weights(C)
    t0 = time.time()
    vols, coarse, labels = [], [], []
    with sfseg.PowerIteration(C, T, H, W) as h:
        for i in range(n_train + n_holdout):
            V = synth.training_volume_torch(i, T, H, W, C)
            labels.append(make_label(h, V, w, radius))     # sets the features
            xc, _ = h.coarse_start(radius, levels=COARSE_LEVELS_TRAIN, tol=COARSE_TOL)
            coarse.append(xc)
            vols.append(V.to(torch.bfloat16))
    torch.cuda.synchronize()
    t_label = time.time() - t0
    hold = range(n_train, n_train + n_holdout)

    def cosine(a, b):
        return float(1.0 - (a * b).sum() / (a.norm() * b.norm()))

    coarse_only = float(np.mean([cosine(coarse[i], labels[i]) for i in hold]))

    def holdout():
        return float(np.mean([net.backward(vols[i], labels[i], extra=coarse[i]) for i in hold]))

    before = holdout()
    trace = []
    t0 = time.time()
    step = 0
    for ep in range(epochs):
        order = np.random.default_rng(ep).permutation(n_train)
        run = 0.0
        for i in order:
            run += net.backward(vols[i], labels[i], extra=coarse[i])
            net.adamw(lr=lr * (0.3 if ep == epochs - 1 else 1.0), weight_decay=1e-4)
            step += 1
        trace.append(run / n_train)
        log(f"epoch {ep}: mean training loss {trace[-1]:.5f}")
    torch.cuda.synchronize()
    t_train = time.time() - t0
    after = holdout()
    return {"holdout_before": before, "holdout_after": after, "holdout_coarse_only": coarse_only, "trace": trace,
            "label_s": t_label, "train_s": t_train, "steps": step}


def save(net: sfseg.WarmStartNet, path: str = DEFAULT_WEIGHTS):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.save(path, net.get_params())


def load(net: sfseg.WarmStartNet, path: str = DEFAULT_WEIGHTS) -> bool:
    if not os.path.exists(path):
        return False
    net.set_params(np.load(path))
    return True


def compare_starts(feats: torch.Tensor, w, radius=(2, 7, 7), tol: float = 1e-4, net=None, chunk: int = 20,
                   max_iters: int = 4000, bf16_until: float = 2e-3, levels: int = 2, coarse_tol: float = COARSE_TOL,
                   kinds=("uniform", "smap", "coarse", "net"), adaptive: bool = True, repeats: int = 1):
    """Wall time (CUDA events around the whole run: coarse solves, the network and every residual
    check included) to reach residual <= tol on the volume from
      uniform_f32       the uniform start, float32 storage (the plain method),
      smap_f32          the S_m start (Alg. 1 line 3), float32 storage,
      coarse_f32        the coarse-to-fine start (sfseg_coarse_start), float32 storage,
      warmstart_bf16    the network's refinement of the coarse start, bf16 storage until the
                        residual reaches bf16_until, then float32 (when a network is given).
    With repeats > 1 the starts are timed in turn that many times; each entry then also gives the
    sorted times of its repeats ("ms_runs") and "ms" is their median."""
    C, T, H, W = feats.shape
    out = {}
    with sfseg.PowerIteration(C, T, H, W) as h:
        h.set_features(feats, w, 0.0)
        x = torch.empty((T, H, W), device="cuda")
        h.power_iterate(None, radius=radius, iters=2, x=x)        # warm-up of every kernel
        h.rayleigh(x, radius)
        h.coarse_start(radius, levels=levels, tol=1.0, max_iters=2)
        runs = [("uniform_f32", "uniform", None), ("smap_f32", "smap", None), ("coarse_f32", "coarse", None)]
        if net is not None:
            runs.append(("warmstart_bf16", "net", bf16_until))
        runs = [r for r in runs if r[1] in kinds]
        for rep in range(repeats):
            for name, kind, b16 in runs:
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                coarse_its = None
                init = "user"
                if kind in ("coarse", "net"):
                    x, coarse_its = h.coarse_start(radius, levels=levels, tol=coarse_tol)
                    if kind == "net":
                        x = h.warmstart(net, feats, x)
                else:
                    init = kind
                x, its, res, trace = iterate_to_residual(h, radius, x, tol, chunk, max_iters, b16, init, adaptive)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                if rep == 0:
                    out[name] = {"ms": ms, "iterations": its, "residual": res, "coarse_iterations": coarse_its,
                                 "trace": [(int(a), float(b)) for a, b in trace[:: max(1, len(trace) // 12)]],
                                 "ms_runs": [ms]}
                else:
                    out[name]["ms_runs"].append(ms)
        for v in out.values():
            v["ms_runs"].sort()
            v["ms"] = float(np.median(v["ms_runs"]))
    return out


def time_inference(T: int, H: int, W: int, C: int = 8, reps: int = 5, weights: str | None = DEFAULT_WEIGHTS):
    """CUDA-event time of the warm-start network on a C x T x H x W bf16 volume (multichannel
    recipe drawn on the device); returns a dict with ms per forward and TFLOP/s (2 x 27 x
    (16*32 + 32*32 + 32*32 + 32*16) flops per voxel as computed, i.e. with the padded channels)."""
    V, _ = synth.multichannel_torch(T, H, W, C, seed=5600, device="cuda", dtype=torch.bfloat16)
    net = sfseg.WarmStartNet(C + 1)
    if weights:
        load(net, weights)
    extra = torch.rand((T, H, W), device="cuda")
    x0 = net.forward(V, extra)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        x0 = net.forward(V, extra)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    flops = 2.0 * 27 * (16 * 32 + 32 * 32 + 32 * 32 + 32 * 16) * T * H * W
    net.close()
    return {"shape": [C, T, H, W], "ms": ms, "tflops_padded": flops / (ms * 1e-3) / 1e12,
            "x0_positive": bool((x0 > 0).all().item())}


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="time the warm-start network's forward pass")
    ap.add_argument("--shape", type=int, nargs=3, default=[32, 256, 512], metavar=("T", "H", "W"))
    ap.add_argument("--reps", type=int, default=5)
    args = ap.parse_args()
    from . import build as _build
    _build.build()
    print(json.dumps(time_inference(*args.shape, reps=args.reps)))
