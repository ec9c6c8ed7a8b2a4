"""Benchmark of the SFSeg power iteration on one GB300 (or N independent replicas).

Workload (one "step"): plain SFSeg at the 480p shape -- C = 1 float32 feature volume of
64 x 480 x 854 (three crossing Gaussian blobs + U(0, 0.15) noise), radius (2, 7, 7), 50 power
iterations from the uniform start, then the Eq. 3 Rayleigh quotient / residual check; all inputs
resident in HBM.  Metric: voxel-iterations per second (N voxels x 50 iterations per step).

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "voxel-iterations/s & HBM frac; time-to-residual 1e-4, warm-start vs plain, 1 GB300"
UNIT = "voxel-iterations/s"
T, H, W = 64, 480, 854
RADIUS = (2, 7, 7)
ITERS = 50
SEED = 2000
WORKLOAD = "plain SFSeg 480p: C=1 fp32 64x480x854, three crossing blobs, radius (2,7,7), 50 iterations"
PROFILE_FILE = os.path.join(ROOT, "profiles", "iter_fast_r277_f32_480p.txt")
KERNEL_SOURCES = ["kernels_fast.cu", "common.cuh"]
FMA_PER_VOXEL = 3 * ((2 * RADIUS[0] + 1) + (2 * RADIUS[1] + 1) + (2 * RADIUS[2] + 1))   # 105 at (2,7,7)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return pk["hbm_gbs"], "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2212_08058_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary, if the
    kernel sources still hash to the value recorded there (else None)."""
    try:
        text = open(PROFILE_FILE).read()
    except OSError:
        return None
    m = re.search(r"source_sha256_16:\s*([0-9a-f]+)", text)
    t = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m or not t or m.group(1) != kernel_source_hash():
        return None
    return float(t.group(1))


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.lines = []
        self.dev = device_index

    def __enter__(self):
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(self.dev).uuid)
            sel = ["-i", uuid if uuid.startswith("GPU-") else "GPU-" + uuid]
        except Exception:
            sel = []
        try:
            self.proc = subprocess.Popen(["nvidia-smi", *sel, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        rows = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) != 7:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[3:]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, fl in rows for i, v in enumerate(fl) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def rank_seed(rank: int) -> int:
    """Each rank times its own volume (independent problems, no data-path collective)."""
    return SEED + rank


def aggregate(ms_local: float, units_per_step_per_rank: float, steps: int, world: int, device=None):
    """Whole-job throughput: the slowest rank's time (max over ranks) for the units all ranks
    processed.  Returns (units/s, max ms)."""
    ms = ms_local
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return world * units_per_step_per_rank * steps / (ms * 1e-3), ms


def cpu_baseline(seconds_budget: float = 20.0):
    """The FP64 oracle (filter form, OpenMP) on the host cores: a bounded sample of the same
    workload -- as many whole Eq. 7 + Eq. 8 iterations of the full 64 x 480 x 854 volume as fit
    in about 10 to 30 s (at least one)."""
    import numpy as np
    import oracle
    from paper_2212_08058_gb300 import synth
    f = synth.crossing_blobs(T, H, W, seed=SEED)[0].astype(np.float64)
    start = np.ones(f.shape)
    t0 = time.perf_counter()
    oracle.power_filter(f, f, 0.1, 1.0, RADIUS, start, 1)
    one = time.perf_counter() - t0
    k = max(1, min(ITERS, int(seconds_budget / max(one, 1e-3))))
    t0 = time.perf_counter()
    x_oracle, _ = oracle.power_filter(f, f, 0.1, 1.0, RADIUS, start, k)
    dt = time.perf_counter() - t0
    nvox = T * H * W
    out = {"value": nvox * k / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
           "sample": f"{k} of the {ITERS} iterations of the full {T}x{H}x{W} volume, FP64 filter form, "
                     f"{dt:.1f} s"}
    # the same filter form on one core (one iteration of an 8-frame slab), and the explicit
    # sparse-matrix form at the small 8 x 64 x 64 drifting-blob case (4.2 M non-zeros)
    threads = oracle.num_threads()
    oracle.set_num_threads(1)
    try:
        slab = f[:8]
        t0 = time.perf_counter()
        oracle.power_filter(slab, slab, 0.1, 1.0, RADIUS, np.ones(slab.shape), 1)
        dt1 = time.perf_counter() - t0
    finally:
        oracle.set_num_threads(threads)
    out["single_core"] = {"value": slab.size / dt1, "unit": UNIT,
                          "sample": f"one iteration of an 8x{H}x{W} slab, FP64 filter form, {dt1:.1f} s"}
    fb = synth.drifting_blob(8, 64, 64, seed=1000)[0].astype(np.float64)
    t0 = time.perf_counter()
    M = oracle.affinity(fb, fb, 0.1, 1.0, (1, 3, 3))
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.power_csr(M, np.ones(fb.size), 20)
    t_iter = time.perf_counter() - t0
    out["csr_small"] = {"value": fb.size * 20 / t_iter, "unit": UNIT, "nnz": int(M.nnz),
                        "build_s": t_build, "cores": threads,
                        "sample": "explicit Eq. 2 matrix of the 8x64x64 drifting blob, radius (1,3,3), 20 iterations"}
    return out, x_oracle, k


def parity_stats(x_gpu, x_ref, tol: float):
    """Max-abs error of a unit-norm GPU iterate against the oracle's at equal iteration count,
    also relative to max |x| and times sqrt(N), and the angle between the two in degrees."""
    import numpy as np
    a = np.asarray(x_gpu, dtype=np.float64).reshape(-1)
    b = np.asarray(x_ref, dtype=np.float64).reshape(-1)
    d = float(np.abs(a - b).max())
    ua, ub = a / np.linalg.norm(a), b / np.linalg.norm(b)
    ang = float(np.degrees(2.0 * np.arcsin(min(1.0, np.linalg.norm(ua - ub) / 2.0))))
    return {"max_abs": d, "max_abs_over_max_x": d / float(np.abs(b).max()), "max_abs_times_sqrt_n": d * np.sqrt(a.size),
            "angle_deg": ang, "tolerance_max_abs": tol, "within_tolerance": d <= tol}


def run_reference(args, rank, world):
    """`--impl reference`: the FP64 CPU oracle as it stands, on the host cores.  Each step is one
    Eq. 7 + Eq. 8 iteration of a 4-frame slab (4 x 480 x 854) of the same volume."""
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_2212_08058_gb300 import synth
    f = synth.crossing_blobs(T, H, W, seed=SEED)[0][:4].astype(np.float64)
    x = np.ones(f.shape)
    for _ in range(args.warmup):
        x, _ = oracle.power_filter(f, f, 0.1, 1.0, RADIUS, x, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        x, _ = oracle.power_filter(f, f, 0.1, 1.0, RADIUS, x, 1)
    dt = time.perf_counter() - t0
    value = f.size * args.steps / dt
    sample = f"one iteration of a 4x{H}x{W} slab of the workload volume per step, FP64 filter form"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def bench_bf16_multichannel(sfseg, synth, steps: int = 10):
    """SFSeg++ with bf16 storage: C = 8 bf16 channels of 64 x 480 x 854 (the multichannel recipe,
    drawn on the device), radius (2,7,7), 50 iterations all in bf16 storage.  Device-resident
    voxel-iterations/s, CUDA events."""
    import torch
    V, w = synth.multichannel_torch(T, H, W, 8, seed=3000, device="cuda", dtype=torch.bfloat16)
    w = w.cpu().numpy()
    h = sfseg.PowerIteration(8, T, H, W)
    x = torch.empty((T, H, W), device="cuda")
    for _ in range(3):
        h.power_iterate(V, w, 0.0, RADIUS, iters=ITERS, iters_bf16=ITERS, x=x)
    torch.cuda.synchronize()
    h.enable_iter_timing(True)
    h.iter_timing()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        h.power_iterate(V, w, 0.0, RADIUS, iters=ITERS, iters_bf16=ITERS, x=x)
    e1.record()
    torch.cuda.synchronize()
    it_ms, it_n = h.iter_timing()
    nvox = T * H * W
    out = {"workload": "SFSeg++ C=8 bf16 64x480x854, radius (2,7,7), 50 iterations in bf16 storage",
           "value": nvox * ITERS * steps / (e0.elapsed_time(e1) * 1e-3), "unit": UNIT,
           "avg_launch_ms": it_ms / max(it_n, 1),
           "hbm_frac_of_measured": 6.0 * nvox / (it_ms * 1e-3 / max(it_n, 1)) / 1e9 / _peaks()[0]}
    h.close()
    return out


# ---- the oracle leg's error statements (run with the cpu_baseline leg, after the GPU parts)

def bf16_parity(sfseg, synth, k: int = 10):
    """The error of the bf16 SFSeg++ result: the same volume and bf16 schedule against the FP64
    oracle on the bf16 channels widened exactly, at a bounded iteration count (the oracle takes
    about half a second per iteration of this volume on the host cores)."""
    import numpy as np
    import torch
    import oracle
    V, w = synth.multichannel_torch(T, H, W, 8, seed=3000, device="cuda", dtype=torch.bfloat16)
    w = w.cpu().numpy()
    with sfseg.PowerIteration(8, T, H, W) as h:
        xg = h.power_iterate(V, w, 0.0, RADIUS, iters=k, iters_bf16=k).cpu().numpy()
    V64 = V.float().cpu().numpy().astype(np.float64)
    del V
    f = oracle.combine(V64, w.astype(np.float64), 0.0)
    del V64
    xo, _ = oracle.power_filter(f, f, 0.1, 1.0, RADIUS, np.ones(f.shape), k)
    return {"iterations": k, "vs": "FP64 oracle on the same bf16 channels, uniform start", **parity_stats(xg, xo, 2e-3)}


def adjoint_parity(sfseg, synth, tol: float = 1e-3):
    """The error of the differentiation result on the learning workload's check case (C = 2,
    8 x 32 x 32, radius (1,3,3), 30 iterations, checkpoint every 5, 1 - soft-IoU): the adjoint's
    dL/dw, dL/db against the FP64 oracle's reverse pass on the explicit Eq. 2 matrix, fed with
    the oracle's own forward iterate and loss gradient."""
    import numpy as np
    import torch
    import oracle
    V, m, _ = synth.multichannel(8, 32, 32, C=2, seed=4002)
    w, b, r, K = np.array([2.0, 1.0]), -1.0, (1, 3, 3), 30
    tgt = (m > 0.5).astype(np.float64)
    with sfseg.PowerIteration(2, 8, 32, 32) as h:
        x = h.power_iterate(torch.from_numpy(V).cuda(), w.astype(np.float32), b, r, iters=K, record_every=5)
        _, g = h.soft_iou_loss(x, torch.from_numpy(tgt.astype(np.float32)).cuda())
        gw, gb = h.backward(g, r)
    f = oracle.combine(V.astype(np.float64), w, b)
    xo, _ = oracle.power_filter(f, f, 0.1, 1.0, r, np.ones(f.shape), K)
    _, gK = oracle.soft_iou_loss(xo, tgt)
    gwo, gbo = oracle.grad_csr(V.astype(np.float64), w, b, 0.1, 1.0, r, np.ones(f.size), K, gK)
    got = np.append(np.asarray(gw, dtype=np.float64), float(gb))
    ref = np.append(gwo, gbo)
    err = float(np.abs(got - ref).max())
    scale = float(np.abs(ref).max())
    return {"case": "C=2 8x32x32, radius (1,3,3), 30 iterations, checkpoint every 5, 1 - soft-IoU",
            "vs": "FP64 oracle reverse pass on the explicit Eq. 2 matrix (its own forward and loss gradient)",
            "max_abs": err, "max_abs_over_max_grad": err / scale, "tolerance_rel": tol,
            "within_tolerance": err <= tol * scale}


def r133_parity(sfseg, synth, k: int = 10):
    """The error of the radius (1,3,3) results (float32 and bf16 storage) on the 480p volume at a
    bounded iteration count, against the FP64 oracle."""
    import numpy as np
    import torch
    import oracle
    Vn = synth.crossing_blobs(T, H, W, seed=SEED)
    V = torch.from_numpy(Vn).cuda()
    with sfseg.PowerIteration(1, T, H, W) as h:
        x32 = h.power_iterate(V, radius=(1, 3, 3), iters=k).cpu().numpy()
        x16 = h.power_iterate(V, radius=(1, 3, 3), iters=k, iters_bf16=k).cpu().numpy()
    f = Vn[0].astype(np.float64)
    xo, _ = oracle.power_filter(f, f, 0.1, 1.0, (1, 3, 3), np.ones(f.shape), k)
    fb = synth.to_bf16_round(Vn[0]).astype(np.float64)
    xb, _ = oracle.power_filter(fb, fb, 0.1, 1.0, (1, 3, 3), np.ones(f.shape), k)
    return {"iterations": k, "vs": "FP64 oracle, same volume, uniform start (bf16: on the bf16-rounded features)",
            "f32": parity_stats(x32, xo, 1e-5), "bf16": parity_stats(x16, xb, 2e-3)}


def separate_maps_parity(sfseg, synth, k: int = 5):
    """The error of the separate-map result (S_m and F_m from two draws) at a bounded iteration
    count against the FP64 oracle with the same two maps."""
    import numpy as np
    import torch
    import oracle
    Vs, Vf = synth.crossing_blobs(T, H, W, seed=SEED), synth.crossing_blobs(T, H, W, seed=SEED + 1)
    with sfseg.PowerIteration(1, T, H, W) as h:
        h.set_features_sf(torch.from_numpy(Vs).cuda(), None, 0.0, torch.from_numpy(Vf).cuda())
        xg = h.power_iterate(None, radius=RADIUS, iters=k).cpu().numpy()
    xo, _ = oracle.power_filter(Vs[0].astype(np.float64), Vf[0].astype(np.float64), 0.1, 1.0, RADIUS,
                                np.ones(Vs.shape[1:]), k)
    return {"iterations": k, "vs": "FP64 oracle with the same S and F maps, uniform start", **parity_stats(xg, xo, 1e-5)}


def soft_binarize_parity(sfseg, synth, k_cont: int = 5, k_tail: int = 2, gain: float = 10.0):
    """The error of Alg. 1's soft-binarisation result on the 480p volume (a bounded run: k_cont
    continuous iterations, then k_tail soft-binarisation steps) against the FP64 oracle's steps
    from its own continuous iterate; and the share of voxels whose hard labels differ."""
    import numpy as np
    import torch
    import oracle
    Vn = synth.crossing_blobs(T, H, W, seed=SEED)
    with sfseg.PowerIteration(1, T, H, W) as h:
        xc = h.power_iterate(torch.from_numpy(Vn).cuda(), radius=RADIUS, iters=k_cont)
        xs, mask = h.soft_binarize(xc, RADIUS, iters=k_tail, gain=gain)
        xs, mask = xs.cpu().numpy().astype(np.float64), mask.cpu().numpy()
    f = Vn[0].astype(np.float64)
    xo, _ = oracle.power_filter(f, f, 0.1, 1.0, RADIUS, np.ones(f.shape), k_cont)
    so, mo = oracle.soft_binarize(f, f, 0.1, 1.0, RADIUS, xo, k_tail, gain)
    err = float(np.abs(xs - so).max())
    return {"continuous_iterations": k_cont, "binarize_steps": k_tail, "gain": gain,
            "vs": "FP64 oracle, same volume and steps", "max_abs": err, "tolerance_max_abs": 1e-5,
            "within_tolerance": err <= 1e-5, "hard_label_mismatch_fraction": float((mask != mo).mean())}


def online_parity(sfseg, synth, q: int = 13, iters: int = 10, frames: int = 3):
    """The error of the online window after the first `frames` pushes of the 480p stream (window
    q, iters per frame) against the FP64 oracle's Sec. 4.5 partial iterations."""
    import numpy as np
    import torch
    import oracle
    Vn = synth.crossing_blobs(T, H, W, seed=SEED)
    V = torch.from_numpy(Vn).cuda()
    with sfseg.OnlineStream(1, q, H, W) as st:
        for k in range(frames):
            st.push(V[:, k].contiguous(), radius=RADIUS, iters=iters)
        win = st.window().cpu().numpy()
    ref = oracle.online(Vn[:, :frames], None, 0.0, 0.1, 1.0, RADIUS, q, iters)[frames - 1]
    err = float(np.abs(win - ref).max())
    return {"frames": frames, "window": q, "iterations_per_frame": iters,
            "vs": "FP64 oracle partial iterations (Sec. 4.5), same stream", "max_abs": err,
            "tolerance_max_abs": 1e-5, "within_tolerance": err <= 1e-5}


def small_graphs_parity(sfseg, synth):
    """The error of the small case's result as the bench runs it, replayed from a CUDA graph (the
    first call captures, the next ones replay), against the FP64 oracle: 8 x 64 x 64 drifting
    blob, radius (1,3,3), 20 iterations from the uniform start."""
    import numpy as np
    import torch
    import oracle
    Vn = synth.drifting_blob(8, 64, 64, seed=1000)
    with sfseg.PowerIteration(1, 8, 64, 64) as h:
        h.set_features(torch.from_numpy(Vn).cuda())
        h.enable_graphs(True)
        x = torch.empty((8, 64, 64), device="cuda")
        for _ in range(3):
            h.power_iterate(None, radius=(1, 3, 3), iters=20, x=x)
        xg = x.cpu().numpy()
    f = Vn[0].astype(np.float64)
    xo, _ = oracle.power_filter(f, f, 0.1, 1.0, (1, 3, 3), np.ones(f.shape), 20)
    return {"iterations": 20, "vs": "FP64 oracle, uniform start (graph replay)", **parity_stats(xg, xo, 1e-5)}


def exact_parity(sfseg, synth, K: int = 15):
    """The error of the exact (Eq. 1) operator's power iteration at the study's radius (2,7,7), on
    a volume small enough for the oracle's explicit Eq. 1 matrix (4 x 20 x 40 drifting blob),
    K normalised steps from the uniform start."""
    import numpy as np
    import torch
    import oracle
    T_, H_, W_, r = 4, 20, 40, (2, 7, 7)
    Vn = synth.drifting_blob(T_, H_, W_, seed=7601)
    f = Vn[0].astype(np.float64)
    Me = oracle.affinity(f, f, 0.1, 1.0, r, exact=True)
    xo, _ = oracle.power_csr(Me, np.ones(T_ * H_ * W_), K)
    with sfseg.PowerIteration(1, T_, H_, W_) as h:
        h.set_features(torch.from_numpy(Vn).cuda())
        xg = h.power_iterate_exact(r, iters=K).cpu().numpy()
    return {"case": f"drifting blob {T_}x{H_}x{W_}, radius (2,7,7), {K} steps",
            "vs": "FP64 oracle power iteration on the explicit Eq. 1 matrix",
            **parity_stats(xg, xo.reshape(T_, H_, W_), 1e-5)}


def network_parity(sfseg, synth, tol: float = 3e-2):
    """The error of the warm-start network's output (the trained weights, 8 bf16 channels and the
    extra channel) on a small volume against the FP64 oracle's plain convolution loops on the
    same bf16-rounded inputs and weights (three hidden activations are rounded to bf16 on the
    GPU, hence the tolerance relative to max x0)."""
    import numpy as np
    import torch
    import oracle
    from paper_2212_08058_gb300 import warmstart
    T_, H_, W_ = 3, 37, 140
    gen = torch.Generator(device="cuda").manual_seed(7100)
    feats = torch.rand((8, T_, H_, W_), device="cuda", generator=gen).to(torch.bfloat16)
    extra = torch.rand((T_, H_, W_), device="cuda", generator=gen)
    net = sfseg.WarmStartNet(9)
    trained = warmstart.load(net)
    params = [(synth.to_bf16_round(np.asarray(wt, dtype=np.float32)).astype(np.float64), bb.astype(np.float64))
              for wt, bb in net.unflatten(net.get_params())]
    x0 = net.forward(feats, extra).cpu().numpy().astype(np.float64)
    net.check()
    net.close()
    inp = np.concatenate([feats.float().cpu().numpy().astype(np.float64),
                          extra.to(torch.bfloat16).float().cpu().numpy().astype(np.float64)[None]], axis=0)
    ref, _ = oracle.warmstart_forward(inp, params)
    err = float(np.abs(x0 - ref).max())
    scale = float(np.abs(ref).max())
    return {"case": f"C=8+1 bf16 {T_}x{H_}x{W_}, {'trained' if trained else 'random-init'} weights",
            "vs": "FP64 oracle convolution loops on the same bf16 inputs and weights",
            "max_abs": err, "max_abs_over_max_x0": err / scale, "tolerance_rel": tol,
            "within_tolerance": err <= tol * scale}


def bench_soft_binarize(sfseg, synth, steps: int = 5, tail: int = 10):
    """Alg. 1 end to end on the 64 x 480 x 854 crossing-blobs volume at radius (2,7,7): 50
    continuous iterations, then `tail` soft-binarisation steps (Alg. 1 step 3).  Reports the
    wall time of one soft-binarisation step (CUDA events) and its share of the run."""
    import torch
    V = torch.from_numpy(synth.crossing_blobs(T, H, W, seed=SEED)).cuda()
    h = sfseg.PowerIteration(1, T, H, W)
    h.set_features(V)
    x = h.power_iterate(None, radius=RADIUS, iters=ITERS)
    for _ in range(2):
        h.soft_binarize(x, RADIUS, iters=tail, gain=10.0)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    t_cont = t_tail = 0.0
    for _ in range(steps):
        e[0].record()
        xc = h.power_iterate(None, radius=RADIUS, iters=ITERS, x=x)
        e[1].record()
        xs, mask = h.soft_binarize(xc, RADIUS, iters=tail, gain=10.0)
        e[2].record()
        torch.cuda.synchronize()
        t_cont += e[0].elapsed_time(e[1])
        t_tail += e[1].elapsed_time(e[2])
    fg = float(mask.float().mean())
    h.close()
    return {"workload": f"Alg. 1 on plain SFSeg 480p: {ITERS} continuous + {tail} soft-binarisation steps, gain 10",
            "ms_per_continuous_iteration": t_cont / steps / ITERS, "ms_per_binarize_step": t_tail / steps / tail,
            "foreground_fraction": fg}


def bench_r133_storage(sfseg, synth, steps: int = 10):
    """Radius (1,3,3) (3 x 7 x 7, the neighbourhood of the paper's Sec. 4.2 counts) on the 480p
    crossing-blobs volume, 50 iterations, float32 storage against bf16 storage.  At this radius
    the step needs 51 FMA per 12 bytes (float32), so bytes matter: CUDA-event launch time and the
    fraction of the measured HBM peak for each storage type."""
    import torch
    V = torch.from_numpy(synth.crossing_blobs(T, H, W, seed=SEED)).cuda()
    h = sfseg.PowerIteration(1, T, H, W)
    h.set_features(V)
    x = torch.empty((T, H, W), device="cuda")
    out = {"workload": "plain SFSeg 480p C=1, radius (1,3,3), 50 iterations"}
    for name, nb, bytes_per in (("f32", 0, 12.0), ("bf16", ITERS, 6.0)):
        for _ in range(2):
            h.power_iterate(None, radius=(1, 3, 3), iters=ITERS, iters_bf16=nb, x=x)
        torch.cuda.synchronize()
        h.enable_iter_timing(True)
        h.iter_timing()
        for _ in range(steps):
            h.power_iterate(None, radius=(1, 3, 3), iters=ITERS, iters_bf16=nb, x=x)
        ms, n = h.iter_timing()
        h.enable_iter_timing(False)
        per = ms / max(n, 1)
        out[name] = {"avg_launch_ms": per, "voxel_iterations_per_s": T * H * W / (per * 1e-3),
                     "hbm_frac_of_measured": bytes_per * T * H * W / (per * 1e-3) / 1e9 / _peaks()[0]}
    h.close()
    return out


def bench_small_graphs(sfseg, synth, calls: int = 100):
    """The small drifting-blob case (C = 1, 8 x 64 x 64, radius (1,3,3), 20 iterations), where
    launch latency dominates: CUDA-event time per power_iterate call with direct launches and
    with the call replayed from a captured CUDA graph (sfseg_enable_graphs)."""
    import torch
    V = torch.from_numpy(synth.drifting_blob(8, 64, 64, seed=1000)).cuda()
    out = {"workload": "drifting blob C=1 8x64x64, radius (1,3,3), 20 iterations per call"}
    for name, on in (("direct_ms_per_call", False), ("graph_ms_per_call", True)):
        h = sfseg.PowerIteration(1, 8, 64, 64)
        h.set_features(V)
        h.enable_graphs(on)
        x = torch.empty((8, 64, 64), device="cuda")
        for _ in range(5):
            h.power_iterate(None, radius=(1, 3, 3), iters=20, x=x)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(calls):
            h.power_iterate(None, radius=(1, 3, 3), iters=20, x=x)
        e1.record()
        torch.cuda.synchronize()
        out[name] = e0.elapsed_time(e1) / calls
        h.close()
    return out


def bench_adjoint(sfseg, synth, steps: int = 5):
    """The learning workload (Sec. 3.4): C = 8 float32 channels of 32 x 240 x 427, radius (1,3,3),
    30 unrolled iterations recorded with a checkpoint every 5, loss 1 - soft-IoU against the
    noiseless mask, and the hand-written adjoint back to the 8 channel weights and the bias.
    CUDA-event times of the recorded forward, the loss and the backward, per step."""
    import torch
    Tb, Hb, Wb, K = 32, 240, 427, 30
    V, m, w = synth.multichannel(Tb, Hb, Wb, C=8, seed=4003)
    feats = torch.from_numpy(V).cuda()
    tgt = torch.from_numpy((m > 0.5).astype("float32")).cuda()
    w = (w * 8.0).astype("float32")
    h = sfseg.PowerIteration(8, Tb, Hb, Wb)
    h.enable_graphs(True)          # the backward pass replays as a CUDA graph
    x = torch.empty((Tb, Hb, Wb), device="cuda")

    def run():
        h.power_iterate(feats, w, -2.0, (1, 3, 3), iters=K, x=x, record_every=5)
        e1.record()
        _, g = h.soft_iou_loss(x, tgt)
        h.backward(g, (1, 3, 3))

    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    for _ in range(2):
        run()
    torch.cuda.synchronize()
    t_fwd = t_bwd = 0.0
    for _ in range(steps):
        e0.record()
        run()
        e2.record()
        torch.cuda.synchronize()
        t_fwd += e0.elapsed_time(e1)
        t_bwd += e1.elapsed_time(e2)
    h.close()
    nvox = Tb * Hb * Wb
    # the reverse pass's algorithmic work per step: two filterings of Eq. 7's three signals (the
    # recomputing step with its Q-pass, and the g-pass), 2 x 3 x 17 FMA per voxel at (1,3,3), and
    # 72 bytes per voxel (recomputing step: read V_k, f, write V_{k+1}, Q_x; g-pass: read v_g, f,
    # V_k, write G, Q_g; element-wise pass: read f, v_g, Q_x, V_k, Q_g, G, gz, write gz, v_g)
    fma_step, bytes_step = 2 * 3 * 17, 72.0
    t_b = t_bwd / steps * 1e-3
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    alu_peak = nsm * 128 * 2 * 2070e6 / 1e12
    ach = 2.0 * fma_step * nvox * K / t_b / 1e12
    hbm = bytes_step * nvox * K / t_b / 1e9
    return {"workload": "C=8 fp32 32x240x427, radius (1,3,3), 30 iterations, checkpoint every 5, 1 - soft-IoU",
            "forward_ms": t_fwd / steps, "loss_and_backward_ms": t_bwd / steps,
            "backward_over_forward": t_bwd / max(t_fwd, 1e-9),
            "forward_voxel_iterations_per_s": nvox * K / (t_fwd / steps * 1e-3),
            "roofline": {"bound": "alu", "achieved": ach, "peak": alu_peak, "unit": "TFLOP/s", "frac": ach / alu_peak,
                         "peak_kind": f"derived: {nsm} SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                         "algorithmic": "per reverse step: 2 filterings x 51 FMA + 72 B per voxel "
                                        "(whole loss + backward time, all 30 steps)",
                         "hbm": {"achieved": hbm, "peak": _peaks()[0], "unit": "GB/s", "frac": hbm / _peaks()[0]}}}


def bench_separate_maps(sfseg, synth, steps: int = 5):
    """Separate unary and pairwise maps (Eq. 9 with two channel sets) at the 480p shape: S_m from
    the crossing-blobs volume, F_m from a second draw of it, radius (2,7,7), 50 iterations,
    float32.  Device-resident voxel-iterations/s and the iteration kernel's launch time."""
    import torch
    Vs = torch.from_numpy(synth.crossing_blobs(T, H, W, seed=SEED)).cuda()
    Vf = torch.from_numpy(synth.crossing_blobs(T, H, W, seed=SEED + 1)).cuda()
    h = sfseg.PowerIteration(1, T, H, W)
    h.set_features_sf(Vs, None, 0.0, Vf)
    x = torch.empty((T, H, W), device="cuda")
    for _ in range(2):
        h.power_iterate(None, radius=RADIUS, iters=ITERS, x=x)
    torch.cuda.synchronize()
    h.enable_iter_timing(True)
    h.iter_timing()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        h.power_iterate(None, radius=RADIUS, iters=ITERS, x=x)
    e1.record()
    torch.cuda.synchronize()
    it_ms, it_n = h.iter_timing()
    h.close()
    return {"workload": "separate S_m / F_m maps, C=1 each, fp32 64x480x854, radius (2,7,7), 50 iterations",
            "value": T * H * W * ITERS * steps / (e0.elapsed_time(e1) * 1e-3), "unit": UNIT,
            "avg_launch_ms": it_ms / max(it_n, 1)}


def bench_exact_kernel(sfseg, synth, ref_iters: int = 1500, alphas=(1.0, 0.5, 0.25), study_iters: int = 6000,
                       checkpoints=(0, 10, 20, 50, 100, 200, 500, 1000, 2000, 4000, 6000)):
    """The exact (Eq. 1) kernel against its first-order approximation (Sec. 4.3, the Fig. 4
    study) on the 480p workload (crossing blobs, 64 x 480 x 854, radius (2,7,7), p = 0.1):
    for each alpha, ref_iters steps of sfseg_power_iterate_exact and of the method (Eq. 7) from
    the uniform start, their Eq. 3 residuals for their own operators, and the angle and the
    IoU of the half-maximum masks between the two (equally iterated from the same start: the
    difference of the operators, not the distance to either eigenvector, whose spectral gap is
    small here); at the first alpha also the paper's set-up: a reference from study_iters exact
    steps, then the method's iterations from a non-negative start 70 degrees away from it, with
    angle and IoU at checkpoints, and both residuals; and the time per exact step."""
    import numpy as np
    import torch

    def angle(a, b):
        a = a.double() / a.double().norm()
        b = b.double() / b.double().norm()
        return float(np.degrees(2.0 * torch.asin(torch.clamp((a - b).norm() / 2.0, max=1.0)).item()))

    def iou(a, b):
        ma, mb = a > 0.5 * a.max(), b > 0.5 * b.max()
        return float((ma & mb).sum().item() / max(1, (ma | mb).sum().item()))

    def residual(y, x):
        y, x = y.double(), x.double()
        rho = float((x * y).sum() / (x * x).sum())
        return float((y - rho * x).norm() / (abs(rho) * x.norm()))

    V = torch.from_numpy(synth.crossing_blobs(T, H, W, seed=SEED)).cuda()
    sweep, out = [], {}
    for ai, alpha in enumerate(alphas):
        h = sfseg.PowerIteration(1, T, H, W, alpha=alpha)
        h.set_features(V)
        x = torch.empty((T, H, W), device="cuda")
        h.power_iterate_exact(RADIUS, iters=2, x=x)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        xe = h.power_iterate_exact(RADIUS, iters=ref_iters, x=x).clone()
        e1.record()
        torch.cuda.synchronize()
        xm = h.power_iterate(None, radius=RADIUS, iters=ref_iters).clone()
        sweep.append({"alpha": alpha, "exact_residual": residual(h.apply_exact(xe, RADIUS), xe),
                      "method_residual": residual(h.apply(xm, RADIUS), xm),
                      "angle_deg": angle(xm, xe), "iou_half_max": iou(xm, xe)})
        if ai == 0:
            out["exact_ms_per_step"] = e0.elapsed_time(e1) / ref_iters
            # series length as the library picks it (tail bound of the series below 2^-24)
            xb = 2.0 * alpha * float(V.max().item()) ** 2
            tail, terms = xb * np.exp(xb), 1
            while tail > 2.0 ** -24:
                tail *= xb / (terms + 1)
                terms += 1
            out["exact_series_terms"] = terms
            # the reference for the 70-degree study: study_iters exact steps
            xe = h.power_iterate_exact(RADIUS, iters=study_iters - ref_iters, x=xe.contiguous(), init="user").clone()
            ref_res = residual(h.apply_exact(xe, RADIUS), xe)
            # a non-negative start 70 degrees from xe: xe + t r, r noise away from the objects
            gen = torch.Generator(device="cuda").manual_seed(SEED)
            r = torch.rand((T, H, W), device="cuda", generator=gen) * (1.0 - xe / xe.max()) ** 4
            lo, hi = 0.0, 1.0
            while angle(xe + hi * r, xe) < 70.0:
                hi *= 2.0
            for _ in range(60):
                mid = 0.5 * (lo + hi)
                lo, hi = (mid, hi) if angle(xe + mid * r, xe) < 70.0 else (lo, mid)
            xt = (xe + hi * r).contiguous()
            curve, done = [], 0
            for c in checkpoints:
                if c > done:
                    xt = h.power_iterate(None, radius=RADIUS, iters=c - done, x=xt, init="user")
                    done = c
                curve.append([c, angle(xt, xe), iou(xt, xe)])
            out["method_from_70_degrees"] = {
                "alpha": alpha, "reference_exact_iterations": study_iters, "reference_residual": ref_res,
                "method_residual_at_end": residual(h.apply(xt, RADIUS), xt),
                "columns": ["iterations", "angle_deg", "iou_half_max"], "rows": curve}
        h.close()
    out["alpha_sweep"] = {"iterations": ref_iters, "rows": sweep}
    return {"workload": "crossing blobs C=1 fp32 64x480x854, radius (2,7,7), p 0.1", **out}


def bench_online(sfseg, synth, q: int = 13, iters: int = 10, frames: int = 64):
    """Online form (Sec. 4.5) on the 480p crossing-blobs stream: a 13-frame sub-window (the
    paper's t = 6 either side of a frame), 10 iterations per incoming frame.  Frames per second
    and voxel-iterations/s of the window work (CUDA events around the whole stream)."""
    import torch
    V = torch.from_numpy(synth.crossing_blobs(T, H, W, seed=SEED)).cuda()
    frames_in = [V[:, k].contiguous() for k in range(frames)]
    st = sfseg.OnlineStream(1, q, H, W)
    for k in range(q):                    # warm-up: fill the window once
        st.push(frames_in[k], radius=RADIUS, iters=iters)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(frames):
        st.push(frames_in[k], radius=RADIUS, iters=iters)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st.close()
    return {"workload": f"online 480p stream, window {q} frames, {iters} iterations per frame, radius (2,7,7)",
            "frames_per_s": frames / (ms * 1e-3), "ms_per_frame": ms / frames,
            "window_voxel_iterations_per_s": frames * q * H * W * iters / (ms * 1e-3)}


def bench_time_to_residual(sfseg, synth, warmstart, tol: float = 1e-4, repeats: int = 3):
    """Wall time to the Eq. 3 residual tol on the C = 8 bf16 120 x 1080 x 1920 volume from four
    starts: uniform and S_m with float32 storage (the plain method), the coarse-to-fine start
    (two coarser levels), and the trained network's refinement of it followed by bf16 storage
    until the residual reaches 2e-3, then float32.  Each start is timed `repeats` times in turn:
    median and the sorted runs."""
    import torch
    T5, H5, W5 = 120, 1080, 1920
    V, _ = synth.multichannel_torch(T5, H5, W5, 8, seed=5500, device="cuda", dtype=torch.bfloat16)
    w = synth.fixed_weights(8)
    net = sfseg.WarmStartNet(9)
    trained = warmstart.load(net)
    res = warmstart.compare_starts(V, w, RADIUS, tol=tol, net=net if trained else None, max_iters=3000,
                                   repeats=repeats)
    if trained:
        # the network's forward pass alone on this volume (what its start costs)
        extra = torch.rand((T5, H5, W5), device="cuda")
        net.forward(V, extra)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            net.forward(V, extra)
        e1.record()
        torch.cuda.synchronize()
        res["network_forward_ms"] = e0.elapsed_time(e1) / 3
        del extra
    net.close()
    del V
    torch.cuda.empty_cache()
    res["volume"] = "C=8 bf16 120x1080x1920 (multichannel recipe on the device), radius (2,7,7)"
    res["tol"] = tol
    res["repeats"] = repeats
    res["warmstart_trained"] = trained
    return res


def bench_net_training(sfseg, synth, steps: int = 20):
    """The warm-start network's training step (forward, cosine loss, data and weight gradients,
    AdamW) on one 16 x 128 x 128 training volume (8 channels + the coarse start), and its weight-
    gradient kernel alone (tcgen05, one 32 -> 32 layer) at 32 x 256 x 512 with the forward
    convolution of the same layer beside it; CUDA events.  Algorithmic flops: 2 x 27 x C_in x
    C_out per voxel for each convolution and each weight gradient."""
    import torch
    C, T, H, W = 8, 16, 128, 128
    V = synth.training_volume_torch(7000, T, H, W, C).to(torch.bfloat16)
    extra = torch.rand((T, H, W), device="cuda")
    target = torch.rand((T, H, W), device="cuda")
    net = sfseg.WarmStartNet(C + 1, seed=3)
    for _ in range(3):
        net.backward(V, target, extra=extra)
        net.adamw(lr=1e-4)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        net.backward(V, target, extra=extra)
        net.adamw(lr=1e-4)
    e1.record()
    torch.cuda.synchronize()
    step_ms = e0.elapsed_time(e1) / steps
    nvox = T * H * W
    fwd = 2 * 27 * (9 * 32 + 32 * 32 + 32 * 32 + 32 * 1)
    dgrad = 2 * 27 * (1 * 32 + 32 * 32 + 32 * 32)
    wgr = fwd
    out = {"training_step": {"volume": f"C={C}+1 bf16 {T}x{H}x{W}", "ms": step_ms,
                             "algorithmic_tflops": (fwd + dgrad + wgr) * nvox / (step_ms * 1e-3) / 1e12,
                             "note": "synchronises once per step (loss read-back)"}}
    Tb, Hb, Wb = 32, 256, 512
    gen = torch.Generator(device="cuda").manual_seed(7001)
    x = torch.rand((Tb, Hb, Wb, 32), device="cuda", generator=gen).to(torch.bfloat16)
    dz = torch.randn((Tb, Hb, Wb, 32), device="cuda", generator=gen).to(torch.bfloat16)
    for name, fn in (("weight_gradient", lambda: net.layer_backward(1, x, dz, want_dx=False)),
                     ("forward_conv", lambda: net.layer_forward(1, x)),
                     ("data_gradient_and_weight_gradient", lambda: net.layer_backward(1, x, dz, want_dx=True))):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(10):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 10
        fl = 2 * 27 * 32 * 32 * Tb * Hb * Wb * (2 if name.startswith("data") else 1)
        out[name] = {"volume": f"{Tb}x{Hb}x{Wb}, 32 -> 32 channels", "ms": ms,
                     "algorithmic_tflops": fl / (ms * 1e-3) / 1e12}
    net.check()
    net.close()
    return out


EXTRAS = {
    "bf16_multichannel": lambda sf, sy: bench_bf16_multichannel(sf, sy),
    "soft_binarize": lambda sf, sy: bench_soft_binarize(sf, sy),
    "online": lambda sf, sy: bench_online(sf, sy),
    "separate_maps": lambda sf, sy: bench_separate_maps(sf, sy),
    "adjoint": lambda sf, sy: bench_adjoint(sf, sy, steps=1),
    "small_graphs": lambda sf, sy: bench_small_graphs(sf, sy),
    "r133_storage": lambda sf, sy: bench_r133_storage(sf, sy, steps=2),
    "exact_kernel": lambda sf, sy: bench_exact_kernel(sf, sy),
    "time_to_residual": lambda sf, sy, ws: bench_time_to_residual(sf, sy, ws),
    "net_training": lambda sf, sy: bench_net_training(sf, sy),
}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the bf16 and time-to-residual lines")
    ap.add_argument("--only", choices=sorted(EXTRAS), help="run one extra measurement alone and print its JSON "
                    "(for profiling that part)")
    args = ap.parse_args()
    if args.only:
        from paper_2212_08058_gb300 import build, sfseg, synth, warmstart
        build.build()
        fn = EXTRAS[args.only]
        res = fn(sfseg, synth, warmstart) if args.only == "time_to_residual" else fn(sfseg, synth)
        print(json.dumps({"only": args.only, **res}), flush=True)
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2212_08058_gb300 import sfseg, synth

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    # inputs: each rank its own volume (independent problems; no data-path collective)
    V = synth.crossing_blobs(T, H, W, seed=rank_seed(rank))
    feats = torch.from_numpy(V).cuda()
    feats_host = torch.from_numpy(V).pin_memory()
    nvox = T * H * W
    h = sfseg.PowerIteration(1, T, H, W, alpha=1.0, p=0.1)
    x = torch.empty((T, H, W), device="cuda")
    x_host = torch.empty((T, H, W), pin_memory=True)
    stream = torch.cuda.current_stream()

    def step(features, xout):
        h.power_iterate(features, radius=RADIUS, iters=ITERS, x=xout)
        return h.rayleigh(xout, RADIUS)      # Eq. 3 residual check (synchronises)

    for _ in range(args.warmup):
        step(feats, x)
    torch.cuda.synchronize()
    n_launch0 = sfseg.kernel_launches()
    tma0, gen0, _ = sfseg.iterate_kernel_stats()

    # ---- device-resident timed region
    h.enable_iter_timing(True)
    h.iter_timing()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            rho, res = step(feats, x)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = sfseg.kernel_launches() - n_launch0
    tma1, gen1, kernel_name = sfseg.iterate_kernel_stats()
    if gen1 != gen0 or tma1 - tma0 != args.steps * ITERS:
        raise RuntimeError(f"the timed steps did not all run on the TMA kernel: {tma1 - tma0} TMA steps, "
                           f"{gen1 - gen0} generic-stencil steps for {args.steps * ITERS} iterations")
    clk_summary = clk.summary()
    it_ms, it_n = h.iter_timing()
    h.enable_iter_timing(False)
    value, ms = aggregate(ms, nvox * ITERS, args.steps, world, device="cuda")
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()

    # ---- end to end through the public call with host buffers: every step uploads its features
    # from pinned host memory and downloads its x to pinned host memory inside the timed region.
    # The copies run on a second stream with two buffers of each, so the upload of step k+1 and
    # the download of step k overlap the computation of step k and k+1.
    copy = torch.cuda.Stream()
    fbuf = [feats, torch.empty_like(feats)]
    xbuf = [x, torch.empty_like(x)]
    xhost = [x_host, torch.empty((T, H, W), pin_memory=True)]

    def e2e_run(nsteps):
        up = [torch.cuda.Event() for _ in range(2)]
        done = [torch.cuda.Event() for _ in range(2)]
        down = [torch.cuda.Event() for _ in range(2)]
        with torch.cuda.stream(copy):
            copy.wait_stream(stream)
            fbuf[0].copy_(feats_host, non_blocking=True)
            up[0].record(copy)
        for k in range(nsteps):
            i = k & 1
            if k + 1 < nsteps:
                with torch.cuda.stream(copy):
                    if k >= 1:
                        copy.wait_event(done[1 - i])       # step k-1 no longer reads buffer 1-i
                    fbuf[1 - i].copy_(feats_host, non_blocking=True)
                    up[1 - i].record(copy)
            stream.wait_event(up[i])
            if k >= 2:
                stream.wait_event(down[i])                 # x of step k-2 has left buffer i
            step(fbuf[i], xbuf[i])
            done[i].record(stream)
            with torch.cuda.stream(copy):
                copy.wait_event(done[i])
                xhost[i].copy_(xbuf[i], non_blocking=True)
                down[i].record(copy)
        for i in range(min(2, nsteps)):
            stream.wait_event(down[i])

    e2e_run(args.warmup)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_run(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ems = e0.elapsed_time(e1)
    evalue, ems = aggregate(ems, nvox * ITERS, args.steps, world, device="cuda")
    # the last step's x arrived in host memory intact
    e2e_ok = bool(torch.equal(xhost[(args.steps - 1) & 1], xbuf[(args.steps - 1) & 1].cpu()))

    if rank == 0:
        peak, peak_kind = _peaks()
        per_launch_s = it_ms * 1e-3 / max(it_n, 1)
        algo_bytes = 12.0 * nvox              # read v and f, write v: float32, per iteration launch
        achieved = algo_bytes / per_launch_s / 1e9
        # At radius (2,7,7) the step needs 105 FMA per 12 bytes, above the GPU's balance of
        # FP32 FMA rate to HBM bandwidth, so the FP32 pipe is the roof: 128 FMA per clock per
        # SM (measured: FFMA2 does not raise it), 2 flops per FMA, at the sampled SM clock.
        clk = clk_summary["sm_mhz"] if clk_summary else 2070.0
        nsm = torch.cuda.get_device_properties(local).multi_processor_count
        alu_peak = nsm * 128 * 2 * clk * 1e6 / 1e12
        alu_achieved = 2.0 * FMA_PER_VOXEL * nvox / per_launch_s / 1e12
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic: three crossing Gaussian blobs + U(0,0.15) noise, seeded",
            "config": {"workload": WORKLOAD, "T": T, "H": H, "W": W, "C": 1, "radius": list(RADIUS),
                       "iters": ITERS, "storage": "f32",
                       "l2": "inputs larger than L2 (f + two iterate buffers = 318 MB > 129 MB)"},
            "roofline": {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak, "unit": "TFLOP/s",
                         "frac": alu_achieved / alu_peak, "traffic": profiled_traffic(),
                         "kernel": kernel_name,
                         "peak_kind": f"derived: {nsm} SMs x 128 FP32 lanes x 2 flop x {clk:.0f} MHz",
                         "algorithmic_flops_per_launch": 2.0 * FMA_PER_VOXEL * nvox,
                         "avg_launch_ms": per_launch_s * 1e3,
                         "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                                 "peak_kind": peak_kind, "algorithmic_bytes_per_launch": algo_bytes}},
            "e2e": {"value": evalue, "unit": UNIT, "h2d_bytes_per_step": nvox * 4,
                    "d2h_bytes_per_step": nvox * 4, "ms_per_step": ems / args.steps,
                    "copies": "pinned host buffers, on a second stream, double-buffered (the next "
                              "step's upload and this step's download overlap the computation)",
                    "last_download_checked": e2e_ok},
            "gpu_launches": launches,
            "kernel_ran": {"iteration_kernel": kernel_name, "tma_steps": tma1 - tma0,
                           "generic_stencil_steps": gen1 - gen0},
            "clocks": clk_summary,
            "residual": res, "rho": rho,
            "paper_context": "0.01 s per iteration per 480x854 frame on a GTX Titan X (Maxwell), "
                             "about 4.1e7 voxel-iterations/s (Sec. 5, running time)",
        }
        if world == 1 and not args.no_extras:
            from paper_2212_08058_gb300 import warmstart
            out["bf16_multichannel"] = bench_bf16_multichannel(sfseg, synth)
            out["soft_binarize"] = bench_soft_binarize(sfseg, synth)
            out["online"] = bench_online(sfseg, synth)
            out["separate_maps"] = bench_separate_maps(sfseg, synth)
            out["adjoint"] = bench_adjoint(sfseg, synth)
            out["small_graphs"] = bench_small_graphs(sfseg, synth)
            out["r133_storage"] = bench_r133_storage(sfseg, synth)
            out["exact_kernel"] = bench_exact_kernel(sfseg, synth)
            out["time_to_residual"] = bench_time_to_residual(sfseg, synth, warmstart)
            out["net_training"] = bench_net_training(sfseg, synth)
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"], x_oracle, k = cpu_baseline()
            # the error of the timed result: the GPU iterate after the oracle's iteration count,
            # same volume and uniform start, against the oracle's
            xg = h.power_iterate(feats, radius=RADIUS, iters=k, x=x).cpu().numpy()
            out["parity"] = {"iterations": k, "vs": "FP64 oracle (filter form), same volume, uniform start",
                             **parity_stats(xg, x_oracle, 1e-5)}
            # the error of the other results, same leg
            if "bf16_multichannel" in out:
                out["bf16_multichannel"]["parity"] = bf16_parity(sfseg, synth)
            if "adjoint" in out:
                out["adjoint"]["parity"] = adjoint_parity(sfseg, synth)
            if "net_training" in out:
                out["net_training"]["parity"] = network_parity(sfseg, synth)
            if "r133_storage" in out:
                out["r133_storage"]["parity"] = r133_parity(sfseg, synth)
            if "separate_maps" in out:
                out["separate_maps"]["parity"] = separate_maps_parity(sfseg, synth)
            if "soft_binarize" in out:
                out["soft_binarize"]["parity"] = soft_binarize_parity(sfseg, synth)
            if "online" in out:
                out["online"]["parity"] = online_parity(sfseg, synth)
            if "small_graphs" in out:
                out["small_graphs"]["parity"] = small_graphs_parity(sfseg, synth)
            if "exact_kernel" in out:
                out["exact_kernel"]["parity"] = exact_parity(sfseg, synth)
        print(json.dumps(out), flush=True)
    h.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
