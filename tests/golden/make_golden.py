"""Writes the golden fixtures of this directory from the FP64 oracle alone (and the seeded input
generator, which holds none of the method's arithmetic).  Run from the repository root:

    python -m tests.golden.make_golden

The paper prints no numeric worked example of the eigenvector, so every stored value here is the
oracle's, recorded so that a later change of the oracle's arithmetic shows up as a failed test
(tests/test_golden.py) and so that the CUDA path has fixed targets besides the live oracle.
"""
import os

import numpy as np

import oracle
from paper_2212_08058_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))

# The small configuration: one drifting blob (sigma 8 px, 2 px per frame) plus U(0, 0.1) noise,
# 8 x 64 x 64, radius (1, 3, 3), alpha = 1, p = 0.1, 20 iterations from the uniform start.
T, H, W = 8, 64, 64
RADIUS = (1, 3, 3)
ALPHA, P, ITERS, SEED = 1.0, 0.1, 20, 1000
SAMPLE_STRIDE = 509          # voxel indices 0, 509, 1018, ... (64 samples across the volume)


def config1():
    V = synth.drifting_blob(T, H, W, seed=SEED)
    f = oracle.combine(V.astype(np.float64))
    x, nu = oracle.power_filter(f, f, P, ALPHA, RADIUS, np.ones(f.shape), ITERS)
    rho, res = oracle.rayleigh(lambda v: oracle.filter_apply(f, f, P, ALPHA, RADIUS, v.reshape(f.shape)), x)
    idx = np.arange(0, T * H * W, SAMPLE_STRIDE)[:64]
    return nu, rho, res, idx, x.ravel()[idx]


def write(name, header, rows):
    with open(os.path.join(HERE, name), "w") as fh:
        for line in header:
            fh.write("# " + line + "\n")
        for row in rows:
            fh.write(" ".join(repr(v) if isinstance(v, float) else str(v) for v in row) + "\n")


def main():
    nu, rho, res, idx, xs = config1()
    cfg = (f"drifting blob {T}x{H}x{W}, seed {SEED}, radius {RADIUS}, alpha {ALPHA}, p {P}, "
           f"{ITERS} iterations from the uniform start")
    write("config1_norms.txt",
          ["Eq. 7 steps with the Eq. 8 normalisation (filter form, FP64 oracle): nu_k = ||A x_{k-1}||",
           cfg, "columns: k nu_k"],
          [(k + 1, float(v)) for k, v in enumerate(nu)])
    write("config1_x_samples.txt",
          ["the unit-norm iterate x_20 of the same run at sampled voxels (flat [T][H][W] index)",
           cfg, f"indices 0, {SAMPLE_STRIDE}, 2*{SAMPLE_STRIDE}, ...", "columns: index x"],
          [(int(i), float(v)) for i, v in zip(idx, xs)])
    write("config1_rayleigh.txt",
          ["Eq. 3 for x_20 of the same run: rho = x'Ax / x'x and ||Ax - rho x|| / (rho ||x||)", cfg,
           "columns: rho residual"],
          [(float(rho), float(res))])
    rows = []
    for r in (1, 3, 7):
        s = max(RADIUS) / 2.0 if r != 7 else 3.5
        rows.append([r, s] + [float(v) for v in oracle.taps(r, s)])
    write("taps.txt",
          ["Eq. 1 / Eq. 7 spatial kernel along one axis: exp(-d^2 / (2 sigma^2)) for d = -r .. r,",
           "unnormalised (G_ii = 1), the default sigma = max(radius) / 2 of the (1,3,3) and (2,7,7) boxes",
           "columns: r sigma g_-r .. g_r"],
          rows)


if __name__ == "__main__":
    main()
