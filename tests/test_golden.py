"""The oracle-written fixtures of tests/golden/ (tests/golden/make_golden.py, which calls only
the FP64 oracle and the seeded input generator): the oracle still reproduces them, so that a
change of its arithmetic fails here; the taps also match their closed form; and the CUDA path
matches them within the float32 iterate tolerance."""
import os

import numpy as np
import pytest

import oracle
from tests.golden import make_golden as mg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return [[float(v) for v in line.split()] for line in fh if line.strip() and not line.startswith("#")]


@pytest.fixture(scope="module")
def run():
    oracle.build()
    return mg.config1()


def test_oracle_reproduces_golden_config1(run):
    nu, rho, res, idx, xs = run
    g = np.array(_rows("config1_norms.txt"))
    np.testing.assert_array_equal(g[:, 0], np.arange(1, mg.ITERS + 1))
    np.testing.assert_allclose(nu, g[:, 1], rtol=1e-12)
    gx = np.array(_rows("config1_x_samples.txt"))
    np.testing.assert_array_equal(gx[:, 0].astype(int), idx)
    np.testing.assert_allclose(xs, gx[:, 1], rtol=1e-11, atol=1e-15)
    (grho, gres), = _rows("config1_rayleigh.txt")
    assert abs(rho - grho) <= 1e-12 * grho
    assert abs(res - gres) <= 1e-9 * gres


def test_golden_taps_closed_form():
    for row in _rows("taps.txt"):
        r, s, g = int(row[0]), row[1], np.array(row[2:])
        d = np.arange(-r, r + 1)
        np.testing.assert_allclose(g, np.exp(-d * d / (2 * s * s)), rtol=1e-15)
        np.testing.assert_allclose(oracle.taps(r, s), g, rtol=1e-15)


@pytest.mark.gpu
def test_cuda_path_matches_golden_config1():
    import torch
    from paper_2212_08058_gb300 import build, sfseg, synth
    build.build()
    V = synth.drifting_blob(mg.T, mg.H, mg.W, seed=mg.SEED)
    with sfseg.PowerIteration(1, mg.T, mg.H, mg.W, alpha=mg.ALPHA, p=mg.P) as h:
        x, nu = h.power_iterate(torch.from_numpy(V).cuda(), radius=mg.RADIUS, iters=mg.ITERS, return_norms=True)
        rho, res = h.rayleigh(x, mg.RADIUS)
        x = x.cpu().numpy().ravel().astype(np.float64)
    g = np.array(_rows("config1_norms.txt"))
    np.testing.assert_allclose(nu, g[:, 1], rtol=1e-5)
    gx = np.array(_rows("config1_x_samples.txt"))
    assert np.abs(x[gx[:, 0].astype(int)] - gx[:, 1]).max() <= 1e-5
    (grho, gres), = _rows("config1_rayleigh.txt")
    assert abs(rho - grho) <= 1e-5 * grho
    assert abs(res - gres) <= 1e-3 * gres
