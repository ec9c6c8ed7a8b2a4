"""The T-sharded power iteration's bookkeeping on CPU: slabs of whole frames with halo frames
exchanged between neighbouring parts and the Eq. 8 norm all-reduced, run as gloo ranks with the
FP64 oracle's Eq. 7 operator on each extended slab, must reproduce the oracle's power iteration
on the whole video (same iterate and norms up to FP64 summation order)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2212_08058_gb300 import sharded, synth

P, ALPHA = 0.1, 1.0


class OracleBackend:
    """The operator of one extended slab from the oracle (test side only)."""

    def __init__(self, f_ext, radius):
        self.f = f_ext
        self.radius = radius
        self.shape = f_ext.shape

    def empty(self):
        return torch.empty(self.shape, dtype=torch.float64)

    def acc(self):
        return torch.zeros(1, dtype=torch.float64)

    def apply(self, x, y):
        y.copy_(torch.from_numpy(oracle.filter_apply(self.f, self.f, P, ALPHA, self.radius, x.numpy())))

    def sumsq(self, x, acc):
        acc += (x * x).sum()

    def normalize(self, x, acc):
        x.mul_(1.0 / float(acc[0]) ** 0.5)

    def check(self):
        pass


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _volume(T, H, W):
    return synth.drifting_blob(T, H, W, seed=1000)[0].astype(np.float64)


def _worker(rank, world, port, T, H, W, radius, iters, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    oracle.build()
    f = _volume(T, H, W)
    slab = sharded.Slab(T, world, rank, radius[0])
    be = OracleBackend(f[slab.e0:slab.e1], radius)
    x_own = torch.ones((slab.t1 - slab.t0, H, W), dtype=torch.float64)
    x, norms = sharded.power_iterate_distributed(be, slab, x_own, iters)
    out[rank] = (slab.t0, slab.t1, x.numpy(), norms)
    dist.barrier()
    dist.destroy_process_group()


def _run(world, T, H, W, radius, iters):
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), T, H, W, radius, iters, out), nprocs=world, join=True)
    parts = [out[r] for r in range(world)]
    return parts


def test_slab_bounds():
    for T in (7, 12, 64):
        for parts in (1, 2, 3, 5):
            if T < parts:
                continue
            bounds = [sharded.slab_bounds(T, parts, r) for r in range(parts)]
            assert bounds[0][0] == 0 and bounds[-1][1] == T
            assert all(a[1] == b[0] for a, b in zip(bounds, bounds[1:]))
            sizes = [b - a for a, b in bounds]
            assert max(sizes) - min(sizes) <= 1
    s = sharded.Slab(12, 3, 1, 2)
    assert (s.t0, s.t1, s.e0, s.e1, s.left, s.right) == (4, 8, 2, 10, 2, 2)
    s = sharded.Slab(12, 3, 0, 2)
    assert (s.e0, s.e1, s.left, s.right) == (0, 6, 0, 2)
    with pytest.raises(ValueError):
        sharded.Slab(5, 5, 2, 2)       # one-frame slabs are thinner than rt = 2
    assert sharded.halo_bytes_per_iteration(sharded.Slab(12, 3, 1, 2), 4, 5) == 4 * 4 * 5 * 4


@pytest.mark.parametrize("world,T,radius", [(2, 12, (2, 3, 3)), (3, 11, (1, 2, 2))], ids=["two_parts", "three_uneven"])
def test_parts_reproduce_the_whole_video(world, T, radius):
    H, W, iters = 14, 18, 7
    parts = _run(world, T, H, W, radius, iters)
    f = _volume(T, H, W)
    xo, nuo = oracle.power_filter(f, f, P, ALPHA, radius, np.ones(f.shape), iters)
    x = np.concatenate([p[2] for p in parts], axis=0)
    assert [p[0] for p in parts] == [sharded.slab_bounds(T, world, r)[0] for r in range(world)]
    assert np.abs(x - xo).max() <= 1e-12
    for p in parts:
        np.testing.assert_allclose(p[3], nuo, rtol=1e-12)


def test_halo_exchange_is_needed():
    """Without the halo frames (each part iterating its own slab alone) the result differs from
    the whole video's: the test above can see a broken exchange."""
    T, H, W, radius, iters = 12, 14, 18, (2, 3, 3), 7
    f = _volume(T, H, W)
    xo, _ = oracle.power_filter(f, f, P, ALPHA, radius, np.ones(f.shape), iters)
    alone = []
    for r in range(2):
        t0, t1 = sharded.slab_bounds(T, 2, r)
        xs, _ = oracle.power_filter(f[t0:t1], f[t0:t1], P, ALPHA, radius, np.ones((t1 - t0, H, W)), iters)
        alone.append(xs)
    x = np.concatenate(alone)
    x /= np.linalg.norm(x)
    assert np.abs(x - xo).max() > 1e-6
