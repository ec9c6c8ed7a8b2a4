"""The slab decomposition on the GPU: several parts of one video in one process (lockstep: the
halo frames copied between the parts' extended slabs, the Eq. 8 norm summed over the parts),
each part a library handle for its extended slab, against the FP64 oracle on the whole video
and against sfseg_power_iterate on the whole video."""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_08058_gb300 import sharded, synth

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5


@pytest.fixture(scope="module")
def sf():
    from paper_2212_08058_gb300 import build, sfseg
    build.build()
    oracle.build()
    return sfseg


@pytest.mark.parametrize("parts,radius", [(3, (2, 7, 7)), (2, (1, 3, 3)), (4, (1, 2, 3))])
def test_lockstep_slabs_match_whole_video(sf, parts, radius):
    T, H, W, iters = 22, 70, 150, 12
    V, _, w = synth.multichannel(T, H, W, C=3, seed=3100)
    feats = torch.from_numpy(V).cuda()
    slabs = [sharded.Slab(T, parts, r, radius[0]) for r in range(parts)]
    backends = [sharded.LibraryBackend(feats[:, s.e0:s.e1].contiguous(), w, 0.0, radius) for s in slabs]
    xs0 = [torch.ones((s.t1 - s.t0, H, W), device="cuda") for s in slabs]
    xs, norms = sharded.power_iterate_lockstep(backends, slabs, xs0, iters)
    x = torch.cat(xs).cpu().numpy().astype(np.float64)
    nu = norms
    for b in backends:
        b.close()
    f = oracle.combine(V.astype(np.float64), w)
    xo, nuo = oracle.power_filter(f, f, 0.1, 1.0, radius, np.ones(f.shape), iters)
    assert np.abs(x - xo).max() <= TOL_F32
    np.testing.assert_allclose(nu, nuo, rtol=1e-5)
    with sf.PowerIteration(3, T, H, W) as h:
        xw = h.power_iterate(feats, w, 0.0, radius, iters=iters).cpu().numpy()
    assert np.abs(x - xw).max() <= TOL_F32


def test_distributed_driver_single_rank_nccl(sf):
    """The distributed driver through NCCL with one rank (its all-reduce on the device; the
    halo exchange needs neighbours, which need more GPUs than this run has), against
    sfseg_power_iterate on the same volume."""
    import os
    import socket

    import torch.distributed as dist
    T, H, W, iters, radius = 16, 64, 100, 10, (2, 7, 7)
    V, _, w = synth.multichannel(T, H, W, C=2, seed=3101)
    feats = torch.from_numpy(V).cuda()
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("nccl", rank=0, world_size=1, device_id=torch.device("cuda", 0))
    try:
        slab = sharded.Slab(T, 1, 0, radius[0])
        be = sharded.LibraryBackend(feats, w, 0.0, radius)
        x, norms = sharded.power_iterate_distributed(be, slab, torch.ones((T, H, W), device="cuda"), iters)
        torch.cuda.synchronize()
        be.close()
    finally:
        dist.destroy_process_group()
    with sf.PowerIteration(2, T, H, W) as h:
        xw, nuw = h.power_iterate(feats, w, 0.0, radius, iters=iters, return_norms=True)
    assert float((x - xw).abs().max()) <= TOL_F32
    np.testing.assert_allclose(norms, nuw, rtol=1e-5)
