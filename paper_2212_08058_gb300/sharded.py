"""Power iteration on a video split along t into slabs of whole frames.

Eq. 7 is a stencil of radius rt along t and Eq. 8 a norm over the whole volume.  So a video cut
into slabs needs, at every iteration, the rt frames on the far side of each cut from the
neighbouring slab (a halo exchange) and one sum over all slabs of their squared norms (an
all-reduce of FP64 partial sums, Eq. 8).  Each part keeps its slab extended by the halo frames
that exist on either side.  The operator applied to the extended slab, with zero padding at its
ends, is exact on the part's own frames: their neighbourhoods lie inside it, and where the
extended slab ends at the video's first or last frame its padding is the video's.  The values
on the halo frames are discarded.

Two drivers share this bookkeeping:
  power_iterate_distributed  one part per process (one GPU each), torch.distributed for the
                             halo frames (point-to-point) and the norm (all-reduce);
  power_iterate_lockstep     several parts in one process, in turn, with the exchange as
                             copies; for volumes above one handle's 2^31-voxel limit on one GPU.
Every arithmetic step runs in the backend: LibraryBackend calls the library (sfseg_apply,
sfseg_sumsq, sfseg_normalize) on a handle made for the extended slab.  The all-reduce of one
FP64 scalar per iteration and the halo copies are the only data movement between parts.
"""
from __future__ import annotations

from dataclasses import dataclass


def slab_bounds(T: int, parts: int, rank: int) -> tuple[int, int]:
    """Own frames [t0, t1) of part `rank` of `parts`: sizes differ by at most one frame."""
    if not 0 <= rank < parts or parts < 1 or T < parts:
        raise ValueError(f"cannot split {T} frames into {parts} parts (rank {rank})")
    base, extra = divmod(T, parts)
    t0 = rank * base + min(rank, extra)
    return t0, t0 + base + (1 if rank < extra else 0)


@dataclass(frozen=True)
class Slab:
    """Part `rank` of `parts` of a T-frame video at temporal radius rt: own frames [t0, t1),
    extended frames [e0, e1) = the own frames and up to rt halo frames on either side."""
    T: int
    parts: int
    rank: int
    rt: int

    def __post_init__(self):
        t0, t1 = slab_bounds(self.T, self.parts, self.rank)
        if self.parts > 1 and t1 - t0 < self.rt:
            raise ValueError(f"a slab of {t1 - t0} frames is thinner than the radius {self.rt}: "
                             "its halo would need frames from beyond the neighbouring slab")

    @property
    def t0(self) -> int:
        return slab_bounds(self.T, self.parts, self.rank)[0]

    @property
    def t1(self) -> int:
        return slab_bounds(self.T, self.parts, self.rank)[1]

    @property
    def e0(self) -> int:
        return max(0, self.t0 - self.rt)

    @property
    def e1(self) -> int:
        return min(self.T, self.t1 + self.rt)

    @property
    def own(self) -> slice:
        """The own frames inside the extended slab."""
        return slice(self.t0 - self.e0, self.t1 - self.e0)

    @property
    def left(self) -> int:
        return self.t0 - self.e0

    @property
    def right(self) -> int:
        return self.e1 - self.t1


class LibraryBackend:
    """The library on one GPU for one extended slab: a handle of the extended slab's shape with
    its features set (Eq. 9 is per voxel, so the slab's own combination is the video's)."""

    def __init__(self, features_ext, weights=None, bias: float = 0.0, radius=(2, 7, 7), sigma=None,
                 alpha: float = 1.0, p: float = 0.1):
        import torch

        from . import sfseg
        C, Te, H, W = features_ext.shape
        self.h = sfseg.PowerIteration(C, Te, H, W, alpha=alpha, p=p)
        self.h.set_features(features_ext, weights, bias)
        self.radius, self.sigma = radius, sigma
        self.shape = (Te, H, W)
        self.device = features_ext.device
        self._torch = torch

    def empty(self):
        return self._torch.empty(self.shape, device=self.device, dtype=self._torch.float32)

    def acc(self):
        return self._torch.zeros(1, device=self.device, dtype=self._torch.float64)

    def apply(self, x, y):
        self.h.apply(x, self.radius, self.sigma, out=y)

    def sumsq(self, x, acc):
        self.h.sumsq(x, acc)

    def normalize(self, x, acc):
        self.h.normalize(x, acc)

    def check(self):
        self.h.check()

    def close(self):
        self.h.close()


def _own(x, slab: Slab):
    return x[slab.own]


def power_iterate_distributed(backend, slab: Slab, x_own, iters: int, group=None):
    """This process's part of `iters` steps of Eq. 7 + Eq. 8 on the whole video, from the start
    vector whose own frames are x_own (any positive scale; the first step normalises it over
    the video).  Returns (x_own after the steps, device tensor of the iters norms
    nu_k = ||A x_{k-1}||, k = 1..iters).  Every part must call it with the same iters."""
    import torch
    import torch.distributed as dist

    x, y = backend.empty(), backend.empty()
    x.zero_()
    _own(x, slab).copy_(x_own)
    acc = backend.acc()
    norms = torch.zeros(max(iters, 1), dtype=torch.float64, device=acc.device)
    backend.sumsq(_own(x, slab), acc)
    dist.all_reduce(acc, group=group)
    backend.normalize(_own(x, slab), acc)
    for k in range(iters):
        _exchange(x, slab, group)
        backend.apply(x, y)
        acc.zero_()
        backend.sumsq(_own(y, slab), acc)
        dist.all_reduce(acc, group=group)
        norms[k] = acc[0]
        backend.normalize(_own(y, slab), acc)
        x, y = y, x
    backend.check()
    return _own(x, slab).clone(), norms[:iters].cpu().numpy() ** 0.5


def _exchange(x, slab: Slab, group=None):
    """Fill the halo frames of x (the extended slab) from the neighbouring parts' own frames,
    and send this part's edge frames to them."""
    import torch.distributed as dist
    own = _own(x, slab)
    ops = []
    if slab.rank > 0:
        n_send = min(slab.rt, slab.T - slab.t0)      # the left part's right halo: frames [t0, t0 + n)
        ops.append(dist.P2POp(dist.isend, own[:n_send], slab.rank - 1, group))
        ops.append(dist.P2POp(dist.irecv, x[:slab.left], slab.rank - 1, group))
    if slab.rank < slab.parts - 1:
        n_send = min(slab.rt, slab.t1)               # the right part's left halo: frames [t1 - n, t1)
        ops.append(dist.P2POp(dist.isend, own[own.shape[0] - n_send:], slab.rank + 1, group))
        ops.append(dist.P2POp(dist.irecv, x[slab.own.stop:], slab.rank + 1, group))
    if ops:
        for r in dist.batch_isend_irecv(ops):
            r.wait()


def power_iterate_lockstep(backends, slabs, xs_own, iters: int):
    """The same steps for several parts in one process (in turn, on one device): the halo
    frames are copied between the parts' extended slabs and the norm is the sum of their
    partial sums (each part's sum of squares accumulates into one device scalar).  Returns
    ([x_own of each part], numpy array of the norms)."""
    import torch

    n = len(slabs)
    xs = [b.empty() for b in backends]
    ys = [b.empty() for b in backends]
    total = backends[0].acc()
    norms = torch.zeros(max(iters, 1), dtype=torch.float64, device=total.device)
    for i in range(n):
        xs[i].zero_()
        _own(xs[i], slabs[i]).copy_(xs_own[i])

    def reduce_and_normalize(vs, k):
        total.zero_()
        for i in range(n):
            backends[i].sumsq(_own(vs[i], slabs[i]), total)
        if k >= 0:
            norms[k] = total[0]
        for i in range(n):
            backends[i].normalize(_own(vs[i], slabs[i]), total)

    reduce_and_normalize(xs, -1)
    for k in range(iters):
        for i in range(n):
            s = slabs[i]
            if i > 0:
                xs[i][:s.left].copy_(_own(xs[i - 1], slabs[i - 1])[-s.left:])
            if i < n - 1:
                xs[i][s.own.stop:].copy_(_own(xs[i + 1], slabs[i + 1])[:s.right])
        for i in range(n):
            backends[i].apply(xs[i], ys[i])
        reduce_and_normalize(ys, k)
        xs, ys = ys, xs
    for b in backends:
        b.check()
    return [_own(xs[i], slabs[i]).clone() for i in range(n)], norms[:iters].cpu().numpy() ** 0.5


def halo_bytes_per_iteration(slab: Slab, H: int, W: int) -> int:
    """float32 bytes this part sends per iteration: its edge frames to each neighbour (the
    all-reduce adds one FP64 value)."""
    n = 0
    if slab.rank > 0:
        n += min(slab.rt, slab.T - slab.t0)
    if slab.rank < slab.parts - 1:
        n += min(slab.rt, slab.t1)
    return 4 * H * W * n
