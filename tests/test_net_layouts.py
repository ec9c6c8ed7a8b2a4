"""Host-side checks of the index arithmetic of the network's two convolution kernels (no GPU).

conv3d_tc keeps each output frame's accumulators in a ring of R blocks of 32 TMEM columns
(R = 5, 8 or 16 for three, two or one output frames per CTA): input row i feeds the output rows
i - dh (dh = 0, 1, 2) through one MMA run into consecutive blocks (a second run where the ring
wraps), output row j lives in block (-j) mod R, the issuer waits for the read of row i - R
before row i enters the ring, and the epilogue reads row i - 2 after input row i.  The
simulation below replays that protocol for every tile height up to 100 and checks that each
(row, tap) lands exactly once in its row's block inside the ring, that a row enters a block
with its first contribution and only after the block's previous row was read, and that a row
is read only when complete.

conv_last_tc stacks the nine (dh, dw) taps of all FR output frames of a row along N: the MMA of
slot frame s and channel half ks takes four (or one) consecutive 16-row blocks of the taps
packed as [Z Z Z W2 W1 W0 Z Z Z] from block 5 - s on, the first MMA of a row (s = 0, ks = 0) does
not accumulate, and the epilogue sums D_{j+dh}[l + dw, 16 g + 3 dh + dw].  A numpy replay of
that layout, including the last frame group of an odd frame count and a ragged last tile, is
compared with the oracle's 3x3x3 convolution.
"""
import numpy as np

import oracle


def _blk(j, R):
    return (R - j % R) % R


def _ring_protocol(R, nout):
    nin = nout + 2
    contrib = {}
    occupant = [None] * R
    got = {}
    read = set()
    for i in range(nin):
        jhi, jlo = min(i, nout - 1), max(i - 2, 0)
        if R <= i < nout:                       # the issuer's wait on the block's last read
            assert (i - R) in read
        dh0, nrow = i - jhi, jhi - jlo + 1
        b0 = _blk(jhi, R)
        n1 = min(nrow, R - b0)
        n2 = nrow - n1
        assert 1 <= n1 <= 3 and 0 <= n2 <= 2 and dh0 + nrow - 1 <= 2   # within the stacked B
        runs = [(b0, dh0, n1)] + ([(0, dh0 + n1, n2)] if n2 else [])
        for bstart, dhs, n in runs:
            assert bstart >= 0 and bstart + n <= R                     # inside the frame's ring
            for m in range(n):
                b, dh = bstart + m, dhs + m
                j = i - dh
                assert 0 <= j < nout and _blk(j, R) == b
                if occupant[b] != j:
                    assert dh == 0 and (occupant[b] is None or occupant[b] in read)
                    occupant[b] = j
                contrib[(j, dh)] = contrib.get((j, dh), 0) + 1
                got[j] = got.get(j, 0) + 1
        if i >= 2 and i - 2 < nout:             # commit of output row i - 2, then its read
            assert got[i - 2] == 3 and occupant[_blk(i - 2, R)] == i - 2
            read.add(i - 2)
    assert all(contrib.get((j, dh)) == 1 for j in range(nout) for dh in range(3))
    assert read == set(range(nout))


def test_conv_accumulator_ring_protocol():
    for fr in (3, 2, 1):
        ring_cols = (512 // fr) // 32 * 32      # TMEM columns of one output frame
        R = ring_cols // 32
        assert R == {3: 5, 2: 8, 1: 16}[fr]
        for nout in range(1, 101):
            _ring_protocol(R, nout)


def _last_layer_replay(x, taps, bias, FR, HR):
    """z of conv_last_tc's tiles, frame groups and stacked-N MMAs, replayed in float64."""
    T, H, W, _ = x.shape
    NF, LT_W = FR + 2, 126
    packed = np.zeros((2, 9 * 16, 16))          # [ks][block * 16 + n][16 channels of the half]
    for dt in range(3):
        blk = 5 - dt
        for ks in range(2):
            packed[ks, blk * 16:blk * 16 + 9, :] = taps[9 * dt:9 * dt + 9, 16 * ks:16 * ks + 16]
    xp = np.zeros((T + NF + 1, H + 2, W + 130, 32))
    xp[1:T + 1, 1:H + 1, 1:W + 1] = x           # index +1: zero fill outside the volume
    z = np.full((T, H, W), np.nan)
    for t0 in range(0, T, FR):
        nfr = min(FR, T - t0)
        for w0 in range(0, W, LT_W):
            for hs in range(0, H, HR):
                nout = min(H, hs + HR) - hs
                D = []
                for i in range(nout + 2):       # input row h = hs - 1 + i
                    d = None
                    for sf in range(NF):        # slot frame t0 - 1 + sf
                        a = xp[t0 + sf, hs + i, w0:w0 + 128]           # voxels w0 - 1 ... w0 + 126
                        for ks in range(2):
                            b = packed[ks, (5 - sf) * 16:(5 - sf) * 16 + 16 * FR]
                            p = a[:, 16 * ks:16 * ks + 16] @ b.T
                            d = p if (sf | ks) == 0 else d + p
                    D.append(d)
                for g in range(nfr):
                    for j in range(nout):
                        zz = bias + sum(D[j + dh][dw:dw + LT_W, 16 * g + 3 * dh + dw]
                                        for dh in range(3) for dw in range(3))
                        n = min(LT_W, W - w0)
                        z[t0 + g, hs + j, w0:w0 + n] = zz[:n]
    return z


def test_last_layer_stacked_taps_layout():
    rng = np.random.default_rng(7)
    T, H, W = 7, 9, 140                         # 7 = 4 + 3 frames; tiles of 126 + 14 voxels
    x = rng.standard_normal((T, H, W, 32))
    taps = rng.standard_normal((27, 32))        # [9 dt + 3 dh + dw][channel]
    bias = 0.25
    wt = taps.reshape(1, 3, 3, 3, 32)
    ref = oracle.conv3d_fwd(x, wt, np.array([bias]))[..., 0]
    for FR, HR in ((4, 4), (4, 16), (1, 16)):
        z = _last_layer_replay(x, taps, bias, FR, HR)
        assert not np.isnan(z).any()
        assert np.abs(z - ref).max() <= 1e-12 * np.abs(ref).max()
