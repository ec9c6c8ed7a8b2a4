// stencil.cuh -- the streaming space-time stencil kernel template shared by the forward
// iteration, the plain operator application and the adjoint.
//
// A CTA owns a TH x 64 tile of (h, w) and walks along t through a chunk of frames.  For each
// incoming frame it stages the halo tile of the NS signals (Op::load) in shared memory, filters
// along w then h (the separable Gaussian of Sec. 4.2), and keeps the 2D-filtered frame in a ring
// of 2rt+1 frames; the t-filter then gives the NS filtered signals of the frame rt behind, which
// Op::epi combines into the outputs.  Zero padding: voxels outside the volume load as zeros.
#pragma once

#include "common.cuh"
#include "launch.h"

namespace sfseg {

constexpr int kTW = 64;          // tile width (w) of the generic stencil
constexpr int kThreads = 256;

// ------------------------------------------------------------------------ streaming stencil
template <class Op>
__global__ void __launch_bounds__(kThreads)
stream_stencil(Op op, Taps tp, int TH, int tchunk, const double* acc_in, double* acc_out,
               double* acc_out2, int* flags) {
    constexpr int NS = Op::NS;
    extern __shared__ float smem[];
    const int rt = tp.rt, rh = tp.rh, rw = tp.rw;
    const int ZH = TH + 2 * rh, ZW = kTW + 2 * rw, nslot = 2 * rt + 1;
    float* Z = smem;                        // [NS][ZH][ZW]  signals of the incoming frame
    float* Q = Z + NS * ZH * ZW;            // [NS][ZH][kTW] after the w-pass
    float* P = Q + NS * ZH * kTW;           // [nslot][NS][TH][kTW] after the h-pass (ring)
    const Geom g = op.g;
    const int w0 = blockIdx.x * kTW, h0 = blockIdx.y * TH;
    const int t0 = blockIdx.z * tchunk;
    const int t1 = min(t0 + tchunk, g.T);
    Op o = op;
    o.begin(acc_in, flags);   // device-resident scalars (norms, dot products)
    float part0 = 0.f, part1 = 0.f;

    for (int tt = t0 - rt; tt < t1 + rt; ++tt) {
        float* Ps = P + ((tt - t0 + rt) % nslot) * NS * TH * kTW;
        if (tt >= 0 && tt < g.T) {
            for (int i = threadIdx.x; i < ZH * ZW; i += blockDim.x) {
                const int r = i / ZW, c = i - r * ZW;
                const int h = h0 - rh + r, w = w0 - rw + c;
                float z[NS];
                if (h >= 0 && h < g.H && w >= 0 && w < g.W) {
                    o.load(tt, h, w, z);
                } else {
#pragma unroll
                    for (int k = 0; k < NS; ++k) z[k] = 0.f;
                }
#pragma unroll
                for (int k = 0; k < NS; ++k) Z[(k * ZH + r) * ZW + c] = z[k];
            }
            __syncthreads();
            for (int i = threadIdx.x; i < ZH * kTW; i += blockDim.x) {
                const int r = i / kTW, c = i - r * kTW;
#pragma unroll
                for (int k = 0; k < NS; ++k) {
                    const float* zr = Z + (k * ZH + r) * ZW + c;
                    float a = 0.f;
                    for (int d = 0; d <= 2 * rw; ++d) a += tp.gw[d] * zr[d];
                    Q[(k * ZH + r) * kTW + c] = a;
                }
            }
            __syncthreads();
            for (int i = threadIdx.x; i < TH * kTW; i += blockDim.x) {
                const int r = i / kTW, c = i - r * kTW;
#pragma unroll
                for (int k = 0; k < NS; ++k) {
                    const float* qc = Q + (k * ZH + r) * kTW + c;
                    float a = 0.f;
                    for (int d = 0; d <= 2 * rh; ++d) a += tp.gh[d] * qc[d * kTW];
                    Ps[(k * TH + r) * kTW + c] = a;
                }
            }
        } else {
            __syncthreads();   // the slot being cleared was read by the previous t-pass
            for (int i = threadIdx.x; i < NS * TH * kTW; i += blockDim.x) Ps[i] = 0.f;
        }
        __syncthreads();
        const int to = tt - rt;   // output frame; to < t1 always holds
        if (to >= t0) {
            for (int i = threadIdx.x; i < TH * kTW; i += blockDim.x) {
                const int r = i / kTW, c = i - r * kTW;
                const int h = h0 + r, w = w0 + c;
                if (h < g.H && w < g.W) {
                    float cc[NS];
#pragma unroll
                    for (int k = 0; k < NS; ++k) cc[k] = 0.f;
                    for (int d = 0; d <= 2 * rt; ++d) {
                        const float* ps = P + ((to + d - t0) % nslot) * NS * TH * kTW + r * kTW + c;
                        const float gd = tp.gt[d];
#pragma unroll
                        for (int k = 0; k < NS; ++k) cc[k] += gd * ps[k * TH * kTW];
                    }
                    o.epi(to, h, w, cc, part0, part1);
                }
            }
        }
    }
    if (acc_out) {
        const double s0 = block_sum((double)part0);
        if (threadIdx.x == 0) atomicAdd(acc_out, s0);
    }
    if (acc_out2) {
        const double s1 = block_sum((double)part1);
        if (threadIdx.x == 0) atomicAdd(acc_out2, s1);
    }
}

static inline size_t stencil_smem(int NS, int TH, const Taps& tp) {
    const int ZH = TH + 2 * tp.rh, ZW = kTW + 2 * tp.rw, nslot = 2 * tp.rt + 1;
    return sizeof(float) * (size_t)NS * ((size_t)ZH * ZW + (size_t)ZH * kTW + (size_t)nslot * TH * kTW);
}

// Choose the frame-chunk length so that the grid has a few CTAs per SM.
static inline int pick_tchunk(int T, int tiles, int rt) {
    const int target = 4 * num_sms();
    int nt = (target + tiles - 1) / tiles;
    if (nt < 1) nt = 1;
    if (nt > T) nt = T;
    int chunk = (T + nt - 1) / nt;
    const int minc = 2 * rt + 1;   // shorter chunks spend most time on the ring warm-up
    if (chunk < minc) chunk = minc < T ? minc : T;
    return chunk;
}

template <class Op>
static void run_stencil(const Op& op, const Taps& tp, int TH, const double* acc_in, double* acc_out,
                        double* acc_out2, int* flags, cudaStream_t s) {
    const Geom& g = op.g;
    const size_t smem = stencil_smem(Op::NS, TH, tp);
    static bool attr_set = false;   // one per Op instantiation
    if (!attr_set) {
        cudaFuncSetAttribute(stream_stencil<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    const int tx = (g.W + kTW - 1) / kTW, ty = (g.H + TH - 1) / TH;
    const int chunk = pick_tchunk(g.T, tx * ty, tp.rt);
    dim3 grid(tx, ty, (g.T + chunk - 1) / chunk);
    stream_stencil<Op><<<grid, kThreads, smem, s>>>(op, tp, TH, chunk, acc_in, acc_out, acc_out2, flags);
    count_launches(1);
}

}  // namespace sfseg
