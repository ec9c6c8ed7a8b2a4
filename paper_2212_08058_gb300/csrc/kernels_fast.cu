// kernels_fast.cu -- the power-iteration step of Eq. 7 for the radii the method is used with,
// (rt, rh, rw) = (1, 3, 3) and (2, 7, 7) (and the coarse-level radii (1, 4, 4), (1, 2, 2)),
// written for sm_103a.
//
// One CTA (128 threads, three per SM) owns a 15 x 64 tile of (h, w) and streams along t through
// a chunk of frames.  Per incoming frame:
//   1. TMA brings the raw halo tile of v (= u x~) and f into shared memory (15 + 2rh rows of
//      80 columns; zero fill outside the volume gives the zero padding, also for whole frames
//      before the first and after the last).  The copies of the next frames are in flight
//      while frame t is computed.
//   2. h-pass: a thread takes a column pair and 5 output rows (40 pairs x 3 row groups = 120 of
//      the 128 threads); it walks down the 5 + 2rh input rows once, forms the three signals z1 = v, z2 = f^2 v, z3 = f v of each, and accumulates
//      them into its 5 x 3 outputs with packed FP32 FMAs (FFMA2, one per column pair).
//   3. w-pass: a thread takes 8 output columns of one row; it loads its window of the h-pass
//      result once as aligned float2 pairs (the odd-aligned pairs are rebuilt in registers at
//      rw > 4; at rw <= 4 their taps run as two scalar FMAs instead) and feeds the three
//      w-filtered signals straight into the t-filter, kept in registers in transposed direct
//      form (2rt running partial sums per value, no frame ring to index).
//   4. Eq. 7 combination for the frame rt behind, the Eq. 8 norm partial and the store of the
//      next state.
// The h-pass result is double-buffered and the epilogue reads f from global memory, so a frame
// needs a single CTA barrier (after its h-pass): warps still finishing frame t overlap with
// warps already starting frame t+1.
// Bytes moved through shared memory per voxel are about 100 at (2,7,7): the TMA write, one
// read of the raw tile per 8 rows, one write and one windowed read of the h-pass result.  No
// pass re-reads its taps from shared memory and the t-filter reads nothing from it.  The frame
// loop is not unrolled, which keeps the kernel small enough for the instruction cache.
#include <cuda.h>


#include "common.cuh"
#include "launch.h"
#include "order_key.cuh"

namespace sfseg {
namespace fast {

#ifndef SFSEG_FAST_TH
#define SFSEG_FAST_TH 15
#endif
#ifndef SFSEG_FAST_RHS
#define SFSEG_FAST_RHS 5
#endif
constexpr int TH = SFSEG_FAST_TH;   // tile rows (at most 16: four rows per warp)
constexpr int TW = 64;         // tile columns
constexpr int PADW = 8;        // columns loaded left and right of the tile (16-byte aligned x)
constexpr int BW = TW + 2 * PADW;   // TMA box width
constexpr int QP = BW + 2;     // row pitch of the h-pass result (2 mod 32 avoids bank conflicts)
constexpr int RHS = SFSEG_FAST_RHS;   // output rows per h-pass item (divides TH)
constexpr int NTHR = 128;
constexpr long long kSpinLimit = 1ll << 26;   // bounded mbarrier wait
// Resident CTAs per SM the register allocation targets, and TMA stages (2: frame t+1 in flight
// while t is computed; 3: t+1 and t+2).  Compile-time tuning knobs.
#ifndef SFSEG_FAST_MINB
#define SFSEG_FAST_MINB 3
#endif
#ifndef SFSEG_FAST_NSTAGE
#define SFSEG_FAST_NSTAGE 2
#endif

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the barrier phase with an iteration limit; returns false if the limit was hit.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    for (long long i = 0; i < kSpinLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// A pair of adjacent stage elements as float2.
__device__ __forceinline__ float2 ld_pair(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ float2 ld_pair(const __nv_bfloat16* p) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
}

// Four pairs of float32 values to columns wbase .. wbase + 7 of an internal-layout row (pitch a
// multiple of 32, wbase of 8): two 16-byte stores when all eight columns are below W, else one
// value at a time.
__device__ __forceinline__ void st_pairs(float* o, const float2 p[4], int wbase, int W) {
    if (wbase + 8 <= W) {
        reinterpret_cast<float4*>(o)[0] = make_float4(p[0].x, p[0].y, p[1].x, p[1].y);
        reinterpret_cast<float4*>(o)[1] = make_float4(p[2].x, p[2].y, p[3].x, p[3].y);
    } else {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            if (wbase + 2 * m < W) o[2 * m] = p[m].x;
            if (wbase + 2 * m + 1 < W) o[2 * m + 1] = p[m].y;
        }
    }
}

template <int RT, int RH, int RW, typename TS, typename TVO, bool OUT_X>
struct Cfg {
    static constexpr int BH = TH + 2 * RH;                // TMA box height
    static constexpr int NSTAGE = SFSEG_FAST_NSTAGE;      // frame t, and the next ones in flight
    static constexpr int BOX_BYTES = (BW * BH * (int)sizeof(TS) + 127) / 128 * 128;
    static constexpr int STAGE_BYTES = 2 * BOX_BYTES;     // v then f
    static constexpr int Q_BYTES = 3 * TH * QP * 4;       // one h-pass result; two are kept
    static constexpr int SMEM = NSTAGE * STAGE_BYTES + 2 * Q_BYTES + NSTAGE * 8 + 128;
    static constexpr int CP_LO = (PADW - RW) / 2;         // first column pair the w-pass needs
    static constexpr int CP_HI = (PADW + TW + RW + 1) / 2;
    static constexpr int NCP = CP_HI - CP_LO;
    static constexpr int NHITEMS = NCP * (TH / RHS);
    static constexpr int ODD = RW & 1;
    static constexpr int NVAL = 8 + 2 * RW + ODD;         // w-pass window values (aligned start)
    static constexpr int NPAIR = (NVAL + 1) / 2;
    static_assert(NHITEMS <= NTHR, "h-pass items must fit the CTA");
    static_assert(TH % RHS == 0 && TH <= 16, "tile rows: a multiple of the h-pass item, at most 16");
    static_assert(RW <= PADW, "halo wider than the loaded pad");
};

struct Params {
    Geom g;
    float inv_alpha, p;
    float2 gt[2 * kMaxRT + 1], gh[2 * kMaxRH + 1], gw[2 * kMaxRW + 1];   // taps as (g, g) pairs
    int tchunk;
    const double* acc_in;
    double* acc_out;
    int* flags;
    void* out;        // next state (internal pitch) or x~ (caller layout)
    const void* f;    // f in global memory (internal pitch), read by the epilogue
    const float* s;   // separate unary map S_m (SEP kernels), or the state V_k (MODE 5); float32,
                      // internal pitch
    void* out2;       // second output: the record x~ (MODE 4) or Q (MODEs 5 and 6)
    // MODE 7 only: term j of the exact kernel's series (see below)
    int exj, exlast;
    float exc[3];     // c_{3j}, c_{3j+1}, c_{3j+2}
    float ex_alpha;
    unsigned* maxkey; // MODE 8: atomicMax of the order key of the largest output
};

// SEP: the unary term u = s^p comes from a separate map S_m (Eq. 9 with its own channels)
// instead of from f.  MODE 0 is the power-iteration step; MODE 4 is the same step that also
// records x~ (internal layout, out2) for the adjoint.  MODEs 1 and 5 serve the adjoint
// (kernels_bwd.cu): with c_0, c_1, c_2 the three filtered signals of the input v (G*v,
// G*(f^2 v), G*(f v)), Q = a1 c_0 - p c_1 + a3 c_2 with a1 = p (1/alpha - f^2) - 2 f^2,
// a3 = 2 (p + 1) f (the f-derivative weights of the step).  MODE 1 stores s Q.  MODE 5 stores
// G = u^2 B (B the Eq. 7 bracket, so G = u A z for v = u z) and Q, and adds sum V_k B over its
// voxels to acc_out, with V_k = u x~_k read from P.s (so that <x_k, A z> = s_k sum V_k B needs
// no division by u).  MODE 6 is the step (MODE 0, the state to out) that also stores s Q to out2:
// the adjoint's recomputation and Q-pass share the filtering of V_k.  MODE 7 serves the exact
// (Eq. 1) kernel, exp(-a (f_i - f_j)^2) = e^{-a f_i^2} e^{-a f_j^2} sum_n c_n f_i^n f_j^n with
// c_n = (2a)^n / n!: for the input v = f^{3j} w, its three filtered signals are the series
// terms n = 3j (G*v), 3j + 1 (G*(f v)) and 3j + 2 (G*(f^2 v)); it adds
// t = f^{3j} (c_{3j} G*v + f (c_{3j+1} G*(f v) + f c_{3j+2} G*(f^2 v))) to out (writes it when
// j = 0), and on the last term stores y = u e^{-a f^2} / a * (sum of the terms) and adds |y|^2 to
// acc_out.  All in the internal layout.  MODE 8 is the step (MODE 0) that also takes the
// largest of its outputs and adds it to P.maxkey (atomicMax of the order key, one per CTA): the
// maximum a soft-binarisation step (Alg. 1 step 3) scales by, without a pass of its own.
template <int RT, int RH, int RW, typename TS, typename TVO, bool OUT_X, bool SEP, int MODE>
__global__ void __launch_bounds__(NTHR, SFSEG_FAST_MINB)
iter_fast(const __grid_constant__ CUtensorMap mv, const __grid_constant__ CUtensorMap mf, Params P) {
    using C = Cfg<RT, RH, RW, TS, TVO, OUT_X>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    float* Qbuf = reinterpret_cast<float*>(smem + C::NSTAGE * C::STAGE_BYTES);   // [2][3][TH][QP]
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::NSTAGE * C::STAGE_BYTES + 2 * C::Q_BYTES);

    const int tid = threadIdx.x;
    const Geom g = P.g;
    const int w0 = blockIdx.x * TW, h0 = blockIdx.y * TH;
    const int t0 = blockIdx.z * P.tchunk;
    const int t1 = min(t0 + P.tchunk, g.T);
    // Frames before t = 0 are zero (zero padding): they would add exactly nothing to the
    // t-filter state, so the first chunk starts at frame 0.  Frames after the last are still
    // streamed, to flush the last rt output frames.
    const int tstart = max(t0 - RT, 0), tend = t1 + RT;

    const float s = inv_norm_from(P.acc_in, P.flags);
    const float2 s2 = f2(s);

    if (tid == 0) {
        for (int i = 0; i < C::NSTAGE; ++i) mbar_init(&bars[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    auto stage_v = [&](int frame) -> const TS* {
        return reinterpret_cast<const TS*>(smem + ((frame - tstart) % C::NSTAGE) * C::STAGE_BYTES);
    };
    auto stage_f = [&](int frame) -> const TS* {
        return reinterpret_cast<const TS*>(smem + ((frame - tstart) % C::NSTAGE) * C::STAGE_BYTES + C::BOX_BYTES);
    };
    int next_issue = tstart;         // thread 0: frames [tstart, next_issue) have been requested
    auto issue = [&](int frame) {   // thread 0 only
        next_issue = frame + 1;
        const int st = (frame - tstart) % C::NSTAGE;
        unsigned char* dst = smem + st * C::STAGE_BYTES;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(&bars[st], 2u * (uint32_t)(BW * C::BH * sizeof(TS)));
        tma_load_3d(dst, &mv, &bars[st], w0 - PADW, h0 - RH, frame);
        tma_load_3d(dst + C::BOX_BYTES, &mf, &bars[st], w0 - PADW, h0 - RH, frame);
    };

    // thread roles
    const int lane = tid & 31, warp = tid >> 5;
    const int wr = warp * 4 + ((lane & 15) >> 2);          // w-pass / epilogue row in the tile
    const int wcs = ((lane >> 4) << 2) | (lane & 3);        // its 8-column segment
    const bool hitem = tid < C::NHITEMS;
    const int hcp = C::CP_LO + tid % C::NCP;                // h-pass column pair
    const int hseg = tid / C::NCP;                          // h-pass row segment

    // the filter taps, copied once from the kernel parameters (measured ~1-2 % faster than reading
    // the parameter bank at every use)
    float2 ghr[2 * RH + 1], gwr[2 * RW + 1], gtr[2 * RT + 1];
#pragma unroll
    for (int d = 0; d <= 2 * RH; ++d) ghr[d] = P.gh[d];
#pragma unroll
    for (int d = 0; d <= 2 * RW; ++d) gwr[d] = P.gw[d];
#pragma unroll
    for (int d = 0; d <= 2 * RT; ++d) gtr[d] = P.gt[d];
    // t-filter in transposed direct form: for each of the 3 signals and 4 column pairs the
    // 2rt running partial sums of the 2rt+1-tap filter; with x[n] the w-filtered frame n and
    // g_j = gt[2rt - j], the output y[n] = sum_j g_j x[n - j] is the t-filtered frame n - rt.
    float2 st[2 * RT][3][4];
#pragma unroll
    for (int a = 0; a < 2 * RT; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int m = 0; m < 4; ++m) st[a][k][m] = make_float2(0.f, 0.f);
    float2 part = make_float2(0.f, 0.f);
    float tmax = 0.f;   // MODE 8: the largest output so far (outputs are >= 0)
    bool ok = true;

    if (tid == 0)
        for (int i = 0; i < C::NSTAGE - 1 && tstart + i < tend; ++i) issue(tstart + i);

#pragma unroll 1
    for (int tt = tstart; tt < tend; ++tt) {
        // The stage of frame tt+NSTAGE-1 last held frame tt-1, whose h-pass every thread
        // finished before the previous step's barrier.
        if (tid == 0 && tt + C::NSTAGE - 1 < tend) issue(tt + C::NSTAGE - 1);
        float* Q = Qbuf + ((tt - tstart) & 1) * (3 * TH * QP);
        const int to = tt - RT;          // output frame of this step
        const int h = h0 + wr;
        const int wbase = w0 + wcs * 8;
        // f of the output frame for the epilogue, requested now so that its latency hides
        // behind the two spatial passes.  Outside the volume f is taken as 0, so those
        // positions give x~ = 0 and add nothing to the norm (row padding is not relied on).
        float2 fo[4];
        float2 so[(SEP || MODE == 5) ? 4 : 1];
#pragma unroll
        for (int m = 0; m < 4; ++m) fo[m] = make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 0; m < ((SEP || MODE == 5) ? 4 : 1); ++m) so[m] = make_float2(0.f, 0.f);
        if (to >= t0 && h < g.H && wr < TH) {
            const TS* fg = reinterpret_cast<const TS*>(P.f) + ((int64_t)to * g.H + h) * g.pitch + wbase;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                if (wbase + 2 * m + 1 < g.W) fo[m] = ld_pair(fg + 2 * m);
                else if (wbase + 2 * m < g.W) fo[m].x = ldf(fg + 2 * m);
            }
            if constexpr (SEP || MODE == 5) {
                const float* sg = P.s + ((int64_t)to * g.H + h) * g.pitch + wbase;
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    if (wbase + 2 * m + 1 < g.W) so[m] = ld_pair(sg + 2 * m);
                    else if (wbase + 2 * m < g.W) so[m].x = sg[2 * m];
                }
            }
        }
        const uint32_t parity = (uint32_t)(((tt - tstart) / C::NSTAGE) & 1);
        const bool arrived = mbar_wait_bounded(&bars[(tt - tstart) % C::NSTAGE], parity);
        // ---------------- h-pass: raw stage -> Q[3][TH][QP]
        if (hitem && arrived) {
            const TS* sv = stage_v(tt) + (hseg * RHS) * BW + 2 * hcp;
            const TS* sf = stage_f(tt) + (hseg * RHS) * BW + 2 * hcp;
            float2 acc[RHS][3];
#pragma unroll
            for (int o = 0; o < RHS; ++o)
#pragma unroll
                for (int k = 0; k < 3; ++k) acc[o][k] = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < RHS + 2 * RH; ++j) {
                const float2 v = ld_pair(sv + j * BW);
                const float2 f = ld_pair(sf + j * BW);
                const float2 z3 = mul2(f, v);
                const float2 z2 = mul2(f, z3);
#pragma unroll
                for (int o = 0; o < RHS; ++o) {
                    const int d = j - o;
                    if (d >= 0 && d <= 2 * RH) {
                        const float2 gd = ghr[d];
                        acc[o][0] = fma2(v, gd, acc[o][0]);
                        acc[o][1] = fma2(z2, gd, acc[o][1]);
                        acc[o][2] = fma2(z3, gd, acc[o][2]);
                    }
                }
            }
#pragma unroll
            for (int o = 0; o < RHS; ++o)
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    *reinterpret_cast<float2*>(Q + (k * TH + hseg * RHS + o) * QP + 2 * hcp) = acc[o][k];
        }
        // The only barrier of the step: Q of this frame is complete, and every thread is done
        // with the h-pass of the previous frame (whose stage the next copy overwrites).
        if (__syncthreads_or(!arrived)) {
            ok = false;
            break;
        }
        // ---------------- w-pass: Q -> x[n], then the t-filter update
        float2 y[3][4];
        if (wr < TH) {
            const int a0 = PADW + wcs * 8 - RW - C::ODD;   // even
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float* qr = Q + (k * TH + wr) * QP + a0;
                float2 pa[C::NPAIR];
#pragma unroll
                for (int j = 0; j < C::NPAIR; ++j) pa[j] = ld_pair(qr + 2 * j);
                float2 acc[4];   // four independent chains (one per column pair)
#pragma unroll
                for (int m = 0; m < 4; ++m) acc[m] = make_float2(0.f, 0.f);
#pragma unroll
                for (int d = 0; d <= 2 * RW; ++d) {
                    const float2 gd = gwr[d];
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const int q = 2 * m + d + C::ODD;
                        if ((q & 1) && RW <= 4) {   // odd-aligned pair: two scalar FMAs
                            acc[m].x = fmaf(pa[q >> 1].y, gd.x, acc[m].x);
                            acc[m].y = fmaf(pa[(q >> 1) + 1].x, gd.x, acc[m].y);
                        } else {
                            const float2 in = (q & 1) ? make_float2(pa[q >> 1].y, pa[(q >> 1) + 1].x) : pa[q >> 1];
                            acc[m] = fma2(in, gd, acc[m]);
                        }
                    }
                }
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const float2 x = acc[m];
                    y[k][m] = fma2(x, gtr[2 * RT], st[0][k][m]);
#pragma unroll
                    for (int j = 0; j < 2 * RT - 1; ++j) st[j][k][m] = fma2(x, gtr[2 * RT - 1 - j], st[j + 1][k][m]);
                    st[2 * RT - 1][k][m] = mul2(x, gtr[0]);
                }
            }
        }
        // ---------------- Eq. 7 combination for frame to = tt - RT
        if (to >= t0 && wr < TH) {
            float2 outv[4];
            float2 outq[(MODE >= 4 && MODE <= 6) ? 4 : 1];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const float2 fv = fo[m];
                const float2 sv = SEP ? so[SEP ? m : 0] : fv;
                const float2 u = make_float2(unary_pow_fast(sv.x, P.p), unary_pow_fast(sv.y, P.p));
                const float2 e = fma2(make_float2(-fv.x, -fv.y), fv, f2(P.inv_alpha));   // 1/alpha - f^2
                if constexpr (MODE == 7) {
                    float2 F = make_float2(1.f, 1.f);
                    const float2 f3 = mul2(fv, mul2(fv, fv));
                    for (int i = 0; i < P.exj; ++i) F = mul2(F, f3);
                    const float2 inner = fma2(mul2(fv, f2(P.exc[2])), y[1][m], mul2(f2(P.exc[1]), y[2][m]));
                    outv[m] = mul2(F, fma2(fv, inner, mul2(f2(P.exc[0]), y[0][m])));
                } else if constexpr (MODE == 0 || MODE == 4 || MODE == 6 || MODE == 8) {
                    float2 B = fma2(e, y[0][m], make_float2(-y[1][m].x, -y[1][m].y));
                    B = fma2(mul2(f2(2.f), fv), y[2][m], B);
                    const float2 xt = mul2(mul2(s2, u), B);
                    part = fma2(xt, xt, part);
                    if constexpr (MODE == 8) tmax = fmaxf(tmax, fmaxf(xt.x, xt.y));
                    outv[m] = OUT_X ? xt : mul2(u, xt);
                    if constexpr (MODE == 4) outq[m] = xt;
                    if constexpr (MODE == 6) {
                        const float2 a1 = fma2(f2(P.p), e, mul2(f2(-2.f), mul2(fv, fv)));
                        const float2 a3 = mul2(f2(2.f * (P.p + 1.f)), fv);
                        const float2 Q = fma2(a1, y[0][m], mul2(f2(-P.p), y[1][m]));
                        outq[MODE == 6 ? m : 0] = mul2(s2, fma2(a3, y[2][m], Q));
                    }
                } else {
                    const float2 a1 = fma2(f2(P.p), e, mul2(f2(-2.f), mul2(fv, fv)));
                    const float2 a3 = mul2(f2(2.f * (P.p + 1.f)), fv);
                    float2 Q = fma2(a1, y[0][m], mul2(f2(-P.p), y[1][m]));
                    Q = mul2(s2, fma2(a3, y[2][m], Q));
                    if constexpr (MODE == 1) {
                        outv[m] = Q;
                    } else {
                        float2 B = fma2(e, y[0][m], make_float2(-y[1][m].x, -y[1][m].y));
                        B = fma2(mul2(f2(2.f), fv), y[2][m], B);
                        outv[m] = mul2(mul2(u, u), B);
                        part = fma2(so[MODE == 5 ? m : 0], B, part);
                        outq[MODE == 5 ? m : 0] = Q;
                    }
                }
            }
            if constexpr (MODE == 4 || MODE == 6) {
                if (h < g.H) {
                    float* o2 = reinterpret_cast<float*>(P.out2) + ((int64_t)to * g.H + h) * g.pitch + wbase;
                    st_pairs(o2, outq, wbase, g.W);
                }
            }
            if constexpr (MODE == 7) {
                if (h < g.H) {
                    float* o = reinterpret_cast<float*>(P.out) + ((int64_t)to * g.H + h) * g.pitch + wbase;
                    if (P.exj > 0) {   // the terms so far
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            if (wbase + 2 * m + 1 < g.W) outv[m] = __fadd2_rn(outv[m], ld_pair(o + 2 * m));
                            else if (wbase + 2 * m < g.W) outv[m].x += o[2 * m];
                        }
                    }
                    if (P.exlast) {
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            const float2 fv = fo[m];
                            const float2 a = make_float2(
                                unary_pow_fast(fv.x, P.p) * expf(-P.ex_alpha * fv.x * fv.x) * P.inv_alpha,
                                unary_pow_fast(fv.y, P.p) * expf(-P.ex_alpha * fv.y * fv.y) * P.inv_alpha);
                            outv[m] = mul2(a, outv[m]);
                            part = fma2(outv[m], outv[m], part);
                        }
                    }
                    st_pairs(o, outv, wbase, g.W);
                }
            } else if constexpr (MODE == 1 || MODE == 5) {
                if (h < g.H) {
                    float* o = reinterpret_cast<float*>(P.out) + ((int64_t)to * g.H + h) * g.pitch + wbase;
                    st_pairs(o, outv, wbase, g.W);
                    if constexpr (MODE == 5) {
                        float* o2 = reinterpret_cast<float*>(P.out2) + ((int64_t)to * g.H + h) * g.pitch + wbase;
                        st_pairs(o2, outq, wbase, g.W);
                    }
                }
            } else
            if (h < g.H) {
                if (OUT_X) {
                    // caller layout: rows of W values, 8-byte aligned when W is even (and the
                    // caller's base is), then one 8-byte store per pair
                    float* o = reinterpret_cast<float*>(P.out) + ((int64_t)to * g.H + h) * g.W + wbase;
                    if (wbase + 8 <= g.W && (reinterpret_cast<uintptr_t>(o) & 7) == 0) {
#pragma unroll
                        for (int m = 0; m < 4; ++m) reinterpret_cast<float2*>(o)[m] = outv[m];
                    } else {
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            if (wbase + 2 * m < g.W) o[2 * m] = outv[m].x;
                            if (wbase + 2 * m + 1 < g.W) o[2 * m + 1] = outv[m].y;
                        }
                    }
                } else {
                    TVO* o = reinterpret_cast<TVO*>(P.out) + ((int64_t)to * g.H + h) * g.pitch + wbase;
                    if (wbase + 8 <= g.W) {
                        if constexpr (sizeof(TVO) == 4) {
                            reinterpret_cast<float4*>(o)[0] = make_float4(outv[0].x, outv[0].y, outv[1].x, outv[1].y);
                            reinterpret_cast<float4*>(o)[1] = make_float4(outv[2].x, outv[2].y, outv[3].x, outv[3].y);
                        } else {
                            __nv_bfloat162 b[4];
#pragma unroll
                            for (int m = 0; m < 4; ++m) b[m] = __float22bfloat162_rn(outv[m]);
                            *reinterpret_cast<uint4*>(o) = *reinterpret_cast<const uint4*>(b);
                        }
                    } else {
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            if (wbase + 2 * m < g.W) stf(o + 2 * m, outv[m].x);
                            if (wbase + 2 * m + 1 < g.W) stf(o + 2 * m + 1, outv[m].y);
                        }
                    }
                }
            }
        }
    }
    if (!ok) {
        if (tid == 0) {
            atomicOr(P.flags, kFlagTimeout);
            // let copies still in flight land before the CTA's shared memory goes away: for each
            // stage, wait (bounded) for the phase of the last frame requested into it
            for (int i = 0; i < C::NSTAGE && tstart + i < next_issue; ++i) {
                const int last = i + ((next_issue - 1 - tstart - i) / C::NSTAGE) * C::NSTAGE;   // relative frame
                mbar_wait_bounded(&bars[i], (uint32_t)((last / C::NSTAGE) & 1));
            }
        }
        return;
    }
    const double tot = block_sum((double)part.x + (double)part.y);
    if (tid == 0 && P.acc_out) atomicAdd(P.acc_out, tot);
    if constexpr (MODE == 8) {
        __shared__ unsigned wmax[NTHR / 32];
        const unsigned kmax = __reduce_max_sync(0xffffffffu, order_key(tmax));
        if (lane == 0) wmax[warp] = kmax;
        __syncthreads();
        if (tid == 0) {
            unsigned m = wmax[0];
            for (int i = 1; i < NTHR / 32; ++i) m = max(m, wmax[i]);
            atomicMax(P.maxkey, m);
        }
    }
}

// ------------------------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

static bool make_map(CUtensorMap* map, const void* base, bool bf16, const Geom& g, int box_h) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const size_t es = bf16 ? 2 : 4;
    cuuint64_t dims[3] = {(cuuint64_t)g.W, (cuuint64_t)g.H, (cuuint64_t)g.T};
    cuuint64_t strides[2] = {(cuuint64_t)g.pitch * es, (cuuint64_t)g.pitch * es * g.H};
    cuuint32_t box[3] = {(cuuint32_t)BW, (cuuint32_t)box_h, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                    const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Frame-chunk length minimising (waves x frames per chunk) for `slots` resident CTAs.
static int pick_chunk(int T, int tiles, int slots, int rt) {
    long best_cost = -1;
    int best = T;
    for (int nt = 1; nt <= T; ++nt) {
        const int chunk = (T + nt - 1) / nt;
        const int nct = (T + chunk - 1) / chunk;
        const long waves = ((long)tiles * nct + slots - 1) / slots;
        const long cost = waves * (chunk + 2 * rt);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = chunk;
        }
    }
    return best;
}

template <int RT, int RH, int RW, typename TS, typename TVO, bool OUT_X, bool SEP = false, int MODE = 0>
static bool launch_t(const void* vin, void* out, const void* f, const Geom& g, const Taps& tp, float inv_alpha,
                     float p, const double* acc_in, double* acc_out, int* flags, cudaStream_t s,
                     const float* s32 = nullptr, void* out2 = nullptr, const ExactTerm* ex = nullptr,
                     unsigned* maxkey = nullptr) {
    using C = Cfg<RT, RH, RW, TS, TVO, OUT_X>;
    constexpr bool bf = sizeof(TS) == 2;
    CUtensorMap mv, mf;
    if (!make_map(&mv, vin, bf, g, C::BH) || !make_map(&mf, f, bf, g, C::BH)) return false;
    auto kern = iter_fast<RT, RH, RW, TS, TVO, OUT_X, SEP, MODE>;
    static int slots_per_sm = -1;
    static unsigned long long attr_set = 0;   // devices on which the attribute is set
    if (!(attr_set & device_bit())) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM) != cudaSuccess) return false;
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, NTHR, C::SMEM);
        slots_per_sm = nb > 0 ? nb : 1;
        attr_set |= device_bit();
    }
    Params P;
    P.g = g;
    P.inv_alpha = inv_alpha;
    P.p = p;
    for (int i = 0; i < 2 * kMaxRT + 1; ++i) P.gt[i] = make_float2(tp.gt[i], tp.gt[i]);
    for (int i = 0; i < 2 * kMaxRH + 1; ++i) P.gh[i] = make_float2(tp.gh[i], tp.gh[i]);
    for (int i = 0; i < 2 * kMaxRW + 1; ++i) P.gw[i] = make_float2(tp.gw[i], tp.gw[i]);
    P.f = f;
    P.s = s32;
    P.out2 = out2;
    P.exj = ex ? ex->j : 0;
    P.exlast = ex ? ex->last : 0;
    for (int i = 0; i < 3; ++i) P.exc[i] = ex ? ex->c[i] : 0.f;
    P.ex_alpha = ex ? ex->alpha : 0.f;
    P.maxkey = maxkey;
    const int tx = (g.W + TW - 1) / TW, ty = (g.H + TH - 1) / TH;
    P.tchunk = pick_chunk(g.T, tx * ty, slots_per_sm * num_sms(), RT);
    P.acc_in = acc_in;
    P.acc_out = acc_out;
    P.flags = flags;
    P.out = out;
    dim3 grid(tx, ty, (g.T + P.tchunk - 1) / P.tchunk);
    kern<<<grid, NTHR, C::SMEM, s>>>(mv, mf, P);
    count_launches(1);
    return true;
}

template <int RT, int RH, int RW>
static bool dispatch(const void* vin, int vin_type, void* out, int out_type, bool out_x, const void* f,
                     const Geom& g, const Taps& tp, float ia, float p, const double* ai, double* ao, int* fl,
                     cudaStream_t s, const float* s32) {
    using bf = __nv_bfloat16;
    if (s32) {   // separate unary map: float32 storage only (the generic stencil serves bf16)
        if (vin_type != kF32) return false;
        if (out_x) return launch_t<RT, RH, RW, float, float, true, true>(vin, out, f, g, tp, ia, p, ai, ao, fl, s, s32);
        return launch_t<RT, RH, RW, float, float, false, true>(vin, out, f, g, tp, ia, p, ai, ao, fl, s, s32);
    }
    if (vin_type == kF32) {
        if (out_x) return launch_t<RT, RH, RW, float, float, true>(vin, out, f, g, tp, ia, p, ai, ao, fl, s);
        return launch_t<RT, RH, RW, float, float, false>(vin, out, f, g, tp, ia, p, ai, ao, fl, s);
    }
    if (out_x) return launch_t<RT, RH, RW, bf, float, true>(vin, out, f, g, tp, ia, p, ai, ao, fl, s);
    if (out_type == kBF16) return launch_t<RT, RH, RW, bf, bf, false>(vin, out, f, g, tp, ia, p, ai, ao, fl, s);
    return launch_t<RT, RH, RW, bf, float, false>(vin, out, f, g, tp, ia, p, ai, ao, fl, s);
}

// The recording step (MODE 4), float32 only.
template <int RT, int RH, int RW>
static bool dispatch_ckpt(const float* vin, void* out, bool out_x, const float* f, const Geom& g, const Taps& tp,
                          float ia, float p, const double* ai, double* ao, float* ckpt, int* fl, cudaStream_t s) {
    if (out_x)
        return launch_t<RT, RH, RW, float, float, true, false, 4>(vin, out, f, g, tp, ia, p, ai, ao, fl, s, nullptr,
                                                                ckpt);
    return launch_t<RT, RH, RW, float, float, false, false, 4>(vin, out, f, g, tp, ia, p, ai, ao, fl, s, nullptr,
                                                             ckpt);
}

// The adjoint's Q-pass (MODE 1), float32 only.
template <int RT, int RH, int RW>
static bool dispatch_filter(const float* vin, int mode, float* out, float* out2, const float* f, const Geom& g,
                            const Taps& tp, float ia, float p, const double* ai, int* fl, cudaStream_t s) {
    (void)out2;
    if (mode != 1) return false;
    return launch_t<RT, RH, RW, float, float, false, false, 1>(vin, out, f, g, tp, ia, p, ai, nullptr, fl, s);
}

// The adjoint's recomputing step with its Q-pass (MODE 6), float32 only.
template <int RT, int RH, int RW>
static bool dispatch_step_q(const float* vin, float* vout, float* Q, const float* f, const Geom& g, const Taps& tp,
                            float ia, float p, const double* ai, int* fl, cudaStream_t s) {
    return launch_t<RT, RH, RW, float, float, false, false, 6>(vin, vout, f, g, tp, ia, p, ai, nullptr, fl, s, nullptr,
                                                             Q);
}

// A term of the exact kernel's series (MODE 7), float32 only.
template <int RT, int RH, int RW>
static bool dispatch_exact(const float* v, float* y, const float* f, const Geom& g, const Taps& tp, float ia, float p,
                           const ExactTerm& ex, double* acc_out, int* fl, cudaStream_t s) {
    return launch_t<RT, RH, RW, float, float, false, false, 7>(v, y, f, g, tp, ia, p, nullptr, acc_out, fl, s, nullptr,
                                                             nullptr, &ex);
}

// The step into the caller layout that also adds its largest output to *maxkey (MODE 8),
// float32, shared maps.
template <int RT, int RH, int RW>
static bool dispatch_max(const float* vin, float* y, const float* f, const Geom& g, const Taps& tp, float ia, float p,
                         unsigned* maxkey, int* fl, cudaStream_t s) {
    return launch_t<RT, RH, RW, float, float, true, false, 8>(vin, y, f, g, tp, ia, p, nullptr, nullptr, fl, s, nullptr,
                                                            nullptr, nullptr, maxkey);
}

// The adjoint's g-pass in state form (MODE 5), float32 only.
template <int RT, int RH, int RW>
static bool dispatch_gpass(const float* vg, float* G, float* Qg, const float* Vk, const float* f, const Geom& g,
                           const Taps& tp, float ia, float p, double* dot, int* fl, cudaStream_t s) {
    return launch_t<RT, RH, RW, float, float, false, false, 5>(vg, G, f, g, tp, ia, p, nullptr, dot, fl, s, Vk, Qg);
}

}  // namespace fast

// Radii with a compiled kernel: the method's (1,3,3) and (2,7,7); (1,4,4), (1,2,2), the radii of
// (2,7,7) on 2x- and 4x-coarsened volumes (sfseg_coarse_start); and the neighbourhoods between
// them, (1,5,5), (2,3,3), (2,5,5), (1,7,7).  Others run on the generic streaming stencil.
#define SFSEG_FAST_RADII(X) X(1, 3, 3) X(2, 7, 7) X(1, 4, 4) X(1, 2, 2) X(1, 5, 5) X(2, 3, 3) X(2, 5, 5) X(1, 7, 7)

bool fast_iterate_supported(const Taps& tp) {
#define SFSEG_IS(A, B, C) if (tp.rt == A && tp.rh == B && tp.rw == C) return true;
    SFSEG_FAST_RADII(SFSEG_IS)
#undef SFSEG_IS
    return false;
}

bool launch_iterate_fast(const void* vin, int vin_type, void* out, int out_type, bool out_x, const void* f,
                         const Geom& g, const Taps& tp, float inv_alpha, float p, const double* acc_in,
                         double* acc_out, int* flags, cudaStream_t s, const float* s32) {
#define SFSEG_GO(A, B, C)                                                                                   \
    if (tp.rt == A && tp.rh == B && tp.rw == C)                                                             \
        return fast::dispatch<A, B, C>(vin, vin_type, out, out_type, out_x, f, g, tp, inv_alpha, p, acc_in, \
                                       acc_out, flags, s, s32);
    SFSEG_FAST_RADII(SFSEG_GO)
#undef SFSEG_GO
    return false;
}

bool launch_iterate_fast_max(const float* vin, float* y, const float* f, const Geom& g, const Taps& tp,
                             float inv_alpha, float p, unsigned* maxkey, int* flags, cudaStream_t s) {
#define SFSEG_GO(A, B, C)                                                                                 \
    if (tp.rt == A && tp.rh == B && tp.rw == C)                                                           \
        return fast::dispatch_max<A, B, C>(vin, y, f, g, tp, inv_alpha, p, maxkey, flags, s);
    SFSEG_FAST_RADII(SFSEG_GO)
#undef SFSEG_GO
    return false;
}

bool launch_iterate_fast_ckpt(const float* vin, void* out, bool out_x, const float* f, const Geom& g, const Taps& tp,
                              float inv_alpha, float p, const double* acc_in, double* acc_out, float* ckpt, int* flags,
                              cudaStream_t s) {
#define SFSEG_GO(A, B, C)                                                                                        \
    if (tp.rt == A && tp.rh == B && tp.rw == C)                                                                  \
        return fast::dispatch_ckpt<A, B, C>(vin, out, out_x, f, g, tp, inv_alpha, p, acc_in, acc_out, ckpt, flags, \
                                            s);
    SFSEG_FAST_RADII(SFSEG_GO)
#undef SFSEG_GO
    return false;
}

bool launch_filter_fast(const float* vin, int mode, float* out, float* out2, const float* f, const Geom& g,
                        const Taps& tp, float inv_alpha, float p, const double* acc_in, int* flags, cudaStream_t s) {
#define SFSEG_GO(A, B, C)                                                                                     \
    if (tp.rt == A && tp.rh == B && tp.rw == C)                                                               \
        return fast::dispatch_filter<A, B, C>(vin, mode, out, out2, f, g, tp, inv_alpha, p, acc_in, flags, s);
    SFSEG_FAST_RADII(SFSEG_GO)
#undef SFSEG_GO
    return false;
}

bool launch_adjoint_gpass_fast(const float* vg, float* G, float* Qg, const float* Vk, const float* f, const Geom& g,
                               const Taps& tp, float inv_alpha, float p, double* dot, int* flags, cudaStream_t s) {
#define SFSEG_GO(A, B, C)                                                                                  \
    if (tp.rt == A && tp.rh == B && tp.rw == C)                                                            \
        return fast::dispatch_gpass<A, B, C>(vg, G, Qg, Vk, f, g, tp, inv_alpha, p, dot, flags, s);
    SFSEG_FAST_RADII(SFSEG_GO)
#undef SFSEG_GO
    return false;
}

bool launch_step_q_fast(const float* vin, float* vout, float* Q, const float* f, const Geom& g, const Taps& tp,
                        float inv_alpha, float p, const double* acc_in, int* flags, cudaStream_t s) {
#define SFSEG_GO(A, B, C)                                                                                  \
    if (tp.rt == A && tp.rh == B && tp.rw == C)                                                            \
        return fast::dispatch_step_q<A, B, C>(vin, vout, Q, f, g, tp, inv_alpha, p, acc_in, flags, s);
    SFSEG_FAST_RADII(SFSEG_GO)
#undef SFSEG_GO
    return false;
}

bool launch_exact_term_fast(const float* v, float* y, const float* f, const Geom& g, const Taps& tp, float inv_alpha,
                            float p, const ExactTerm& ex, double* acc_out, int* flags, cudaStream_t s) {
#define SFSEG_GO(A, B, C)                                                                                  \
    if (tp.rt == A && tp.rh == B && tp.rw == C)                                                            \
        return fast::dispatch_exact<A, B, C>(v, y, f, g, tp, inv_alpha, p, ex, acc_out, flags, s);
    SFSEG_FAST_RADII(SFSEG_GO)
#undef SFSEG_GO
    return false;
}

}  // namespace sfseg
