// net.cu -- the learned warm start: a 4-layer 3x3x3 convolutional network that predicts a
// start vector x0 >= 0 for the power iteration from the raw input channels.  (The paper starts
// from a uniform vector or from S_m, Alg. 1 line 3; the network is an addition to the method.)
//
//   L1: C_in (<= 16, zero-padded to 16) -> 32, ReLU      L2, L3: 32 -> 32, ReLU
//   L4: 32 -> 1, softplus (its own kernel, conv_last_tc: the nine (dh, dw) taps of each output
//       frame on N)
//
// Activations are bf16 in channels-last layout [T][H][W][C]; every convolution is an implicit
// GEMM on the 5th-generation tensor cores (tcgen05.mma, kind::f16, bf16 x bf16 -> fp32 in TMEM):
//   D[v, co] = sum_{tap, ci} X[v + tap, ci] W[co, tap, ci],   M = 128 voxels of one row along w,
//   K = 16 input channels per instruction.  Each input row is read once: its 9 (dt, dw) taps x
//   C_in/16 MMAs each carry the three taps along h at once (N = 3 x output channels, D over the
//   accumulators of the three output rows it feeds, a ring of blocks in TMEM).
// The A operand is read straight from a TMA-filled ring of input rows in the canonical
// no-swizzle K-major layout ([8-channel chunk][frames][130 voxels][8 channels]); a tap's shift
// along w is a 16-byte offset of the descriptor's start address, along t a 2080-byte offset.
// All weights of the layer stay in shared memory.  A CTA computes up to three consecutive output
// frames from input slots of two more frames: one warp issues the TMA copies, one per output
// frame issues its MMAs (each into its part of TMEM), four per frame read each finished row's
// accumulator from TMEM, zero it, and run the epilogue.  The
// backward pass reuses the same kernel for the data gradient (flipped taps, transposed
// channels, ReLU mask in the epilogue); the weight gradient is its own tcgen05 kernel with the
// voxels as the reduction dimension (wgrad_tc).
#include <cuda.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sfseg.h"
#include "common.cuh"
#include "launch.h"

namespace sfseg {
namespace net {

constexpr int MT = 128;                 // voxels per MMA tile (rows of A)
constexpr int RW = MT + 2;              // voxels per loaded row (w halo of 1)
#ifndef SFSEG_NET_NSLOT
#define SFSEG_NET_NSLOT 4
#endif
constexpr int NSLOT = SFSEG_NET_NSLOT;  // input-row ring (rows in flight ahead of the MMAs: NSLOT - 2)
constexpr int NTHR = 192;               // 6 warps
// Output rows per CTA: the tallest of 64, 32, 16 that still gives the grid 4 waves (taller
// tiles load fewer halo rows and amortise each CTA's weight copy and TMEM set-up).
constexpr int kHrChoices[3] = {64, 32, 16};
constexpr long long kSpin = 1ll << 26;

enum Epi { EPI_RELU = 0, EPI_MASK = 2 };

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mb_init(uint64_t* b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mb_expect(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mb_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ bool mb_try(uint64_t* b, uint32_t par) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(par)
        : "memory");
    return ok != 0;
}
// Bounded wait: on timeout raise the flag and report failure (the caller then stops issuing).
__device__ __forceinline__ bool mb_wait(uint64_t* b, uint32_t par, int* flags) {
    for (long long i = 0; i < kSpin; ++i)
        if (mb_try(b, par)) return true;
    atomicOr(flags, kFlagTimeout);
    return false;
}
// Bounded wait that reports nothing (used after a timeout has already been flagged).
__device__ __forceinline__ void mb_settle(uint64_t* b, uint32_t par) {
    for (long long i = 0; i < kSpin; ++i)
        if (mb_try(b, par)) return;
}
__device__ __forceinline__ void tma4(void* dst, const CUtensorMap* m, uint64_t* b, int c0, int c1, int c2, int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(su32(dst)), "l"(m), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(su32(b))
        : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(su32(dst)), "l"(src), "r"(bytes), "r"(su32(b))
                 : "memory");
}
// Shared-memory matrix descriptor: canonical K-major layout without swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor, kind::f16: bf16 A and B (K-major), fp32 D, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(MT >> 4) << 24);
}
__device__ __forceinline__ void umma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d), "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void umma_commit(uint64_t* b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t (&r)[N]);
template <>
__device__ __forceinline__ void tmem_ld<32>(uint32_t t, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(t));
}
template <>
__device__ __forceinline__ void tmem_ld<16>(uint32_t t, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(t));
}

// Writes zeros to N columns of this warp's 32 TMEM lanes starting at taddr.
template <int N>
__device__ __forceinline__ void tmem_zero(uint32_t t);
template <>
__device__ __forceinline__ void tmem_zero<32>(uint32_t t) {
    const uint32_t z = 0u;
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};"
        ::"r"(t), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z),
          "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z),
          "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z)
        : "memory");
}
template <>
__device__ __forceinline__ void tmem_zero<16>(uint32_t t) {
    const uint32_t z = 0u;
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};"
        ::"r"(t), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z),
          "r"(z), "r"(z), "r"(z), "r"(z)
        : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

struct ConvArgs {
    int T, H, W;
    int HR;                       // output rows per CTA
    const __nv_bfloat16* wpack;   // packed weights (layout of the smem B operand)
    const float* bias;            // [COUT] or null
    void* out;                    // bf16 [T][H][W][COUT]
    const __nv_bfloat16* mask;    // EPI_MASK: activation [T][H][W][COUT] whose sign gates the output
    int* flags;
};

// The three taps along h of one (dt, dw, ks) share one MMA: an input row h' feeds the output
// rows h' + 1, h', h' - 1 through the weights of dh = 0, 1, 2, so B stacks the three weight
// blocks along N (N = 3 COUT) and D spans the accumulators of three output rows.  Each output
// frame of the CTA has a ring of R blocks of COUT columns in its share of the TMEM columns;
// output row j uses block (-j) mod R, so the rows i, i - 1, i - 2 fed by input row i sit in
// consecutive blocks (an MMA is split in two where the ring wraps, and trimmed at the tile's
// first and last rows).  A block is zeroed when its row has been read, so every MMA accumulates.
// An input slot holds FR + 2 frames of one row; the issuer of output frame t0 + q reads its
// frames q, q + 1, q + 2.
// FR output frames per CTA, one MMA-issuing thread each: several issuers keep the tensor pipe
// busier than one (each waits on its own barriers and its MMAs' operand reads), and the frames
// share each loaded input row (FR + 2 frames of it instead of three per output frame).  Measured
// at 1080p: three frames per CTA take the 16-channel first layer from 7.19 to 6.59 ms against
// two, and the 32-channel layers from 11.37 to 11.34 ms.  Fewer frames per CTA serve volumes too
// small to fill the GPU with three.
template <int CIN, int COUT, int FR_>
struct ConvCfg {
    static constexpr int FR = FR_;                            // output frames per CTA
    static constexpr int NF = FR + 2;                         // frames per input slot
    static constexpr int NCH = CIN / 8;                       // 8-channel chunks of A
    static constexpr int KS = CIN / 16;                       // MMAs per tap
    static constexpr int CHUNK_DATA = NF * RW * 16;           // one 8-channel chunk of NF frames
    static constexpr int CHUNK = (CHUNK_DATA + 127) / 128 * 128;   // its stride (128-byte aligned TMA target)
    static constexpr int SLOT_BYTES = NCH * CHUNK;
    static constexpr int WBYTES = 27 * KS * 2 * COUT * 16;    // packed weights
    static constexpr int RING = (512 / FR) / 32 * 32;         // TMEM columns of one output frame
    static constexpr int R = RING / COUT;                     // accumulator blocks in its ring
    // input-row slots: measured at 1080p, 3 for 32 input channels (11.5 ms per layer against
    // 11.8 with 2 and 11.9 with 4) and 5 for 16 (7.17 ms against 7.22 with 4 and 7.45 with 8)
    static constexpr int NS = CIN >= 32 ? 3 : 5;
    static constexpr int NTHR = 32 * (1 + FR + 4 * FR);       // producer, issuers, 4 epilogue warps per frame
    // full[NS], empty[NS], accf[FR][R], acce[FR][R], wbar, drain[FR]
    static constexpr int NB = 2 * NS + 2 * FR * R + 1 + FR;
    static constexpr int SMEM_NEED = WBYTES + NS * SLOT_BYTES + NB * 8 + 16 + 128;
    // at least 120 KB so that one CTA holds the SM's tensor memory alone
    static constexpr int SMEM = SMEM_NEED > 120 * 1024 ? SMEM_NEED : 120 * 1024;
    static_assert(FR >= 1 && FR <= 3, "one to three output frames per CTA");
    static_assert(R >= 4 && 3 * COUT <= 256 && COUT % 16 == 0, "accumulator ring");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

template <int CIN, int COUT, int EPI, int FR>
__global__ void __launch_bounds__(ConvCfg<CIN, COUT, FR>::NTHR, 1)
conv3d_tc(const __grid_constant__ CUtensorMap xin, ConvArgs a) {
    using C = ConvCfg<CIN, COUT, FR>;
    extern __shared__ __align__(128) unsigned char sm_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)sm_raw + 127) & ~(uintptr_t)127);
    unsigned char* wsm = sm;                                   // weights
    unsigned char* ring = sm + C::WBYTES;                      // the input-row slots
    uint64_t* bar = reinterpret_cast<uint64_t*>(ring + C::NS * C::SLOT_BYTES);
    uint64_t* full = bar;                        // [NS]
    uint64_t* empty = bar + C::NS;               // [NS]: released by each active issuer
    uint64_t* accf = bar + 2 * C::NS;            // [FR][R]: the row in accumulator block b is complete
    uint64_t* acce = accf + C::FR * C::R;        // [FR][R]: block b has been read and zeroed
    uint64_t* wbar = acce + C::FR * C::R;
    uint64_t* drain = wbar + 1;                  // [FR]: completion of an issuer's MMAs, awaited after a timeout
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + C::NB);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // work item: (group of up to FR output frames, w segment, row range)
    const int HR = a.HR;
    const int nws = (a.W + MT - 1) / MT, nhr = (a.H + HR - 1) / HR;
    int item = blockIdx.x;
    const int hr = item % nhr;
    item /= nhr;
    const int ws = item % nws;
    const int t0 = (item / nws) * C::FR;
    const int nfr = min(C::FR, a.T - t0);        // output frames of this CTA (1 at an odd T's end)
    const int w0 = ws * MT, hs = hr * HR, he = min(a.H, hs + HR);
    const int nout = he - hs, nin = nout + 2;

    if (threadIdx.x == 0) {
        for (int i = 0; i < C::NS; ++i) {
            mb_init(&full[i], 1);
            mb_init(&empty[i], (uint32_t)nfr);
        }
        for (int i = 0; i < C::FR * C::R; ++i) {
            mb_init(&accf[i], 1);
            mb_init(&acce[i], 4);
        }
        mb_init(wbar, 1);
        for (int q = 0; q < C::FR; ++q) mb_init(&drain[q], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    auto blk = [&](int j) { return (C::R - j % C::R) % C::R; };   // accumulator block of output row j
    const int epi = warp - 1 - C::FR;            // epilogue warp index, 4 per output frame
    if (epi >= 0) {   // the epilogue warps zero their frame's ring (their lane quadrants) once
        const uint32_t base = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((epi >> 2) * C::RING);
#pragma unroll 1
        for (int b = 0; b < C::R; ++b) tmem_zero<COUT>(base + (uint32_t)(b * COUT));
        tmem_st_wait();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    int issued = 0;                  // producer: input rows requested so far
    if (warp == 0) {
        if (lane == 0) {   // ---------------- producer: weights, then the input rows
            mb_expect(wbar, C::WBYTES);
            bulk_g2s(wsm, a.wpack, C::WBYTES, wbar);
            for (int i = 0; i < nin; ++i) {
                const int s = i % C::NS;
                if (i >= C::NS && !mb_wait(&empty[s], (uint32_t)((i / C::NS - 1) & 1), a.flags)) break;
                issued = i + 1;
                mb_expect(&full[s], C::NCH * C::CHUNK_DATA);
                unsigned char* dst = ring + s * C::SLOT_BYTES;
                for (int k = 0; k < C::NCH; ++k) tma4(dst + k * C::CHUNK, &xin, &full[s], 8 * k, w0 - 1, hs - 1 + i, t0 - 1);
            }
        }
    } else if (epi < 0) {
        const int q = warp - 1;      // output frame t0 + q
        if (lane == 0 && q < nfr) {   // ---------------- MMA issuer of one output frame
            bool ok = mb_wait(wbar, 0, a.flags);
            const uint32_t wbase = su32(wsm), rbase = su32(ring);
            const uint32_t dbase = tmem + (uint32_t)(q * C::RING);
            uint64_t* af = accf + q * C::R;
            uint64_t* ae = acce + q * C::R;
            constexpr uint32_t TILE = 2 * 3 * COUT * 16;          // stacked B tile of one (dt, dw, ks)
            for (int i = 0; ok && i < nin; ++i) {
                ok = mb_wait(&full[i % C::NS], (uint32_t)((i / C::NS) & 1), a.flags);
                // output rows fed by input row i: j = i - dh for dh = 0, 1, 2, within [0, nout)
                const int jhi = min(i, nout - 1), jlo = max(i - 2, 0);
                // row i enters the ring: its block must have been read back from row i - R
                if (ok && i < nout && i >= C::R)
                    ok = mb_wait(&ae[blk(i)], (uint32_t)(((i - C::R) / C::R) & 1), a.flags);
                if (!ok) break;
                tc_fence_after();
                const int dh0 = i - jhi, nrow = jhi - jlo + 1;
                const int b0 = blk(jhi);
                const int n1 = min(nrow, C::R - b0), n2 = nrow - n1;   // before and after the wrap
                const uint32_t id1 = idesc_bf16(n1 * COUT), id2 = idesc_bf16((n2 > 0 ? n2 : 1) * COUT);
                const uint32_t d1 = dbase + (uint32_t)(b0 * COUT), d2 = dbase;
                const uint64_t a0 = sdesc(rbase + (uint32_t)((i % C::NS) * C::SLOT_BYTES + q * RW * 16), C::CHUNK, 128);
                // B of rows dh0 .. and of the rows after the wrap: same tiles, later start rows
                const uint64_t bA = sdesc(wbase + (uint32_t)(dh0 * COUT * 16), 3 * COUT * 16, 128);
                const uint64_t bB = sdesc(wbase + (uint32_t)((dh0 + n1) * COUT * 16), 3 * COUT * 16, 128);
                // The row's MMAs as one branch-free run, then those of the rows after the wrap as a
                // second: a conditional MMA between consecutive ones halved the issue rate (measured).
                // Each accumulator block still receives its contributions in the same order.
#pragma unroll
                for (int dt = 0; dt < 3; ++dt)
#pragma unroll
                    for (int dw = 0; dw < 3; ++dw)
#pragma unroll
                        for (int ks = 0; ks < C::KS; ++ks) {
                            const uint64_t ad = a0 + (uint64_t)((2 * ks * C::CHUNK + dt * RW * 16 + dw * 16) >> 4);
                            const uint64_t toff = (uint64_t)((((dt * 3 + dw) * C::KS + ks) * TILE) >> 4);
                            umma(d1, ad, bA + toff, id1, 1u);
                        }
                if (n2 > 0) {
#pragma unroll
                    for (int dt = 0; dt < 3; ++dt)
#pragma unroll
                        for (int dw = 0; dw < 3; ++dw)
#pragma unroll
                            for (int ks = 0; ks < C::KS; ++ks) {
                                const uint64_t ad = a0 + (uint64_t)((2 * ks * C::CHUNK + dt * RW * 16 + dw * 16) >> 4);
                                const uint64_t toff = (uint64_t)((((dt * 3 + dw) * C::KS + ks) * TILE) >> 4);
                                umma(d2, ad, bB + toff, id2, 1u);
                            }
                }
                umma_commit(&empty[i % C::NS]);
                if (i >= 2 && i - 2 < nout) umma_commit(&af[blk(i - 2)]);
            }
        }
    } else if ((epi >> 2) < nfr) {   // ---------------- epilogue: 4 warps per output frame
        const int f = epi >> 2;          // output frame t0 + f
        const int qd = warp & 3;         // TMEM lane quadrant of this warp
        const int v = qd * 32 + lane;    // voxel within the tile
        const int w = w0 + v;
        const int t = t0 + f;
        uint64_t* af = accf + f * C::R;
        uint64_t* ae = acce + f * C::R;
        // the bias in registers, read once (the output stores may alias it as far as the compiler
        // knows, which would otherwise reload it for every row)
        float bz[EPI == EPI_RELU ? COUT : 1];
#pragma unroll
        for (int c = 0; c < (int)(sizeof(bz) / sizeof(float)); ++c) bz[c] = EPI == EPI_MASK ? 0.f : a.bias[c];
        for (int j = 0; j < nout; ++j) {
            const int b = blk(j);
            const bool ok = mb_wait(&af[b], (uint32_t)((j / C::R) & 1), a.flags);
            tc_fence_after();
            uint32_t r[COUT];
            const uint32_t taddr = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(f * C::RING + b * COUT);
            tmem_ld<COUT>(taddr, r);
            tmem_ld_wait();
            tmem_zero<COUT>(taddr);      // the block's next row accumulates from zero
            tmem_st_wait();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mb_arrive(&ae[b]);
            if (!ok) break;
            const int h = hs + j;
            if (w >= a.W) continue;
            const int64_t vox = ((int64_t)t * a.H + h) * a.W + w;
            {
                __nv_bfloat162 o[COUT / 2];
                if constexpr (EPI == EPI_RELU) {
#pragma unroll
                    for (int c = 0; c < COUT / 2; ++c) {
                        const float x0 = fmaxf(__uint_as_float(r[2 * c]) + bz[2 * c], 0.f);
                        const float x1 = fmaxf(__uint_as_float(r[2 * c + 1]) + bz[2 * c + 1], 0.f);
                        o[c] = __floats2bfloat162_rn(x0, x1);
                    }
                } else {   // EPI_MASK: dL/dz of the layer below = dL/da * [a > 0]
                    const uint4* mp = reinterpret_cast<const uint4*>(a.mask + vox * COUT);
#pragma unroll
                    for (int c4 = 0; c4 < COUT / 8; ++c4) {
                        const uint4 m4 = mp[c4];
                        const __nv_bfloat162* mm = reinterpret_cast<const __nv_bfloat162*>(&m4);
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float2 mf = __bfloat1622float2(mm[e]);
                            const int c = c4 * 4 + e;
                            o[c] = __floats2bfloat162_rn(mf.x > 0.f ? __uint_as_float(r[2 * c]) : 0.f,
                                                         mf.y > 0.f ? __uint_as_float(r[2 * c + 1]) : 0.f);
                        }
                    }
                }
                uint4* op = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(a.out) + vox * COUT);
#pragma unroll
                for (int c4 = 0; c4 < COUT / 8; ++c4) op[c4] = reinterpret_cast<const uint4*>(o)[c4];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (*reinterpret_cast<volatile int*>(a.flags) & kFlagTimeout) {
        // A bounded wait gave up (here or in another CTA): let this CTA's copies and MMAs still
        // in flight land before its shared memory and TMEM are released.  Each wait is bounded.
        if (warp == 0 && lane == 0) {
            mb_settle(wbar, 0);
            for (int s = 0; s < C::NS && s < issued; ++s) {
                const int last = s + ((issued - 1 - s) / C::NS) * C::NS;
                mb_settle(&full[s], (uint32_t)((last / C::NS) & 1));
            }
        } else if (epi < 0 && lane == 0 && warp - 1 < nfr) {
            umma_commit(&drain[warp - 1]);   // arrives when every MMA this thread issued has completed
            mb_settle(&drain[warp - 1], 0);
        }
        __syncthreads();
    }
    tc_fence_after();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

// -------------------------------------------------------------- last layer (32 -> 1, tcgen05)
// The last layer has one output channel.  Stacking its three h-taps along N as the other layers
// do would compute 16 padded outputs per tap; here the nine (dh, dw) taps of a frame offset
// are the N dimension instead: for input row i (one h), voxel v along w and output frame t,
//   D_{t,i}[v, 3 dh + dw] = sum_{dt, ci} x[t + dt - 1, i, v, ci] W[dt, dh, dw, ci]   (9 -> 16 columns)
// into a ring of TMEM blocks, one 16-column block per input row and output frame.  An input
// frame s of the CTA's slot feeds output frames s - dt + 1 for dt = 0, 1, 2, so one MMA per input
// frame and channel half (M = 128 voxels, K = 16 channels) covers the blocks of all FR output
// frames of a row at once (N = 16 FR): its B operand stacks, for output frame q, the taps of
// frame offset dt = s - q, or zeros where s - q is outside 0..2.  The taps are packed as
// [Z Z Z W2 W1 W0 Z Z Z] (16-row blocks along N, Z zero), so that the B of slot frame s is the FR
// blocks from block 5 - s on, and the first MMA of a row (slot frame 0) also clears the blocks
// of the other output frames.  Per input row that is 2 (FR + 2) MMAs instead of 6 FR.  Output row
// j (input rows j, j+1, j+2 = h - 1, h, h + 1) then takes
// z[w] = b + sum_{dh, dw} D_{j+dh}[w + dw - 1, 3 dh + dw]: the epilogue sums the three rows in
// each lane, exchanges the three dw sums through shared memory (a lane's neighbours along w may
// sit in another warp) and adds them.  M = 128 voxels cover 126 outputs and their w halo, so the
// tiles are 126 voxels wide.
constexpr int LT_W = MT - 2;                 // outputs per tile along w
constexpr int LT_NBLK = 9;                   // 16-row tap blocks along N: Z Z Z W2 W1 W0 Z Z Z
constexpr int LT_CH = LT_NBLK * 16 * 16;     // one 8-channel chunk of the taps (2304 bytes)
constexpr int LT_BBYTES = 2 * 2 * LT_CH;     // [ks][chunk][9 x 16 taps][8 channels] bf16

struct LastArgs {
    int T, H, W, HR;
    const __nv_bfloat16* wtap;   // packed taps, LT_BBYTES bytes
    const float* bias;           // [1]
    float* z;                    // [T][H][W]
    float* x0;                   // softplus(z), [T][H][W]
    int* flags;
};

// FR output frames per CTA from input slots of FR + 2 frames (each output frame reads three of
// them): the input bytes copied per output voxel fall from 3 x 64 to (FR + 2) / FR x 64.  The
// ring holds R rows; a row's FR blocks (one per output frame) are adjacent, and each output
// frame has its own four epilogue warps.  One frame per CTA (a ring of 16 blocks in 256 columns,
// two CTAs per SM) serves volumes too small for the four-frame grid.
template <int FR>
struct LastCfg {
    static constexpr int NF = FR + 2;                     // frames per input slot
    static constexpr int CHUNK_DATA = NF * RW * 16;       // one 8-channel chunk of NF frames
    static constexpr int CHUNK = (CHUNK_DATA + 127) / 128 * 128;
    static constexpr int SLOT = 4 * CHUNK;                // one input row: 4 chunks of 8 channels
    static constexpr int CTAS = FR == 1 ? 2 : 1;          // CTAs per SM
    static constexpr int COLS = 512 / CTAS;               // TMEM columns of the CTA
    static constexpr int R = COLS / (16 * FR);            // rows in the ring (FR blocks each)
    static constexpr int NS = NSLOT;                      // input-row slots
    static constexpr int NTHR = 32 * (2 + 4 * FR);        // producer, issuer, 4 epilogue warps per frame
    // per frame: the dw sums of two rows and each epilogue warp's wait status (double buffer)
    static constexpr int XS1 = 2 * 3 * 128 * 4 + 2 * 4 * 4;
    static constexpr int XS = FR * XS1;
    static constexpr int NB = 2 * NS + 2 * FR * R + 2;    // full, empty, accf[FR][R], acce[FR][R], wbar, drain
    static constexpr int SMEM = LT_BBYTES + NS * SLOT + XS + NB * 8 + 16 + 128;
    static_assert(R >= 4, "accumulator ring");
    static_assert(FR <= 4, "named barriers 1..FR");
    static_assert(SMEM * CTAS <= 227 * 1024, "shared memory");
};

template <int FR>
__global__ void __launch_bounds__(LastCfg<FR>::NTHR, LastCfg<FR>::CTAS)
conv_last_tc(const __grid_constant__ CUtensorMap xin, LastArgs a) {
    using L = LastCfg<FR>;
    extern __shared__ __align__(128) unsigned char sm_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)sm_raw + 127) & ~(uintptr_t)127);
    unsigned char* wsm = sm;
    unsigned char* ring = sm + LT_BBYTES;
    unsigned char* xs0 = ring + L::NS * L::SLOT;            // [FR][XS1]
    uint64_t* bar = reinterpret_cast<uint64_t*>(xs0 + L::XS);
    uint64_t* full = bar;
    uint64_t* empty = bar + L::NS;
    uint64_t* accf = bar + 2 * L::NS;            // [FR][R]: input row's D complete
    uint64_t* acce = accf + FR * L::R;           // [FR][R]: block read by every output row that needs it
    uint64_t* wbar = acce + FR * L::R;
    uint64_t* drain = wbar + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + L::NB);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int HR = a.HR;
    const int nws = (a.W + LT_W - 1) / LT_W, nhr = (a.H + HR - 1) / HR;
    int item = blockIdx.x;
    const int hr = item % nhr;
    item /= nhr;
    const int ws = item % nws;
    const int t0 = (item / nws) * FR;
    const int nfr = min(FR, a.T - t0);           // output frames of this CTA
    const int w0 = ws * LT_W, hs = hr * HR, he = min(a.H, hs + HR);
    const int nout = he - hs, nin = nout + 2;

    if (threadIdx.x == 0) {
        for (int i = 0; i < L::NS; ++i) {
            mb_init(&full[i], 1);
            mb_init(&empty[i], 1);
        }
        for (int i = 0; i < FR * L::R; ++i) {
            mb_init(&accf[i], 1);
            mb_init(&acce[i], 4);
        }
        mb_init(wbar, 1);
        mb_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(L::COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    int issued = 0;
    if (warp == 0) {
        if (lane == 0) {   // ---------------- producer: the taps, then the input rows
            mb_expect(wbar, LT_BBYTES);
            bulk_g2s(wsm, a.wtap, LT_BBYTES, wbar);
            for (int i = 0; i < nin; ++i) {
                const int s = i % L::NS;
                if (i >= L::NS && !mb_wait(&empty[s], (uint32_t)((i / L::NS - 1) & 1), a.flags)) break;
                issued = i + 1;
                mb_expect(&full[s], 4 * L::CHUNK_DATA);
                unsigned char* dst = ring + s * L::SLOT;
                for (int k = 0; k < 4; ++k) tma4(dst + k * L::CHUNK, &xin, &full[s], 8 * k, w0 - 1, hs - 1 + i, t0 - 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {   // ---------------- MMA issuer: 2 (FR + 2) MMAs per input row
            bool ok = mb_wait(wbar, 0, a.flags);
            const uint32_t wbase = su32(wsm), rbase = su32(ring);
            constexpr uint32_t ID = idesc_bf16(16 * FR);
            for (int i = 0; ok && i < nin; ++i) {
                ok = mb_wait(&full[i % L::NS], (uint32_t)((i / L::NS) & 1), a.flags);
                // the blocks of row i: read back by every output row of row i - R
                if (i >= L::R)
                    for (int q = 0; ok && q < nfr; ++q)
                        ok = mb_wait(&acce[q * L::R + i % L::R], (uint32_t)(((i - L::R) / L::R) & 1), a.flags);
                if (!ok) break;
                tc_fence_after();
                const uint64_t a0 = sdesc(rbase + (uint32_t)((i % L::NS) * L::SLOT), L::CHUNK, 128);
                // row i's blocks of all FR output frames (those past the last frame are not read)
                const uint32_t d = tmem + (uint32_t)((i % L::R) * FR * 16);
#pragma unroll
                for (int sf = 0; sf < L::NF; ++sf)   // slot frame t0 - 1 + sf
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        const uint64_t ad = a0 + (uint64_t)((2 * ks * L::CHUNK + sf * RW * 16) >> 4);
                        const uint64_t bd = sdesc(wbase + (uint32_t)(2 * ks * LT_CH + (5 - sf) * 256), LT_CH, 128);
                        umma(d, ad, bd, ID, (sf | ks) ? 1u : 0u);
                    }
                umma_commit(&empty[i % L::NS]);
                for (int q = 0; q < nfr; ++q) umma_commit(&accf[q * L::R + i % L::R]);
            }
        }
    } else if (((warp - 2) >> 2) < nfr) {   // ---------------- epilogue: 4 warps per output frame
        const int g = (warp - 2) >> 2;          // output frame t0 + g
        const int qd = warp & 3;                // TMEM lane quadrant
        const int l = qd * 32 + lane;           // TMEM lane = voxel w0 - 1 + l
        const int t = t0 + g;
        uint64_t* af = accf + g * L::R;
        uint64_t* ae = acce + g * L::R;
        float* xs = reinterpret_cast<float*>(xs0 + g * L::XS1);   // [2][3][128], then [2][4] statuses
        const float b = a.bias[0];
        // Each input row's block is read once: its taps of offset dh go to the running sums of
        // output row r - dh (pj[2]: row r - 2, complete after this row; pj[1]: r - 1; pj[0]: r).
        float pj[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
        bool ok = true;
        for (int r = 0; r < nin; ++r) {
            ok = ok && mb_wait(&af[r % L::R], (uint32_t)((r / L::R) & 1), a.flags);
            tc_fence_after();
            uint32_t v[16];
            tmem_ld<16>(tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(((r % L::R) * FR + g) * 16), v);
            tmem_ld_wait();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mb_arrive(&ae[r % L::R]);   // the block is not read again
#pragma unroll
            for (int dw = 0; dw < 3; ++dw) {
                pj[2][dw] = pj[1][dw] + __uint_as_float(v[6 + dw]);
                pj[1][dw] = pj[0][dw] + __uint_as_float(v[3 + dw]);
                pj[0][dw] = __uint_as_float(v[dw]);
            }
            const int j = r - 2;                 // output row completed by input row r
            if (j < 0) continue;
            float* xb = xs + (j & 1) * 3 * 128;
            int* okb = reinterpret_cast<int*>(xs + 2 * 3 * 128) + (j & 1) * 4;
#pragma unroll
            for (int dw = 0; dw < 3; ++dw) xb[dw * 128 + l] = pj[2][dw];
            if (lane == 0) okb[qd] = ok ? 1 : 0;
            asm volatile("bar.sync %0, 128;" ::"r"(1 + g) : "memory");
            // the four warps leave together if any of their waits gave up
            if (!(okb[0] & okb[1] & okb[2] & okb[3])) break;
            const int h = hs + j, w = w0 + l;
            if (l < LT_W && w < a.W) {
                const float z = b + xb[l] + xb[128 + l + 1] + xb[256 + l + 2];
                const int64_t vox = ((int64_t)t * a.H + h) * a.W + w;
                a.z[vox] = z;
                a.x0[vox] = z > 20.f ? z : log1pf(expf(z));   // softplus
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (*reinterpret_cast<volatile int*>(a.flags) & kFlagTimeout) {
        if (warp == 0 && lane == 0) {
            mb_settle(wbar, 0);
            for (int s = 0; s < L::NS && s < issued; ++s) {
                const int last = s + ((issued - 1 - s) / L::NS) * L::NS;
                mb_settle(&full[s], (uint32_t)((last / L::NS) & 1));
            }
        } else if (warp == 1 && lane == 0) {
            umma_commit(drain);
            mb_settle(drain, 0);
        }
        __syncthreads();
    }
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(L::COLS) : "memory");
}

// Taps of the last layer for conv_last_tc: out[((ks * 2 + chunk) * 9 + blk) * 16 + n][e] =
// W[0][9 dt + 3 dh + dw][16 ks + 8 chunk + e] for blk = 5 - dt (dt = 0, 1, 2) and n = 3 dh + dw < 9,
// zero for n >= 9 and for the blocks 0..2 and 6..8.
__global__ void pack_last_taps(const float* W, __nv_bfloat16* out) {
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < LT_BBYTES / 2; idx += gridDim.x * blockDim.x) {
        int r = idx;
        const int e = r % 8; r /= 8;
        const int n = r % 16; r /= 16;
        const int blk = r % LT_NBLK; r /= LT_NBLK;
        const int ch = r % 2; r /= 2;
        const int ks = r;
        const int dt = 5 - blk;
        float v = 0.f;
        if (n < 9 && dt >= 0 && dt <= 2) v = W[(9 * dt + n) * 32 + ks * 16 + ch * 8 + e];
        out[idx] = __float2bfloat16_rn(v);
    }
}

// ------------------------------------------------------------------ weight gradient (tcgen05)
// dW[co][tap][ci] = sum_v dz[v][co] x[v + tap][ci] and db[co] = sum_v dz[v][co] as GEMMs with the
// voxels as the reduction dimension K.  A work unit is (x frame t, dz row h, a 128-voxel segment
// along w).  With the x frame fixed, the taps (dt, dh, dw) of one unit form three products, one
// per dw:
//   D_dw[(j, ci), (s, co)] += sum_k x[t, h - 1 + j, w0 + k + dw - 1, ci] * dz[t - 1 + s, h, w0 + k, co]
// for j = dh + 1 in 0..2 and s = 1 - dt in 0..2: M = 128 stacks four 32-channel row blocks of x
// (the fourth is a constant 1, so its rows of D sum dz: the bias gradient), N stacks the three dz
// frames (3 x 32 channels; 3 x 16 for the last layer's one channel padded to 16).  Both operands
// are read in the MN-major layout straight from the TMA copies of the channels-last activations:
// [block][8-channel chunk][voxels][8 channels], where a core matrix is 8 voxels (K) x 8 channels
// (16 bytes) and a shift by one voxel along w is a 16-byte offset of the descriptor's start.  In
// the descriptor of this no-swizzle MN-major layout the leading-dimension offset is the step
// between groups of 8 voxels along K (128 bytes) and the stride-dimension offset the step between
// 8-channel chunks along M or N (measured: the other assignment gives wrong sums).
// Every unit of a CTA accumulates into the same TMEM columns; at the end the CTA writes its
// partial sums to a scratch slice and a second kernel adds the slices in a fixed order.
constexpr int WG_XV = MT + 2;                              // x voxels per row (w halo 1)
constexpr int WG_CHA = (WG_XV * 16 + 127) / 128 * 128;     // A chunk stride (2176 B)
constexpr int WG_CHB = MT * 16;                            // B chunk stride (2048 B)
constexpr int WG_A_BYTES = 16 * WG_CHA;                    // 4 row blocks x 4 chunks
#ifndef SFSEG_NET_WG_NS
#define SFSEG_NET_WG_NS 3
#endif
constexpr int WG_NS = SFSEG_NET_WG_NS;   // stages (2 measured 4 % slower; 4 exceed the shared memory)

template <int NCI, int NCO>
struct WgCfg {
    static constexpr int N = 3 * NCO * 8;                  // 96 or 48
    static constexpr int B_BYTES = 3 * NCO * WG_CHB;
    static constexpr int STAGE = WG_A_BYTES + B_BYTES;
    static constexpr int TMEM_COLS = 3 * N <= 256 ? 256 : 512;
    // (the barriers sit after the stages; 8 KB more keep every descriptor offset inside the
    // allocation whatever the operand reach)
    static constexpr int SMEM = WG_NS * STAGE + (2 * WG_NS + 2) * 8 + 16 + 128 + 8192;
    static constexpr int PART = 3 * N * 128;               // floats of one CTA's partial sums
};

struct WgArgs {
    int T, H, W, nws, units, per;   // per: units of each CTA (the last may have fewer, none has 0)
    float* part;     // [gridDim.x][3 dw][N][128 m]
    int* flags;
};

// Instruction descriptor, kind::f16: bf16 A and B, both MN-major, fp32 D, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_bf16_mn(int n) { return idesc_bf16(n) | (1u << 15) | (1u << 16); }

template <int NCI, int NCO>
__global__ void __launch_bounds__(NTHR, 1)
wgrad_tc(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap dzmap, WgArgs a) {
    using C = WgCfg<NCI, NCO>;
    extern __shared__ __align__(128) unsigned char sm_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)sm_raw + 127) & ~(uintptr_t)127);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + WG_NS * C::STAGE);
    uint64_t* full = bar;               // [WG_NS]
    uint64_t* empty = bar + WG_NS;      // [WG_NS]
    uint64_t* done = bar + 2 * WG_NS;   // every MMA of the CTA has completed
    uint64_t* drain = done + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 2 * WG_NS + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // this CTA's contiguous range of units
    const int u0 = blockIdx.x * a.per, u1 = min(a.units, u0 + a.per);
    const int nu = max(u1 - u0, 0);

    // the constant row block (ones) of every stage, and the channel chunks an input with fewer
    // than 32 channels (NCI < 4) does not fill (zeros); no copy ever writes either
    for (int i = threadIdx.x; i < WG_NS * 16 * WG_CHA / 16; i += blockDim.x) {
        const int st = i / (16 * WG_CHA / 16), r = i % (16 * WG_CHA / 16);
        const int blk = r / (WG_CHA / 16);          // (j, c) block: j = blk / 4, c = blk % 4
        uint4* p = reinterpret_cast<uint4*>(sm + st * C::STAGE) + r;
        if (blk >= 12) *p = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);   // bf16 1.0 x 8
        else if (blk % 4 >= NCI) *p = make_uint4(0u, 0u, 0u, 0u);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
        for (int i = 0; i < WG_NS; ++i) {
            mb_init(&full[i], 1);
            mb_init(&empty[i], 1);
        }
        mb_init(done, 1);
        mb_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(C::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    int issued = 0;
    bool mma_ok = true;
    if (warp == 0) {
        if (lane == 0) {   // ---------------- producer
            for (int i = 0; i < nu; ++i) {
                const int s = i % WG_NS;
                if (i >= WG_NS && !mb_wait(&empty[s], (uint32_t)((i / WG_NS - 1) & 1), a.flags)) break;
                issued = i + 1;
                int u = u0 + i;
                const int ws = u % a.nws;
                u /= a.nws;
                const int h = u % a.H, t = u / a.H;
                const int w0 = ws * MT;
                unsigned char* st = sm + s * C::STAGE;
                mb_expect(&full[s], 3u * NCI * (uint32_t)(WG_XV * 16) + 3u * NCO * (uint32_t)WG_CHB);
                for (int j = 0; j < 3; ++j)
                    for (int c = 0; c < NCI; ++c)
                        tma4(st + (j * 4 + c) * WG_CHA, &xmap, &full[s], 8 * c, w0 - 1, h - 1 + j, t);
                for (int f = 0; f < 3; ++f)
                    for (int c = 0; c < NCO; ++c)
                        tma4(st + WG_A_BYTES + (f * NCO + c) * WG_CHB, &dzmap, &full[s], 8 * c, w0, h, t - 1 + f);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {   // ---------------- MMA issuer
            const uint32_t base = su32(sm);
            constexpr uint32_t ID = idesc_bf16_mn(C::N);
            for (int i = 0; i < nu; ++i) {
                const int s = i % WG_NS;
                if (!mb_wait(&full[s], (uint32_t)((i / WG_NS) & 1), a.flags)) {
                    mma_ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t sa = base + (uint32_t)(s * C::STAGE), sb = sa + WG_A_BYTES;
#pragma unroll
                for (int dw = 0; dw < 3; ++dw)
#pragma unroll
                    for (int kk = 0; kk < MT / 16; ++kk) {
                        const uint64_t ad = sdesc(sa + (uint32_t)((kk * 16 + dw) * 16), 128, WG_CHA);
                        const uint64_t bd = sdesc(sb + (uint32_t)(kk * 16 * 16), 128, WG_CHB);
                        umma(tmem + (uint32_t)(dw * C::N), ad, bd, ID, (i > 0 || kk > 0) ? 1u : 0u);
                    }
                umma_commit(&empty[s]);
            }
            umma_commit(done);   // arrives when all of this thread's MMAs have completed
        }
    } else {   // ---------------- epilogue: warps 2..5 write the partial sums
        const int q = warp & 3;
        const bool ok = mb_wait(done, 0, a.flags);
        tc_fence_after();
        if (ok && nu > 0) {
            float* out = a.part + (size_t)blockIdx.x * C::PART;
            const int m = q * 32 + lane;
#pragma unroll 1
            for (int c0 = 0; c0 < 3 * C::N; c0 += 16) {
                uint32_t r[16];
                tmem_ld<16>(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, r);
                tmem_ld_wait();
#pragma unroll
                for (int e = 0; e < 16; ++e) out[(size_t)(c0 + e) * 128 + m] = __uint_as_float(r[e]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (*reinterpret_cast<volatile int*>(a.flags) & kFlagTimeout) {
        // a bounded wait gave up: let the copies and MMAs this CTA issued land before its shared
        // memory and tensor memory are released (each wait bounded)
        if (warp == 0 && lane == 0) {
            for (int s = 0; s < WG_NS && s < issued; ++s) {
                const int last = s + ((issued - 1 - s) / WG_NS) * WG_NS;
                mb_settle(&full[s], (uint32_t)((last / WG_NS) & 1));
            }
        } else if (warp == 1 && lane == 0) {
            umma_commit(drain);
            mb_settle(drain, 0);
        }
        __syncthreads();
    }
    (void)mma_ok;
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS) : "memory");
}

// Sum of the CTAs' partial sums in a fixed order: dW[co][tap][ci] with tap = 9 (dt + 1) +
// 3 (dh + 1) + (dw + 1) from row block j = dh + 1, dz frame s = 1 - dt; db[co] from the constant
// row block (m = 96) of the dz frame s = 1 (the others repeat it).
template <int NCI, int NCO>
__global__ void wgrad_reduce(const float* part, int nparts, int cout, int cin, float* dW, float* db) {
    using C = WgCfg<NCI, NCO>;
    const int total = cout * 27 * cin;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total + cout; idx += gridDim.x * blockDim.x) {
        int n, m, dw;
        if (idx < total) {
            const int ci = idx % cin, tap = (idx / cin) % 27, co = idx / (cin * 27);
            const int dtp = tap / 9, dhp = (tap / 3) % 3;
            dw = tap % 3;
            n = (2 - dtp) * NCO * 8 + co;
            m = dhp * 32 + ci;
        } else {
            const int co = idx - total;
            dw = 1;
            n = NCO * 8 + co;
            m = 96;
        }
        double acc = 0.0;
        for (int p = 0; p < nparts; ++p) acc += (double)part[(size_t)p * C::PART + ((size_t)dw * C::N + n) * 128 + m];
        if (idx < total) dW[idx] = (float)acc;
        else db[idx - total] = (float)acc;
    }
}

// ------------------------------------------------------------------------ small kernels
// Caller's channels [C][T][H][W] (float or bf16), plus an optional float [T][H][W] channel after
// them -> bf16 [T][H][W][16], remaining channels zero.
template <typename TIn>
__global__ void to_channels_last(const TIn* f, int C, const float* extra, int64_t N, __nv_bfloat16* out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        __nv_bfloat16 v[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            float a = 0.f;
            if (c < C) a = ldf(f + (int64_t)c * N + i);
            else if (c == C && extra) a = extra[i];
            v[c] = __float2bfloat16_rn(a);
        }
        uint4* o = reinterpret_cast<uint4*>(out + i * 16);
        o[0] = reinterpret_cast<const uint4*>(v)[0];
        o[1] = reinterpret_cast<const uint4*>(v)[1];
    }
}

// Pack fp32 weights W[co][27][ci] (co < cout, ci < cin) into the B-operand layout
// [dt][dw][ks][chunk(2)][dh][COUTP][8] bf16 with zero padding to COUTP x CINP (tap =
// 9 dt + 3 dh + dw): each (dt, dw, ks) tile stacks the three dh blocks along N; `flip` packs
// the data-gradient kernel instead: W'[ci][tap][co] = W[co][26 - tap][ci].
__global__ void pack_weights(const float* W, int cout, int cin, int COUTP, int CINP, int flip, __nv_bfloat16* out) {
    const int KS = CINP / 16;
    const int total = 27 * KS * 2 * COUTP * 8;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        int r = idx;
        const int e = r % 8; r /= 8;
        const int n = r % COUTP; r /= COUTP;
        const int dh = r % 3; r /= 3;
        const int ch = r % 2; r /= 2;
        const int ks = r % KS; r /= KS;
        const int dw = r % 3; r /= 3;
        const int dt = r;
        const int tap = 9 * dt + 3 * dh + dw;
        const int k = ks * 16 + ch * 8 + e;     // input-channel index of the packed conv
        float v = 0.f;
        if (!flip) {
            if (n < cout && k < cin) v = W[((int64_t)n * 27 + tap) * cin + k];
        } else {   // packed conv: out channel n = ci of W, in channel k = co of W
            if (n < cin && k < cout) v = W[((int64_t)k * 27 + (26 - tap)) * cin + n];
        }
        out[idx] = __float2bfloat16_rn(v);
    }
}

// Cosine-loss pieces: sums of x*g, x*x, g*g (FP64 via block sums).
__global__ void cos_sums(const float* x, const float* g, int64_t n, double* acc) {
    float a = 0.f, b = 0.f, c = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        a += x[i] * g[i];
        b += x[i] * x[i];
        c += g[i] * g[i];
    }
    double s = block_sum((double)a);
    if (threadIdx.x == 0) atomicAdd(acc, s);
    s = block_sum((double)b);
    if (threadIdx.x == 0) atomicAdd(acc + 1, s);
    s = block_sum((double)c);
    if (threadIdx.x == 0) atomicAdd(acc + 2, s);
}

// dL/dz4 for L = 1 - <x,g>/(|x||g|), x = softplus(z4): written as channel 0 of a 16-channel bf16
// tensor (the input of the last layer's data-gradient convolution), other channels zero.
__global__ void cos_grad(const float* x, const float* g, const float* z, int64_t n, const double* acc,
                         __nv_bfloat16* dz16) {
    const double xg = acc[0], xx = acc[1], gg = acc[2];
    const double nx = sqrt(xx), ng = sqrt(gg);
    const float c1 = (float)(1.0 / (nx * ng)), c2 = (float)(xg / (nx * ng) / xx);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float dx = -(g[i] * c1 - x[i] * c2);
        const float sg = 1.f / (1.f + expf(-z[i]));
        __nv_bfloat16 v[16];
        v[0] = __float2bfloat16_rn(dx * sg);
#pragma unroll
        for (int c = 1; c < 16; ++c) v[c] = __float2bfloat16_rn(0.f);
        uint4* o = reinterpret_cast<uint4*>(dz16 + i * 16);
        o[0] = reinterpret_cast<const uint4*>(v)[0];
        o[1] = reinterpret_cast<const uint4*>(v)[1];
    }
}

// AdamW (decoupled weight decay) on fp32 parameters.
__global__ void adamw_kernel(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2,
                             float eps, float wd, float bc1, float bc2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * ((mi / bc1) / (sqrtf(vi / bc2) + eps) + wd * p[i]);
    }
}

}  // namespace net
}  // namespace sfseg

// ================================================================================ host side
using namespace sfseg;
using namespace sfseg::net;

namespace {

typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                             const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode() {
    static EncodeFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeFn)p;
    }
    return fn;
}

// 4D map over a channels-last bf16 activation [T][H][W][C]; box = 8 channels x 130 voxels x
// 1 row x 3 frames (one A chunk of one input row).
bool act_map(CUtensorMap* m, const void* base, int C, int T, int H, int W, int frames = 3) {
    EncodeFn fn = encode();
    if (!fn) return false;
    cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)T};
    cuuint64_t str[3] = {(cuuint64_t)C * 2, (cuuint64_t)C * 2 * W, (cuuint64_t)C * 2 * W * H};
    cuuint32_t box[4] = {8, (cuuint32_t)RW, 1, (cuuint32_t)frames};
    cuuint32_t es[4] = {1, 1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, str, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 4D map over a channels-last bf16 activation [T][H][W][C] with a box of 8 channels x bw voxels
// x 1 row x 1 frame (one chunk of one row).
bool row_map(CUtensorMap* m, const void* base, int C, int T, int H, int W, int bw) {
    EncodeFn fn = encode();
    if (!fn) return false;
    cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)T};
    cuuint64_t str[3] = {(cuuint64_t)C * 2, (cuuint64_t)C * 2 * W, (cuuint64_t)C * 2 * W * H};
    cuuint32_t box[4] = {8, (cuuint32_t)bw, 1, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, str, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int blocks_for(int64_t n, int per = 256) {
    int64_t b = (n + per - 1) / per;
    const int cap = 16 * num_sms();
    return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

}  // namespace

struct sfseg_net {
    int cin = 8;
    int64_t off[8] = {0};     // W1 b1 W2 b2 W3 b3 W4 b4
    int64_t np = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    int64_t step = 0;
    bool packed = false;
    __nv_bfloat16* wf[4] = {nullptr, nullptr, nullptr, nullptr};   // forward packs
    __nv_bfloat16* wb[4] = {nullptr, nullptr, nullptr, nullptr};   // data-gradient packs (layers 2..4)
    int64_t cap = 0;
    __nv_bfloat16 *x16 = nullptr, *a1 = nullptr, *a2 = nullptr, *a3 = nullptr, *dz16 = nullptr, *dza = nullptr,
                  *dzb = nullptr;
    float *z4 = nullptr, *x0 = nullptr;
    float* wg_part = nullptr;   // per-CTA partial sums of the weight-gradient kernel
    double* acc = nullptr;
    int* flags = nullptr;
    bool have_fwd = false;
};

namespace {

int nfail(int code, const std::string& m) { return set_last_error(code, m.c_str()); }

#define NET_CUDA(call)                                                                                  \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess)                                                                          \
            return nfail(e_ == cudaErrorMemoryAllocation ? SFSEG_ERR_OOM : SFSEG_ERR_CUDA,              \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                           \
    } while (0)

const int kCout[4] = {32, 32, 32, 1};

int layer_cin(const sfseg_net* n, int l) { return l == 0 ? n->cin : 32; }

// Forward buffers (x16, a1, a2, z4, x0) always; a3 and the gradient buffers only for training.
// Inference writes layer 3's output over layer 1's (layer 3 reads a2, so a1 is free by then):
// 168 bytes per voxel instead of 392.
int ensure_ws(sfseg_net* n, int64_t N, bool train) {
    if (n->cap < N) {
        cudaFree(n->x16); cudaFree(n->a1); cudaFree(n->a2); cudaFree(n->a3);
        cudaFree(n->dz16); cudaFree(n->dza); cudaFree(n->dzb); cudaFree(n->z4); cudaFree(n->x0);
        n->x16 = n->a1 = n->a2 = n->a3 = n->dz16 = n->dza = n->dzb = nullptr;
        n->z4 = n->x0 = nullptr;
        n->cap = 0;
        NET_CUDA(cudaMalloc(&n->x16, N * 16 * 2));
        NET_CUDA(cudaMalloc(&n->a1, N * 32 * 2));
        NET_CUDA(cudaMalloc(&n->a2, N * 32 * 2));
        NET_CUDA(cudaMalloc(&n->z4, N * 4));
        NET_CUDA(cudaMalloc(&n->x0, N * 4));
        n->cap = N;
    }
    if (train && !n->dz16) {
        NET_CUDA(cudaMalloc(&n->a3, n->cap * 32 * 2));
        NET_CUDA(cudaMalloc(&n->dz16, n->cap * 16 * 2));
        NET_CUDA(cudaMalloc(&n->dza, n->cap * 32 * 2));
        NET_CUDA(cudaMalloc(&n->dzb, n->cap * 32 * 2));
    }
    return SFSEG_OK;
}

// The launch shape of the calling thread's most recent launch of each convolution kernel
// (0: conv3d_tc, 1: conv_last_tc), for sfseg_net_launch_shape.
struct LaunchShape {
    int frames, rows, ctas;
};
thread_local LaunchShape last_shape[2] = {{0, 0, 0}, {0, 0, 0}};

template <int CIN, int COUT, int EPI, int FR>
int launch_conv(const void* in, int T, int H, int W, const ConvArgs& a, int items, cudaStream_t s) {
    using Cf = ConvCfg<CIN, COUT, FR>;
    CUtensorMap m;
    if (!act_map(&m, in, CIN, T, H, W, Cf::NF)) return nfail(SFSEG_ERR_CUDA, "tensor map encoding failed");
    auto k = conv3d_tc<CIN, COUT, EPI, FR>;
    static unsigned long long attr_set = 0;   // devices on which the attribute is set
    if (!(attr_set & device_bit())) {
        NET_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, Cf::SMEM));
        attr_set |= device_bit();
    }
    k<<<items, Cf::NTHR, Cf::SMEM, s>>>(m, a);
    count_launches(1);
    NET_CUDA(cudaGetLastError());
    last_shape[0] = {FR, a.HR, items};
    return SFSEG_OK;
}

// Three output frames per CTA when that grid still gives 4 waves at some tile height, else two,
// else one;
// then the tallest tile of 64, 32, 16 output rows that gives 4 waves (taller tiles load fewer
// halo rows and amortise each CTA's weight copy and TMEM set-up).
template <int CIN, int COUT, int EPI>
int run_conv(const void* in, int T, int H, int W, const __nv_bfloat16* wpack, const float* bias, void* out,
             const __nv_bfloat16* mask, int* flags, cudaStream_t s) {
    ConvArgs a;
    a.T = T; a.H = H; a.W = W;
    a.wpack = wpack; a.bias = bias; a.out = out; a.mask = mask; a.flags = flags;
    const int nws = (W + MT - 1) / MT;
    int fr = 1, items = 0;
    a.HR = kHrChoices[2];
    for (int f : {3, 2, 1}) {
        bool found = false;
        for (int hr : kHrChoices) {
            const int n = (T + f - 1) / f * nws * ((H + hr - 1) / hr);
            if (n >= 4 * num_sms()) {
                fr = f, a.HR = hr, items = n, found = true;
                break;
            }
        }
        if (found) break;
    }
    if (items == 0) items = T * nws * ((H + a.HR - 1) / a.HR);   // small volume: one frame, 16 rows
    if (fr == 3) return launch_conv<CIN, COUT, EPI, 3>(in, T, H, W, a, items, s);
    return fr == 2 ? launch_conv<CIN, COUT, EPI, 2>(in, T, H, W, a, items, s)
                   : launch_conv<CIN, COUT, EPI, 1>(in, T, H, W, a, items, s);
}

template <int FR>
int launch_last(const __nv_bfloat16* in, int T, int H, int W, const LastArgs& a, int items, cudaStream_t s) {
    using L = LastCfg<FR>;
    CUtensorMap m;
    if (!act_map(&m, in, 32, T, H, W, L::NF)) return nfail(SFSEG_ERR_CUDA, "tensor map encoding failed");
    static unsigned long long attr_set = 0;   // devices on which the attribute is set
    if (!(attr_set & device_bit())) {
        NET_CUDA(cudaFuncSetAttribute(conv_last_tc<FR>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM));
        attr_set |= device_bit();
    }
    conv_last_tc<FR><<<items, L::NTHR, L::SMEM, s>>>(m, a);
    count_launches(1);
    NET_CUDA(cudaGetLastError());
    last_shape[1] = {FR, a.HR, items};
    return SFSEG_OK;
}

// The last layer (32 -> 1) on its own kernel, 126-voxel tiles along w (conv_last_tc): four output
// frames per CTA when that grid gives 4 waves (one CTA per SM) at some tile height, else one
// (two CTAs per SM, 4 waves where the volume allows).
int run_last(const __nv_bfloat16* in, int T, int H, int W, const __nv_bfloat16* wtap, const float* bias, float* z,
             float* x0, int* flags, cudaStream_t s) {
    LastArgs a;
    a.T = T; a.H = H; a.W = W;
    a.wtap = wtap; a.bias = bias; a.z = z; a.x0 = x0; a.flags = flags;
    const int nws = (W + LT_W - 1) / LT_W;
    for (int hr : kHrChoices) {
        const int n = (T + 3) / 4 * nws * ((H + hr - 1) / hr);
        if (n >= 4 * num_sms()) {
            a.HR = hr;
            return launch_last<4>(in, T, H, W, a, n, s);
        }
    }
    int items = 0;
    for (int hr : kHrChoices) {
        a.HR = hr;
        items = T * nws * ((H + hr - 1) / hr);
        if (items >= 8 * num_sms()) break;
    }
    return launch_last<1>(in, T, H, W, a, items, s);
}

int pack_all(sfseg_net* n, cudaStream_t s) {
    if (n->packed) return SFSEG_OK;
    const int cinp[4] = {16, 32, 32, 32}, coutp[4] = {32, 32, 32, 16};
    for (int l = 0; l < 4; ++l) {
        if (l == 3) {   // the last layer's forward taps in conv_last_tc's layout
            pack_last_taps<<<(LT_BBYTES / 2 + 255) / 256, 256, 0, s>>>(n->p + n->off[6], n->wf[3]);
        } else {
            const int total = 27 * (cinp[l] / 16) * 2 * coutp[l] * 8;
            pack_weights<<<(total + 255) / 256, 256, 0, s>>>(n->p + n->off[2 * l], kCout[l], layer_cin(n, l),
                                                             coutp[l], cinp[l], 0, n->wf[l]);
        }
        count_launches(1);
        if (l > 0) {   // data gradient of layer l: input = dz of its output (COUT_l channels, padded)
            const int ci2 = l == 3 ? 16 : 32;
            const int tot2 = 27 * (ci2 / 16) * 2 * 32 * 8;
            pack_weights<<<(tot2 + 255) / 256, 256, 0, s>>>(n->p + n->off[2 * l], kCout[l], 32, 32, ci2, 1, n->wb[l]);
            count_launches(1);
        }
    }
    NET_CUDA(cudaGetLastError());
    n->packed = true;
    return SFSEG_OK;
}

int check_flags(sfseg_net* n, cudaStream_t s) {
    int fl = 0;
    NET_CUDA(cudaMemcpyAsync(&fl, n->flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    NET_CUDA(cudaStreamSynchronize(s));
    if (fl) {
        NET_CUDA(cudaMemsetAsync(n->flags, 0, sizeof(int), s));
        return nfail(SFSEG_ERR_TIMEOUT, "a bounded wait inside the convolution kernel gave up");
    }
    return SFSEG_OK;
}

int net_forward(sfseg_net* n, const void* feats, int dtype, int C, const float* extra, int T, int H, int W, bool train,
                cudaStream_t s) {
    const int64_t N = (int64_t)T * H * W;
    if (int rc = ensure_ws(n, N, train)) return rc;
    __nv_bfloat16* a3 = train ? n->a3 : n->a1;   // inference: layer 3 overwrites layer 1's output
    if (int rc = pack_all(n, s)) return rc;
    if (dtype == SFSEG_F32)
        to_channels_last<float><<<blocks_for(N), 256, 0, s>>>((const float*)feats, C, extra, N, n->x16);
    else
        to_channels_last<__nv_bfloat16><<<blocks_for(N), 256, 0, s>>>((const __nv_bfloat16*)feats, C, extra, N,
                                                                       n->x16);
    count_launches(1);
    if (int rc = run_conv<16, 32, EPI_RELU>(n->x16, T, H, W, n->wf[0], n->p + n->off[1], n->a1, nullptr,
                                            n->flags, s))
        return rc;
    if (int rc = run_conv<32, 32, EPI_RELU>(n->a1, T, H, W, n->wf[1], n->p + n->off[3], n->a2, nullptr,
                                            n->flags, s))
        return rc;
    if (int rc = run_conv<32, 32, EPI_RELU>(n->a2, T, H, W, n->wf[2], n->p + n->off[5], a3, nullptr,
                                            n->flags, s))
        return rc;
    if (int rc = run_last(a3, T, H, W, n->wf[3], n->p + n->off[7], n->z4, n->x0, n->flags, s))
        return rc;
    n->have_fwd = true;
    return SFSEG_OK;
}

template <int NCI, int NCO>
int run_wgrad(sfseg_net* n, int cout, int cin, const __nv_bfloat16* dz, const __nv_bfloat16* x, int T, int H, int W,
              float* dW, float* db, cudaStream_t s) {
    using Cf = WgCfg<NCI, NCO>;
    CUtensorMap xm, dm;
    if (!row_map(&xm, x, NCI * 8, T, H, W, WG_XV) || !row_map(&dm, dz, NCO * 8, T, H, W, MT))
        return nfail(SFSEG_ERR_CUDA, "tensor map encoding failed");
    if (!n->wg_part) NET_CUDA(cudaMalloc(&n->wg_part, (size_t)num_sms() * WgCfg<4, 4>::PART * sizeof(float)));
    auto k = wgrad_tc<NCI, NCO>;
    static unsigned long long attr_set = 0;   // devices on which the attribute is set
    if (!(attr_set & device_bit())) {
        NET_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, Cf::SMEM));
        attr_set |= device_bit();
    }
    WgArgs a;
    a.T = T; a.H = H; a.W = W;
    a.nws = (W + MT - 1) / MT;
    a.units = T * H * a.nws;
    a.part = n->wg_part;
    a.flags = n->flags;
    a.per = (a.units + num_sms() - 1) / num_sms();
    const int grid = (a.units + a.per - 1) / a.per;   // every CTA gets at least one unit
    k<<<grid, NTHR, Cf::SMEM, s>>>(xm, dm, a);
    wgrad_reduce<NCI, NCO><<<(cout * 27 * cin + cout + 255) / 256, 256, 0, s>>>(n->wg_part, grid, cout, cin, dW, db);
    count_launches(2);
    NET_CUDA(cudaGetLastError());
    return SFSEG_OK;
}

// dW (float32 [cout][27][cin], overwritten) and db (float32 [cout], overwritten) of layer l from
// dz (bf16 [N][dzc]) and the layer's input x (bf16 [N][xc]), on the tensor cores.
int wgrad_into(sfseg_net* n, int l, int cin, const __nv_bfloat16* dz, int dzc, const __nv_bfloat16* x, int xc, int T,
               int H, int W, float* dW, float* db, cudaStream_t s) {
    if (xc == 16 && dzc == 32) return run_wgrad<2, 4>(n, kCout[l], cin, dz, x, T, H, W, dW, db, s);
    if (xc == 32 && dzc == 32) return run_wgrad<4, 4>(n, kCout[l], cin, dz, x, T, H, W, dW, db, s);
    if (xc == 32 && dzc == 16) return run_wgrad<4, 2>(n, kCout[l], cin, dz, x, T, H, W, dW, db, s);
    return nfail(SFSEG_ERR_UNSUPPORTED, "weight gradient: unsupported channel counts");
}

int wgrad(sfseg_net* n, int l, const __nv_bfloat16* dz, int dzc, const __nv_bfloat16* x, int xc, int T, int H, int W,
          cudaStream_t s) {
    return wgrad_into(n, l, layer_cin(n, l), dz, dzc, x, xc, T, H, W, n->g + n->off[2 * l], n->g + n->off[2 * l + 1],
                      s);
}

uint64_t splitmix(uint64_t& x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int check_vol(int C, int T, int H, int W, const void* feats) {
    if (!feats) return nfail(SFSEG_ERR_INVALID_ARG, "null features");
    if (C < 1 || C > 16) return nfail(SFSEG_ERR_INVALID_ARG, "the network takes 1..16 channels");
    if (T < 1 || H < 1 || W < 1) return nfail(SFSEG_ERR_SHAPE, "empty volume");
    if ((int64_t)T * H * W >= (int64_t(1) << 31)) return nfail(SFSEG_ERR_SHAPE, "volume too large");
    return SFSEG_OK;
}

}  // namespace

extern "C" {

int sfseg_net_create(int c_in, uint64_t seed, sfseg_net** out) {
    if (!out) return nfail(SFSEG_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    if (c_in < 1 || c_in > 16) return nfail(SFSEG_ERR_INVALID_ARG, "c_in must be in [1, 16]");
    sfseg_net* n = new sfseg_net();
    n->cin = c_in;
    int64_t o = 0;
    for (int l = 0; l < 4; ++l) {
        n->off[2 * l] = o;
        o += (int64_t)kCout[l] * 27 * layer_cin(n, l);
        n->off[2 * l + 1] = o;
        o += kCout[l];
    }
    n->np = o;
    // He-normal weights (Box-Muller on a splitmix64 stream), zero biases.
    std::vector<float> h((size_t)o, 0.f);
    uint64_t st = seed;
    for (int l = 0; l < 4; ++l) {
        const double sd = std::sqrt(2.0 / (27.0 * layer_cin(n, l)));
        for (int64_t i = n->off[2 * l]; i < n->off[2 * l + 1]; ++i) {
            const double u1 = ((splitmix(st) >> 11) + 1.0) / 9007199254740993.0;
            const double u2 = (splitmix(st) >> 11) / 9007199254740992.0;
            h[(size_t)i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
        }
    }
    const int cinp[4] = {16, 32, 32, 32}, coutp[4] = {32, 32, 32, 16};
    cudaError_t e = cudaSuccess;
    auto al = [&](void** p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes); };
    al((void**)&n->p, o * 4);
    al((void**)&n->g, o * 4);
    al((void**)&n->m, o * 4);
    al((void**)&n->v, o * 4);
    for (int l = 0; l < 4; ++l) al((void**)&n->wf[l], (size_t)27 * (cinp[l] / 16) * 2 * coutp[l] * 8 * 2);
    for (int l = 1; l < 4; ++l) al((void**)&n->wb[l], (size_t)27 * ((l == 3 ? 16 : 32) / 16) * 2 * 32 * 8 * 2);
    al((void**)&n->acc, 8 * sizeof(double));
    al((void**)&n->flags, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(n->p, h.data(), o * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(n->m, 0, o * 4);
    if (e == cudaSuccess) e = cudaMemset(n->v, 0, o * 4);
    if (e == cudaSuccess) e = cudaMemset(n->flags, 0, sizeof(int));
    if (e != cudaSuccess) {
        sfseg_net_destroy(n);
        return nfail(e == cudaErrorMemoryAllocation ? SFSEG_ERR_OOM : SFSEG_ERR_CUDA,
                     std::string("sfseg_net_create: ") + cudaGetErrorString(e));
    }
    *out = n;
    return SFSEG_OK;
}

int sfseg_net_destroy(sfseg_net* n) {
    if (!n) return SFSEG_OK;
    cudaDeviceSynchronize();
    cudaFree(n->p); cudaFree(n->g); cudaFree(n->m); cudaFree(n->v);
    for (int l = 0; l < 4; ++l) { cudaFree(n->wf[l]); cudaFree(n->wb[l]); }
    cudaFree(n->x16); cudaFree(n->a1); cudaFree(n->a2); cudaFree(n->a3);
    cudaFree(n->dz16); cudaFree(n->dza); cudaFree(n->dzb); cudaFree(n->z4); cudaFree(n->x0);
    cudaFree(n->wg_part); cudaFree(n->acc); cudaFree(n->flags);
    delete n;
    return SFSEG_OK;
}

int sfseg_net_num_params(sfseg_net* n, int64_t* count) {
    if (!n || !count) return nfail(SFSEG_ERR_INVALID_ARG, "null argument");
    *count = n->np;
    return SFSEG_OK;
}

int sfseg_net_get_params(sfseg_net* n, float* host, int64_t count) {
    if (!n || !host) return nfail(SFSEG_ERR_INVALID_ARG, "null argument");
    if (count != n->np) return nfail(SFSEG_ERR_SHAPE, "parameter count mismatch");
    NET_CUDA(cudaMemcpy(host, n->p, n->np * 4, cudaMemcpyDeviceToHost));
    return SFSEG_OK;
}

int sfseg_net_set_params(sfseg_net* n, const float* host, int64_t count) {
    if (!n || !host) return nfail(SFSEG_ERR_INVALID_ARG, "null argument");
    if (count != n->np) return nfail(SFSEG_ERR_SHAPE, "parameter count mismatch");
    NET_CUDA(cudaMemcpy(n->p, host, n->np * 4, cudaMemcpyHostToDevice));
    n->packed = false;
    return SFSEG_OK;
}

int sfseg_net_forward(sfseg_net* n, const void* features, int dtype, int C, const float* extra, int T, int H, int W,
                      float* x0_out,
                      void* stream) {
    if (!n || !x0_out) return nfail(SFSEG_ERR_INVALID_ARG, "null argument");
    if (int rc = check_vol(C, T, H, W, features)) return rc;
    if (dtype != SFSEG_F32 && dtype != SFSEG_BF16) return nfail(SFSEG_ERR_DTYPE, "dtype must be F32 or BF16");
    if (C + (extra ? 1 : 0) > n->cin) return nfail(SFSEG_ERR_SHAPE, "more channels than the network was built for");
    cudaStream_t s = (cudaStream_t)stream;
    if (int rc = net_forward(n, features, dtype, C, extra, T, H, W, false, s)) return rc;
    NET_CUDA(cudaMemcpyAsync(x0_out, n->x0, (size_t)T * H * W * 4, cudaMemcpyDeviceToDevice, s));
    return SFSEG_OK;
}

int sfseg_net_backward(sfseg_net* n, const void* features, int dtype, int C, const float* extra, int T, int H, int W,
                       const float* target,
                       double* loss, float* grads_out, void* stream) {
    if (!n || !target || !loss) return nfail(SFSEG_ERR_INVALID_ARG, "null argument");
    if (int rc = check_vol(C, T, H, W, features)) return rc;
    if (dtype != SFSEG_F32 && dtype != SFSEG_BF16) return nfail(SFSEG_ERR_DTYPE, "dtype must be F32 or BF16");
    if (C + (extra ? 1 : 0) > n->cin) return nfail(SFSEG_ERR_SHAPE, "more channels than the network was built for");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = (int64_t)T * H * W;
    if (int rc = net_forward(n, features, dtype, C, extra, T, H, W, true, s)) return rc;
    NET_CUDA(cudaMemsetAsync(n->acc, 0, 8 * sizeof(double), s));
    NET_CUDA(cudaMemsetAsync(n->g, 0, n->np * 4, s));
    cos_sums<<<blocks_for(N), 256, 0, s>>>(n->x0, target, N, n->acc);
    cos_grad<<<blocks_for(N), 256, 0, s>>>(n->x0, target, n->z4, N, n->acc, n->dz16);
    count_launches(2);
    // layer 4
    if (int rc = wgrad(n, 3, n->dz16, 16, n->a3, 32, T, H, W, s)) return rc;
    if (int rc = run_conv<16, 32, EPI_MASK>(n->dz16, T, H, W, n->wb[3], nullptr, n->dza, n->a3, n->flags, s))
        return rc;
    // layer 3
    if (int rc = wgrad(n, 2, n->dza, 32, n->a2, 32, T, H, W, s)) return rc;
    if (int rc = run_conv<32, 32, EPI_MASK>(n->dza, T, H, W, n->wb[2], nullptr, n->dzb, n->a2, n->flags, s))
        return rc;
    // layer 2
    if (int rc = wgrad(n, 1, n->dzb, 32, n->a1, 32, T, H, W, s)) return rc;
    if (int rc = run_conv<32, 32, EPI_MASK>(n->dzb, T, H, W, n->wb[1], nullptr, n->dza, n->a1, n->flags, s))
        return rc;
    // layer 1
    if (int rc = wgrad(n, 0, n->dza, 32, n->x16, 16, T, H, W, s)) return rc;
    double a[3];
    NET_CUDA(cudaMemcpyAsync(a, n->acc, sizeof(a), cudaMemcpyDeviceToHost, s));
    if (int rc = check_flags(n, s)) return rc;
    *loss = 1.0 - a[0] / std::sqrt(a[1] * a[2]);
    if (grads_out) NET_CUDA(cudaMemcpy(grads_out, n->g, n->np * 4, cudaMemcpyDeviceToHost));
    return SFSEG_OK;
}

int sfseg_net_layer_forward(sfseg_net* n, int layer, const void* in, int T, int H, int W, void* out, float* out2,
                            void* stream) {
    if (!n || !in || !out) return nfail(SFSEG_ERR_INVALID_ARG, "null argument");
    if (layer < 0 || layer > 3) return nfail(SFSEG_ERR_INVALID_ARG, "layer must be in [0, 3]");
    if (layer == 3 && !out2) return nfail(SFSEG_ERR_INVALID_ARG, "the last layer needs out2 (softplus output)");
    if (T < 1 || H < 1 || W < 1) return nfail(SFSEG_ERR_SHAPE, "empty volume");
    if ((int64_t)T * H * W >= (int64_t(1) << 31)) return nfail(SFSEG_ERR_SHAPE, "volume too large");
    cudaStream_t s = (cudaStream_t)stream;
    if (int rc = pack_all(n, s)) return rc;
    const float* b = n->p + n->off[2 * layer + 1];
    const __nv_bfloat16* x = (const __nv_bfloat16*)in;
    if (layer == 0) return run_conv<16, 32, EPI_RELU>(x, T, H, W, n->wf[0], b, out, nullptr, n->flags, s);
    if (layer < 3) return run_conv<32, 32, EPI_RELU>(x, T, H, W, n->wf[layer], b, out, nullptr, n->flags, s);
    return run_last(x, T, H, W, n->wf[3], b, (float*)out, out2, n->flags, s);
}

int sfseg_net_layer_backward(sfseg_net* n, int layer, const void* in, const void* dz, int T, int H, int W,
                             void* dx_out, float* dW_out, float* db_out, void* stream) {
    if (!n || !in || !dz || !dW_out || !db_out) return nfail(SFSEG_ERR_INVALID_ARG, "null argument");
    if (layer < 0 || layer > 3) return nfail(SFSEG_ERR_INVALID_ARG, "layer must be in [0, 3]");
    if (T < 1 || H < 1 || W < 1) return nfail(SFSEG_ERR_SHAPE, "empty volume");
    if ((int64_t)T * H * W >= (int64_t(1) << 31)) return nfail(SFSEG_ERR_SHAPE, "volume too large");
    cudaStream_t s = (cudaStream_t)stream;
    if (int rc = pack_all(n, s)) return rc;
    const int cin = layer_cin(n, layer), cinp = layer == 0 ? 16 : 32, dzc = layer == 3 ? 16 : 32;
    const __nv_bfloat16* x = (const __nv_bfloat16*)in;
    const __nv_bfloat16* g = (const __nv_bfloat16*)dz;
    if (int rc = wgrad_into(n, layer, cin, g, dzc, x, cinp, T, H, W, dW_out, db_out, s)) return rc;
    if (dx_out && layer > 0) {
        if (layer == 3)
            return run_conv<16, 32, EPI_MASK>(g, T, H, W, n->wb[3], nullptr, dx_out, x, n->flags, s);
        return run_conv<32, 32, EPI_MASK>(g, T, H, W, n->wb[layer], nullptr, dx_out, x, n->flags, s);
    }
    return SFSEG_OK;
}

int sfseg_net_check(sfseg_net* n, void* stream) {
    if (!n) return nfail(SFSEG_ERR_INVALID_ARG, "null net");
    return check_flags(n, (cudaStream_t)stream);
}

int sfseg_net_launch_shape(int kernel, int* frames, int* rows, int* ctas) {
    if (kernel < 0 || kernel > 1) return nfail(SFSEG_ERR_INVALID_ARG, "kernel must be 0 or 1");
    if (!frames || !rows || !ctas) return nfail(SFSEG_ERR_INVALID_ARG, "null output");
    *frames = last_shape[kernel].frames;
    *rows = last_shape[kernel].rows;
    *ctas = last_shape[kernel].ctas;
    return SFSEG_OK;
}

int sfseg_net_adamw(sfseg_net* n, float lr, float beta1, float beta2, float eps, float weight_decay, void* stream) {
    if (!n) return nfail(SFSEG_ERR_INVALID_ARG, "null net");
    if (!(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return nfail(SFSEG_ERR_INVALID_ARG, "bad AdamW hyper-parameters");
    cudaStream_t s = (cudaStream_t)stream;
    n->step += 1;
    const float bc1 = 1.f - std::pow(beta1, (float)n->step), bc2 = 1.f - std::pow(beta2, (float)n->step);
    adamw_kernel<<<blocks_for(n->np), 256, 0, s>>>(n->p, n->g, n->m, n->v, n->np, lr, beta1, beta2, eps, weight_decay,
                                                   bc1, bc2);
    count_launches(1);
    NET_CUDA(cudaGetLastError());
    n->packed = false;
    return SFSEG_OK;
}

}  // extern "C"
