// common.cuh -- device helpers shared by the sfseg kernels (sm_103a).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sfseg {

constexpr int kMaxRT = 4;
constexpr int kMaxRH = 8;
constexpr int kMaxRW = 8;

// Error flag bits written by kernels into the handle's device flag word.
constexpr int kFlagBadFeature = 1;   // a feature value was negative, NaN or Inf
constexpr int kFlagZeroNorm = 2;     // an iterate norm was exactly zero
constexpr int kFlagNonfinite = 4;    // an iterate norm was NaN or Inf
constexpr int kFlagTimeout = 8;      // a bounded wait inside a kernel gave up

// 1D factors of the separable Gaussian (Sec. 4.2), index d + r for offset d in [-r, r].
struct Taps {
    int rt, rh, rw;
    float gt[2 * kMaxRT + 1];
    float gh[2 * kMaxRH + 1];
    float gw[2 * kMaxRW + 1];
};

// Geometry of the handle's volumes.  Internal volumes have a padded row pitch (a multiple of
// 8 elements, so every row starts 16-byte aligned for bf16 and float); the caller's volumes
// use pitch W.
struct Geom {
    int T, H, W;
    int pitch;   // elements per row of internal volumes
};

__device__ __forceinline__ float ldf(const float* p) { return *p; }
__device__ __forceinline__ float ldf(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ void stf(float* p, float v) { *p = v; }
__device__ __forceinline__ void stf(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

// Unary term u = s^p with 0^p := 0 (p > 0).
__device__ __forceinline__ float unary_pow(float s, float p) {
    return s > 0.f ? exp2f(p * log2f(s)) : 0.f;
}

// Faster variant on the special-function unit: u = 2^(p log2 s) with the approximate log2 and
// exp2 instructions (relative error a few 1e-7 for p <= 1).  s = 0 gives log2 s = -inf and
// u = +0, so no branch is needed (s < 0 never reaches here: features are checked >= 0).
__device__ __forceinline__ float unary_pow_fast(float s, float p) {
    float l, u;
    asm("lg2.approx.f32 %0, %1;" : "=f"(l) : "f"(s));
    asm("ex2.approx.f32 %0, %1;" : "=f"(u) : "f"(p * l));
    return u;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of `v` over the block (any blockDim that is a multiple of 32, at most 1024).
// All threads must call it; the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();   // protects red[] against a previous call
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        r = lane < nw ? red[lane] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

// 1/sqrt(acc) of an FP64 sum of squares, with the flag raised (and 0 returned) when the sum is
// zero or not finite, so that later iterations produce zeros instead of NaNs.
__device__ __forceinline__ float inv_norm_from(const double* acc, int* flags) {
    if (acc == nullptr) return 1.f;
    const double a = *acc;
    if (!(a > 0.0) || !(a < 1e300)) {
        if (threadIdx.x == 0 && flags) atomicOr(flags, a == 0.0 ? kFlagZeroNorm : kFlagNonfinite);
        return 0.f;
    }
    return (float)(1.0 / sqrt(a));
}

}  // namespace sfseg
