// voxels.cuh -- the visiting order of the element-wise kernels: rows (t, h) over the grid's
// blocks, columns w over a block's threads, so that neighbouring threads touch neighbouring
// addresses and no thread divides an index to find its row.
#pragma once

#include "common.cuh"

namespace sfseg {

// f(i, j) for every voxel: i its index in the caller's layout [T][H][W], j in the internal
// pitched layout [T][H][pitch].
template <typename F>
__device__ __forceinline__ void for_each_voxel(const Geom& g, F&& f) {
    const int64_t rows = (int64_t)g.T * g.H;
    for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const int64_t i0 = row * g.W, j0 = row * g.pitch;
        for (int w = threadIdx.x; w < g.W; w += blockDim.x) f(i0 + w, j0 + w);
    }
}

// With pairs: f2(i, j) for the column pairs (i, i + 1) of the caller layout and (j, j + 1) of the
// internal layout, every row taken two columns at a time (W even, and every caller-layout array
// 8-byte aligned, so that both layouts' pairs are 8-byte aligned: the pitch is a multiple of 32).
// Without: f1(i, j) for every voxel, as for_each_voxel.
template <typename F2, typename F1>
__device__ __forceinline__ void for_each_voxel_pairs(const Geom& g, bool pairs, F2&& f2, F1&& f1) {
    if (!pairs) {
        for_each_voxel(g, f1);
        return;
    }
    const int64_t rows = (int64_t)g.T * g.H;
    const int np = g.W >> 1;
    for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const int64_t i0 = row * g.W, j0 = row * g.pitch;
        for (int c = threadIdx.x; c < np; c += blockDim.x) f2(i0 + 2 * c, j0 + 2 * c);
    }
}

__device__ __forceinline__ float2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ float2 ld2(const __nv_bfloat16* p) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
}
__device__ __forceinline__ void st2(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }
__device__ __forceinline__ void st2(__nv_bfloat16* p, float2 v) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(v.x, v.y);
}

inline bool aligned8(const void* a, const void* b = nullptr, const void* c = nullptr) {
    return (((uintptr_t)a | (uintptr_t)b | (uintptr_t)c) & 7) == 0;
}

// f4(i) for the groups [4i, 4i + 4) of [0, n) and f1(i) for the n % 4 elements after them when
// vec (every array the caller touches is 16-byte aligned), else f1(i) for every element: the
// flat element-wise passes then move 16 bytes per access.
template <typename F4, typename F1>
__device__ __forceinline__ void for_each_flat(int64_t n, bool vec, F4&& f4, F1&& f1) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t first = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t done = 0;
    if (vec) {
        const int64_t n4 = n >> 2;
        for (int64_t i = first; i < n4; i += stride) f4(i);
        done = n4 << 2;
    }
    for (int64_t i = done + first; i < n; i += stride) f1(i);
}

inline bool aligned16(const void* a, const void* b = nullptr) {
    return (((uintptr_t)a | (uintptr_t)b) & 15) == 0;
}

// Launch shape for for_each_voxel: up to 256 threads (a multiple of 32 covering W when W is
// small), at most `per_sm` blocks per SM.
struct RowLaunch {
    int blocks, threads;
};
inline RowLaunch row_launch(const Geom& g, int sms, int per_sm = 16) {
    const int64_t rows = (int64_t)g.T * g.H;
    int threads = g.W >= 256 ? 256 : ((g.W + 31) / 32) * 32;
    int64_t b = rows < (int64_t)per_sm * sms ? rows : (int64_t)per_sm * sms;
    return {(int)(b > 0 ? b : 1), threads > 0 ? threads : 32};
}

}  // namespace sfseg
