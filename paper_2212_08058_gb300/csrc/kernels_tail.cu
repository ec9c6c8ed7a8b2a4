// kernels_tail.cu -- the soft-binarisation iterations that end the method (Alg. 1 step 3,
// Sec. 4.1).  After the continuous power iterations, each further step applies the Eq. 7
// operator, y = A x, and then squashes the result towards {0, 1} with a sigmoid; the hard
// segmentation is the final x thresholded at 1/2.  The sigmoid acts on y scaled to maximum 1,
//     x <- 1 / (1 + exp(-gain (y / max(y) - center))),
// so that gain and centre mean the same thing for any volume size (the paper leaves the
// sigmoid's parameterisation open).
//
// A step is the stencil launch (y in caller layout; for shared maps and a radius with a TMA
// kernel the launch also takes max(y), kernels_fast.cu mode 8, else one reduction does), and one
// elementwise pass that writes x, and, for the next step, the stencil's input state u * x in
// the internal layout (so the next stencil launch needs no separate conversion).
#include "common.cuh"
#include "launch.h"
#include "order_key.cuh"
#include "voxels.cuh"

namespace sfseg {

__global__ void max_key_kernel(const float* y, int64_t n, unsigned* key) {
    unsigned m = 0u;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, order_key(y[i]));
    m = __reduce_max_sync(0xffffffffu, m);
    __shared__ unsigned wmax[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) wmax[warp] = m;
    __syncthreads();
    if (warp == 0) {
        m = lane < (int)(blockDim.x >> 5) ? wmax[lane] : 0u;
        m = __reduce_max_sync(0xffffffffu, m);
        if (lane == 0) atomicMax(key, m);
    }
}

// x = sigmoid(gain (y / max y - center)) for the N voxels (caller layout).  Optional outputs:
// v (internal layout, u * x, the next stencil input) and mask (x > 1/2 as 0/1 bytes).
__global__ void sigmoid_step_kernel(const float* y, const unsigned* key, float gain, float center, const float* f32,
                                    const float* s32, float p, Geom g, float* x, float* v, unsigned char* mask,
                                    int* flags) {
    const float m = order_value(*key);
    if (!(m > 0.f) || isinf(m)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(flags, m > 0.f ? kFlagNonfinite : kFlagZeroNorm);
        return;
    }
    const float gm = -gain;
    for_each_voxel(g, [&](int64_t i, int64_t j) {
        const float xi = 1.f / (1.f + expf(gm * (y[i] / m - center)));
        x[i] = xi;
        if (mask) mask[i] = xi > 0.5f ? 1 : 0;
        if (v) v[j] = unary_pow_fast(s32 ? s32[j] : f32[j], p) * xi;
    });
}

static int grid_for(int64_t n) {
    const int64_t b = (n + 255) / 256;
    const int cap = 8 * num_sms();
    return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

void launch_max_key(const float* y, int64_t n, unsigned* key, cudaStream_t s) {
    cudaMemsetAsync(key, 0, sizeof(unsigned), s);
    max_key_kernel<<<grid_for(n), 256, 0, s>>>(y, n, key);
    count_launches(1);
}

void launch_sigmoid_step(const float* y, const unsigned* key, float gain, float center, const float* f32, float p,
                         Geom g, float* x, float* v, unsigned char* mask, int* flags, cudaStream_t s,
                         const float* s32) {
    const RowLaunch rl = row_launch(g, num_sms());
    sigmoid_step_kernel<<<rl.blocks, rl.threads, 0, s>>>(y, key, gain, center, f32, s32, p, g, x, v, mask, flags);
    count_launches(1);
}

}  // namespace sfseg
