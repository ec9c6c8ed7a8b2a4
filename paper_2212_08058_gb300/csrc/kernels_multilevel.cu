// kernels_multilevel.cu -- restriction and prolongation between a volume and its 2x-coarsened
// copy, for starting the power iteration from a coarse solution.
//
// The slowly converging components of the iterate are smooth at the scale of the objects (the
// spectral gap of the Eq. 7 operator shrinks with the size of the volume in pixels), so the
// same operator on a pooled volume, with the Gaussian's widths measured in coarse pixels, has
// nearly the same principal eigenvector at those scales and converges in as many iterations at
// an eighth of the cost.  Upsampled, it is a start vector whose remaining error is local.
#include "common.cuh"
#include "launch.h"
#include "order_key.cuh"

namespace sfseg {

// out[Tc][Hc][Wc] = mean of f over the (pt x ph x pw) block that lies inside the volume.
// f in the internal layout of `g`; out in caller layout (pitch Wc).  Rows (tc, hc) over the
// blocks, columns over the threads.
__global__ void pool_f_kernel(const float* f, Geom g, int pt, int ph, int pw, int Tc, int Hc, int Wc, float* out) {
    const int64_t rows = (int64_t)Tc * Hc;
    for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const int tc = (int)(row / Hc), hc = (int)(row - (int64_t)tc * Hc);
        for (int wc = threadIdx.x; wc < Wc; wc += blockDim.x) {
            float s = 0.f;
            int n = 0;
            for (int a = 0; a < pt; ++a) {
                const int t = tc * pt + a;
                if (t >= g.T) continue;
                for (int b = 0; b < ph; ++b) {
                    const int h = hc * ph + b;
                    if (h >= g.H) continue;
                    for (int c = 0; c < pw; ++c) {
                        const int w = wc * pw + c;
                        if (w >= g.W) continue;
                        s += f[((int64_t)t * g.H + h) * g.pitch + w];
                        ++n;
                    }
                }
            }
            out[row * Wc + wc] = n ? s / (float)n : 0.f;
        }
    }
}

// Linear interpolation weights of destination index d on an axis coarsened by p (half-pixel
// centres: source coordinate (d + 0.5) / p - 0.5, clamped to the coarse extent).
__device__ __forceinline__ void lin(int d, int p, int nc, int& i0, int& i1, float& w1) {
    if (p == 1) {
        i0 = i1 = min(d, nc - 1);
        w1 = 0.f;
        return;
    }
    float src = (d + 0.5f) / (float)p - 0.5f;
    src = fminf(fmaxf(src, 0.f), (float)(nc - 1));
    i0 = (int)src;
    i1 = min(i0 + 1, nc - 1);
    w1 = src - (float)i0;
}

// x[T][H][W] (caller layout) = trilinear interpolation of xc[Tc][Hc][Wc].  Rows (t, h) over
// the blocks (their t and h weights computed once per row), columns over the threads.
__global__ void upsample_kernel(const float* xc, int Tc, int Hc, int Wc, int pt, int ph, int pw, int T, int H, int W,
                                float* x) {
    const int64_t rows = (int64_t)T * H;
    for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const int t = (int)(row / H), h = (int)(row - (int64_t)t * H);
        int t0, t1, h0, h1;
        float at, ah;
        lin(t, pt, Tc, t0, t1, at);
        lin(h, ph, Hc, h0, h1, ah);
        const float* r00 = xc + ((int64_t)t0 * Hc + h0) * Wc;
        const float* r01 = xc + ((int64_t)t0 * Hc + h1) * Wc;
        const float* r10 = xc + ((int64_t)t1 * Hc + h0) * Wc;
        const float* r11 = xc + ((int64_t)t1 * Hc + h1) * Wc;
        for (int w = threadIdx.x; w < W; w += blockDim.x) {
            int w0, w1i;
            float aw;
            lin(w, pw, Wc, w0, w1i, aw);
            const float c00 = r00[w0] + aw * (r00[w1i] - r00[w0]);
            const float c01 = r01[w0] + aw * (r01[w1i] - r01[w0]);
            const float c10 = r10[w0] + aw * (r10[w1i] - r10[w0]);
            const float c11 = r11[w0] + aw * (r11[w1i] - r11[w0]);
            const float c0 = c00 + ah * (c01 - c00);
            const float c1 = c10 + ah * (c11 - c10);
            x[row * W + w] = c0 + at * (c1 - c0);
        }
    }
}

// x /= max(x), the maximum given as an order-preserving key (no-op unless it is positive and
// finite).
__global__ void scale_by_max_kernel(float* x, int64_t n, const unsigned* key) {
    const float m = order_value(*key);
    if (!(m > 0.f) || isinf(m)) return;
    const float inv = 1.f / m;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] *= inv;
}

static int grid_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    const int cap = 16 * num_sms();
    return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

static int row_threads(int w) { return w >= 256 ? 256 : ((w + 31) / 32) * 32; }
static int row_blocks(int64_t rows) {
    const int64_t cap = 16 * (int64_t)num_sms();
    return (int)(rows < cap ? (rows > 0 ? rows : 1) : cap);
}

void launch_pool_f(const float* f, Geom g, int pt, int ph, int pw, int Tc, int Hc, int Wc, float* out, cudaStream_t s) {
    pool_f_kernel<<<row_blocks((int64_t)Tc * Hc), row_threads(Wc), 0, s>>>(f, g, pt, ph, pw, Tc, Hc, Wc, out);
    count_launches(1);
}

void launch_upsample(const float* xc, int Tc, int Hc, int Wc, int pt, int ph, int pw, int T, int H, int W, float* x,
                     cudaStream_t s) {
    upsample_kernel<<<row_blocks((int64_t)T * H), row_threads(W), 0, s>>>(xc, Tc, Hc, Wc, pt, ph, pw, T, H, W, x);
    count_launches(1);
}

void launch_scale_by_max(float* x, int64_t n, unsigned* key, cudaStream_t s) {
    launch_max_key(x, n, key, s);
    scale_by_max_kernel<<<grid_for(n), 256, 0, s>>>(x, n, key);
    count_launches(1);
}

}  // namespace sfseg
