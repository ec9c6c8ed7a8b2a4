// kernels_bwd.cu -- adjoint of the unrolled power iteration (learning the Eq. 9 weights,
// Sec. 3.4) and the soft-IoU learning loss.
//
// Forward step k (A = A(f) symmetric, x_k unit norm):  y = A x_k, nu = ||y||, x_{k+1} = y / nu.
// Reverse step, given g_{k+1} = dL/dx_{k+1}:
//     g_y     = (g_{k+1} - x_{k+1} <x_{k+1}, g_{k+1}>) / nu
//     g_k     = A g_y                                       (A' = A)
//     dL/df  += d/df [ g_y' A(f) x_k ]
// With A_ij = u_i u_j (1/alpha - (f_i - f_j)^2) G_ij and u = f^p, the last term is, per voxel i,
//     alpha_i S1_i + beta_i S3_i - d_i S2_i,       d_i = p f_i^(p-1),
//     alpha_i = d_i (1/alpha - f_i^2) - 2 u_i f_i,  beta_i = 2 d_i f_i + 2 u_i,
//     S1 = g_y G*(u x) + x G*(u g_y),  S2 = g_y G*(f^2 u x) + x G*(f^2 u g_y),
//     S3 = g_y G*(f u x) + x G*(f u g_y),
// so one streaming pass filters six signals (three of x_k, three of g_y).  Through the Eq. 9
// sigmoid, dL/dz_i = f_i (1 - f_i) dL/df_i, which removes the f^(p-1) singularity:
//     dL/dz_i = (1 - f_i) u_i [ (p (1/alpha - f_i^2) - 2 f_i^2) S1 + 2 (p + 1) f_i S3 - p S2 ].
// The per-voxel dL/dz is accumulated over all steps; dL/dw_c = sum_i dL/dz_i V_c,i and
// dL/db = sum_i dL/dz_i follow in one reduction.
#include "common.cuh"
#include "launch.h"
#include "stencil.cuh"
#include "voxels.cuh"

namespace sfseg {

struct OpAdjoint {
    static constexpr int NS = 6;
    const float* xk;      // x~_k   (internal layout), x_k = sk * x~_k
    const float* xn;      // x~_{k+1},  x_{k+1} = sn * x~_{k+1}, nu_{k+1} = 1 / sn
    const float* gn;      // g_{k+1}
    const double* acc_k;  // ||x~_k||^2
    const double* acc_n;  // ||x~_{k+1}||^2
    const double* dot_n;  // <x_{k+1}, g_{k+1}>
    const float* f;
    float* gk_out;        // g_k (nullable)
    float* gz;            // accumulated dL/dz
    Geom g;
    float inv_alpha, p;
    float sk, sn, dotn;

    __device__ __forceinline__ void begin(const double*, int* flags) {
        sk = inv_norm_from(acc_k, flags);
        sn = inv_norm_from(acc_n, flags);
        dotn = (float)*dot_n;
    }
    __device__ __forceinline__ void xg(int64_t i, float& x, float& gy) const {
        x = sk * xk[i];
        gy = (gn[i] - sn * xn[i] * dotn) * sn;
    }
    __device__ __forceinline__ void load(int t, int h, int w, float (&z)[NS]) const {
        const int64_t i = ((int64_t)t * g.H + h) * g.pitch + w;
        const float fv = f[i];
        const float u = unary_pow(fv, p);
        float x, gy;
        xg(i, x, gy);
        const float z1 = u * x, w1 = u * gy;
        z[0] = z1;
        z[2] = fv * z1;
        z[1] = fv * z[2];
        z[3] = w1;
        z[5] = fv * w1;
        z[4] = fv * z[5];
    }
    __device__ __forceinline__ void epi(int t, int h, int w, const float (&c)[NS], float& acc0,
                                        float&) const {
        const int64_t i = ((int64_t)t * g.H + h) * g.pitch + w;
        const float fv = f[i];
        const float u = unary_pow(fv, p);
        float x, gy;
        xg(i, x, gy);
        const float f2 = fv * fv;
        const float gk = u * ((inv_alpha - f2) * c[3] - c[4] + 2.f * fv * c[5]);
        if (gk_out) gk_out[i] = gk;
        acc0 += x * gk;
        const float S1 = gy * c[0] + x * c[3];
        const float S2 = gy * c[1] + x * c[4];
        const float S3 = gy * c[2] + x * c[5];
        gz[i] += (1.f - fv) * u * ((p * (inv_alpha - f2) - 2.f * f2) * S1 + 2.f * (p + 1.f) * fv * S3 - p * S2);
    }
};

void launch_adjoint_step(const float* xk, const double* acc_k, const float* xn, const double* acc_n,
                         const float* gn, const double* dot_n, float* gk_out, double* dot_k, float* gz,
                         const float* f32, Geom g, const Taps& tp, float inv_alpha, float p, cudaStream_t s) {
    OpAdjoint op;
    op.xk = xk;
    op.xn = xn;
    op.gn = gn;
    op.acc_k = acc_k;
    op.acc_n = acc_n;
    op.dot_n = dot_n;
    op.f = f32;
    op.gk_out = gk_out;
    op.gz = gz;
    op.g = g;
    op.inv_alpha = inv_alpha;
    op.p = p;
    op.sk = op.sn = op.dotn = 0.f;
    run_stencil(op, tp, 8, nullptr, dot_k, nullptr, nullptr, s);
}

// v = u x, both in the internal layout.
__global__ void state_internal_kernel(const float* x, const float* f, float p, Geom g, float* v) {
    for_each_voxel(g, [&](int64_t, int64_t j) { v[j] = unary_pow_fast(f[j], p) * x[j]; });
}


// ---- the reverse step in the stencil's state form (TMA kernel only).  With V_k = u x~_k (the
// state the forward step itself carries), G_k = u g_k and v_g = u g_y, a step is: Q_x from V_k
// (mode 1, scaled by s_k = 1/||x~_k||), the g-pass on v_g (mode 5: G_k, Q_g and sum V_k B), and
// one element-wise pass that adds the feature term and forms the next step's v_g.  The
// recomputation between checkpoints is the plain step on V (mode 0).

// v_g of the first reverse step: u g_y = s_K u (g_K - s_K x~_K <x_K, g_K>).
__global__ void adjoint_first_kernel(const float* xK, const double* accK, const float* gK, const double* dotK,
                                     const float* f, float p, Geom g, float* vg) {
    const float sK = inv_norm_from(accK, nullptr);
    const float d = (float)*dotK;
    for_each_voxel(g, [&](int64_t, int64_t j) {
        vg[j] = unary_pow_fast(f[j], p) * ((gK[j] - sK * xK[j] * d) * sK);
    });
}

void launch_adjoint_first(const float* xK, const double* accK, const float* gK, const double* dotK,
                          const float* f32, float p, Geom g, float* vg, cudaStream_t s) {
    const RowLaunch rl = row_launch(g, num_sms(), 8);
    adjoint_first_kernel<<<rl.blocks, rl.threads, 0, s>>>(xK, accK, gK, dotK, f32, p, g, vg);
    count_launches(1);
}

// gz += (1 - f) (v_g Q_x + s_k V_k Q_g)  (= (1 - f) u (g_y Q_x + x_k Q_g)), and, when vg_next is
// given, the next step's v_g = u g_y(k-1) = s_k (G_k - s_k <x_k, g_k> V_k) with
// <x_k, g_k> = s_k * dsum (dsum = sum V_k B from the g-pass).
__global__ void adjoint_combine_state_kernel(const float* f, const float* vg, const float* qx, const float* Vk,
                                             const float* qg, const float* Gk, const double* acc_k,
                                             const double* dsum, Geom g, float* gz, float* vg_next) {
    const float sk = inv_norm_from(acc_k, nullptr);
    const float dot = sk * (float)*dsum;
    // rows (t, h) over the blocks, four columns per thread (internal rows start 128-byte
    // aligned), the ragged end of a row one column at a time
    const int64_t rows = (int64_t)g.T * g.H;
    const int w4 = g.W / 4;
    for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const int64_t j0 = row * g.pitch;
        for (int c = threadIdx.x; c < w4; c += blockDim.x) {
            const int64_t j = j0 + 4 * c;
            const float4 v = *reinterpret_cast<const float4*>(Vk + j);
            const float4 ff = *reinterpret_cast<const float4*>(f + j);
            const float4 a = *reinterpret_cast<const float4*>(vg + j);
            const float4 b = *reinterpret_cast<const float4*>(qx + j);
            const float4 q = *reinterpret_cast<const float4*>(qg + j);
            float4 z = *reinterpret_cast<const float4*>(gz + j);
            z.x += (1.f - ff.x) * (a.x * b.x + sk * v.x * q.x);
            z.y += (1.f - ff.y) * (a.y * b.y + sk * v.y * q.y);
            z.z += (1.f - ff.z) * (a.z * b.z + sk * v.z * q.z);
            z.w += (1.f - ff.w) * (a.w * b.w + sk * v.w * q.w);
            *reinterpret_cast<float4*>(gz + j) = z;
            if (vg_next) {
                const float4 G = *reinterpret_cast<const float4*>(Gk + j);
                *reinterpret_cast<float4*>(vg_next + j) =
                    make_float4(sk * (G.x - sk * dot * v.x), sk * (G.y - sk * dot * v.y), sk * (G.z - sk * dot * v.z),
                                sk * (G.w - sk * dot * v.w));
            }
        }
        for (int w = 4 * w4 + threadIdx.x; w < g.W; w += blockDim.x) {
            const int64_t j = j0 + w;
            const float v = Vk[j];
            gz[j] += (1.f - f[j]) * (vg[j] * qx[j] + sk * v * qg[j]);
            if (vg_next) vg_next[j] = sk * (Gk[j] - sk * dot * v);
        }
    }
}

void launch_adjoint_combine_state(const float* f32, const float* vg, const float* qx, const float* Vk,
                                  const float* qg, const float* Gk, const double* acc_k, const double* dsum, Geom g,
                                  float* gz, float* vg_next, cudaStream_t s) {
    const int w4 = g.W / 4;
    const int threads = w4 >= 128 ? 128 : (w4 > 0 ? (w4 + 31) / 32 * 32 : 32);
    const int64_t rows = (int64_t)g.T * g.H;
    const int64_t cap = (int64_t)16 * num_sms();
    const int blocks = (int)(rows < cap ? (rows > 0 ? rows : 1) : cap);
    adjoint_combine_state_kernel<<<blocks, threads, 0, s>>>(f32, vg, qx, Vk, qg, Gk, acc_k, dsum, g, gz, vg_next);
    count_launches(1);
}

// V = u x~ for a checkpoint (internal layout), the start of a recomputed segment.
void launch_state_internal(const float* x, const float* f32, float p, Geom g, float* v, cudaStream_t s) {
    const RowLaunch rl = row_launch(g, num_sms());
    state_internal_kernel<<<rl.blocks, rl.threads, 0, s>>>(x, f32, p, g, v);
    count_launches(1);
}

// g_K from the caller's layout into the internal layout, and <x_K, g_K>.
__global__ void grad_in_kernel(const float* gx_user, const float* xK, const double* accK, float* g_out, Geom g,
                               double* dot_out) {
    const float sK = inv_norm_from(accK, nullptr);
    const int64_t HW = (int64_t)g.H * g.W, N = HW * g.T;
    float part = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i / HW, rem = i - t * HW;
        const int64_t h = rem / g.W, wc = rem - h * g.W;
        const int64_t j = (t * g.H + h) * g.pitch + wc;
        const float gv = gx_user[i];
        g_out[j] = gv;
        part += sK * xK[j] * gv;
    }
    const double b = block_sum((double)part);
    if (threadIdx.x == 0) atomicAdd(dot_out, b);
}

void launch_grad_in(const float* gx_user, const float* xK, const double* accK, float* g_out, Geom g,
                    double* dot_out, cudaStream_t s) {
    const int64_t N = (int64_t)g.T * g.H * g.W;
    int blocks = (int)((N + 255) / 256);
    if (blocks > 8 * num_sms()) blocks = 8 * num_sms();
    grad_in_kernel<<<blocks, 256, 0, s>>>(gx_user, xK, accK, g_out, g, dot_out); count_launches(1);
}

// acc[c] += sum_i gz_i V_c,i  (c < C),  acc[C] += sum_i gz_i.
template <typename TIn>
__global__ void weight_grad_kernel(const TIn* feat, int C, Geom g, const float* gz, double* acc) {
    constexpr int kMaxC = 64;
    float part[kMaxC + 1];
    for (int c = 0; c <= C; ++c) part[c] = 0.f;
    const int64_t HW = (int64_t)g.H * g.W, N = HW * g.T;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i / HW, rem = i - t * HW;
        const int64_t h = rem / g.W, wc = rem - h * g.W;
        const float gv = gz[(t * g.H + h) * g.pitch + wc];
        part[C] += gv;
        for (int c = 0; c < C; ++c) part[c] += gv * ldf(feat + (int64_t)c * N + i);
    }
    for (int c = 0; c <= C; ++c) {
        const double b = block_sum((double)part[c]);
        if (threadIdx.x == 0) atomicAdd(acc + c, b);
    }
}

void launch_weight_grad(const void* feat, int feat_dtype, int C, Geom g, const float* gz, double* acc,
                        cudaStream_t s) {
    const int64_t N = (int64_t)g.T * g.H * g.W;
    int blocks = (int)((N + 255) / 256);
    if (blocks > 4 * num_sms()) blocks = 4 * num_sms();
    if (feat_dtype == kF32)
        weight_grad_kernel<float><<<blocks, 256, 0, s>>>((const float*)feat, C, g, gz, acc);
    else
        weight_grad_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>((const __nv_bfloat16*)feat, C, g, gz, acc);
    count_launches(1);
}

// ----------------------------------------------------------------------- soft-IoU loss
// Order-preserving key of (value, -index): larger value first, then the smaller index.
__device__ __forceinline__ unsigned long long amax_key(float v, int64_t i) {
    unsigned int b = __float_as_uint(v);
    b = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
    return ((unsigned long long)b << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned int)i);
}
__device__ __forceinline__ float key_value(unsigned long long k) {
    unsigned int b = (unsigned int)(k >> 32);
    b = (b & 0x80000000u) ? (b & 0x7FFFFFFFu) : ~b;
    return __uint_as_float(b);
}

__global__ void amax_kernel(const float* x, int64_t n, unsigned long long* out) {
    unsigned long long best = 0ull;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = amax_key(x[i], i);
        best = k > best ? k : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
        best = other > best ? other : best;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

__global__ void iou_sums_kernel(const float* x, const float* tg, int64_t n, const unsigned long long* amax,
                                double* acc) {
    const float m = key_value(*amax);
    float a = 0.f, b = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float xh = x[i] / m, gv = tg[i];
        a += xh * gv;
        b += xh + gv - xh * gv;
    }
    const double sa = block_sum((double)a);
    if (threadIdx.x == 0) atomicAdd(acc, sa);
    const double sb = block_sum((double)b);
    if (threadIdx.x == 0) atomicAdd(acc + 1, sb);
}

__global__ void iou_grad_kernel(const float* x, const float* tg, int64_t n, const unsigned long long* amax,
                                double* acc, float* grad) {
    const float m = key_value(*amax);
    const double I = acc[0], U = acc[1];
    const float cu = (float)(1.0 / U), ci = (float)(I / (U * U));
    float a = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gv = tg[i];
        const float dxh = -(gv * cu - ci * (1.f - gv));
        grad[i] = dxh / m;
        a += dxh * x[i];
    }
    const double sa = block_sum((double)a);
    if (threadIdx.x == 0) atomicAdd(acc + 2, sa);
}

__global__ void iou_fix_kernel(const unsigned long long* amax, const double* acc, float* grad) {
    const float m = key_value(*amax);
    const unsigned int idx = 0xFFFFFFFFu - (unsigned int)(*amax & 0xFFFFFFFFull);
    grad[idx] -= (float)(acc[2] / ((double)m * m));
}

void launch_soft_iou(const float* x, const float* tgt, int64_t n, float* grad, double* acc,
                     unsigned long long* amax, cudaStream_t s) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 8 * num_sms()) blocks = 8 * num_sms();
    amax_kernel<<<blocks, 256, 0, s>>>(x, n, amax); count_launches(1);
    iou_sums_kernel<<<blocks, 256, 0, s>>>(x, tgt, n, amax, acc); count_launches(1);
    if (grad) {
        iou_grad_kernel<<<blocks, 256, 0, s>>>(x, tgt, n, amax, acc, grad); count_launches(1);
        iou_fix_kernel<<<1, 1, 0, s>>>(amax, acc, grad); count_launches(1);
    }
}

}  // namespace sfseg
