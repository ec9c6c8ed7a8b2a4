// kernels_generic.cu -- the streaming space-time stencil for any supported radius, plus the
// small kernels around it (channel combination, start vector, reductions).
//
// The Eq. 7 operator needs the 3D Gaussian filtering of three signals
//     z1 = u x,  z2 = f^2 u x,  z3 = f u x           (u = s^p, s = f: shared maps, Sec. 5.1.2)
// followed by the per-voxel combination
//     A x = u [ (1/alpha - f^2) G*z1 - G*z2 + 2 f G*z3 ].
// A CTA owns a TH x 64 tile of (h, w) and walks along t through a chunk of frames.  For each
// incoming frame it stages the halo tile of the three signals in shared memory, filters along w
// then h (Sec. 4.2: the separable form), and keeps the 2D-filtered frame in a ring of 2rt+1
// frames; the t-filter and the combination then produce the output frame rt behind.
//
// Power iteration runs in a scaled form: the stored state is v_k = u * x~_k where x~_k = A x_{k-1}
// is the un-normalised iterate, whose squared norm the previous launch has accumulated in FP64.
// The Eq. 8 division by the norm is folded into the next step (A is linear), so no launch waits
// for a global reduction, and z1 = v needs no power in the halo.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "launch.h"
#include "stencil.cuh"
#include "voxels.cuh"

namespace sfseg {

// ----------------------------------------------------------------------------- stencil ops
// v-space power-iteration step.  OUT_X selects writing x~ (last step) instead of u x~.
template <typename TVI, typename TVO, typename TF, bool OUT_X>
struct OpIter {
    static constexpr int NS = 3;
    const TVI* v;
    const TF* f;
    TVO* out;
    int out_pitch;
    float* ckpt;
    const float* sm;   // separate unary map (nullable: s = f)
    Geom g;
    float inv_alpha, p, s;

    __device__ __forceinline__ void begin(const double* acc_in, int* flags) {
        s = inv_norm_from(acc_in, flags);
    }
    __device__ __forceinline__ void load(int t, int h, int w, float (&z)[NS]) const {
        const int64_t i = ((int64_t)t * g.H + h) * g.pitch + w;
        const float z1 = ldf(v + i), fv = ldf(f + i);
        const float z3 = fv * z1;
        z[0] = z1;
        z[1] = fv * z3;
        z[2] = z3;
    }
    __device__ __forceinline__ void epi(int t, int h, int w, const float (&c)[NS], float& acc0,
                                        float&) const {
        const int64_t i = ((int64_t)t * g.H + h) * g.pitch + w;
        const float fv = ldf(f + i);
        const float u = unary_pow(sm ? sm[i] : fv, p);
        const float B = (inv_alpha - fv * fv) * c[0] - c[1] + 2.f * fv * c[2];
        const float xt = s * u * B;
        acc0 += xt * xt;
        if (OUT_X) stf(out + ((int64_t)t * g.H + h) * out_pitch + w, xt);
        else stf(out + i, u * xt);
        if (ckpt) ckpt[i] = xt;
    }
};

// x-space application y = s A x (FP32 storage), used for residuals and recomputation.
struct OpApply {
    static constexpr int NS = 3;
    const float* x;
    int x_pitch;
    const float* f;
    float* out;
    int out_pitch;
    const float* sm;   // separate unary map (nullable: s = f)
    Geom g;
    float inv_alpha, p, s;

    __device__ __forceinline__ void begin(const double* acc_in, int* flags) {
        s = inv_norm_from(acc_in, flags);
    }
    __device__ __forceinline__ void load(int t, int h, int w, float (&z)[NS]) const {
        const float xv = x[((int64_t)t * g.H + h) * x_pitch + w];
        const int64_t j = ((int64_t)t * g.H + h) * g.pitch + w;
        const float fv = f[j];
        const float z1 = unary_pow(sm ? sm[j] : fv, p) * xv;
        const float z3 = fv * z1;
        z[0] = z1;
        z[1] = fv * z3;
        z[2] = z3;
    }
    __device__ __forceinline__ void epi(int t, int h, int w, const float (&c)[NS], float& acc0,
                                        float&) const {
        const int64_t j = ((int64_t)t * g.H + h) * g.pitch + w;
        const float fv = f[j];
        const float u = unary_pow(sm ? sm[j] : fv, p);
        const float y = s * u * ((inv_alpha - fv * fv) * c[0] - c[1] + 2.f * fv * c[2]);
        acc0 += y * y;
        out[((int64_t)t * g.H + h) * out_pitch + w] = y;
    }
};

static std::atomic<int64_t> g_launches{0};
// Which kernel ran the power-iteration steps: counts of steps issued on the TMA kernel and on the
// generic stencil, and the name of the last step's kernel instantiation.
static std::atomic<int64_t> g_steps_tma{0}, g_steps_generic{0};
static std::mutex g_step_mu;
static char g_step_name[96] = "";

static void note_step(bool tma, const Taps& tp, int vin_type, int out_type, bool out_x, bool record, bool sep) {
    (tma ? g_steps_tma : g_steps_generic).fetch_add(1, std::memory_order_relaxed);
    char buf[96];
    std::snprintf(buf, sizeof(buf), "%s<%d,%d,%d,%s,%s%s%s>", tma ? "iter_fast" : "stream_stencil<OpIter>", tp.rt,
                  tp.rh, tp.rw, vin_type == kF32 ? "float" : "bf16",
                  out_x ? "float(caller x)" : (out_type == kBF16 ? "bf16" : "float"), record ? ",record" : "",
                  sep ? ",separate maps" : "");
    std::lock_guard<std::mutex> lk(g_step_mu);
    std::memcpy(g_step_name, buf, sizeof(buf));
}

void iterate_kernel_stats(int64_t* tma_steps, int64_t* generic_steps, char* name, int len) {
    if (tma_steps) *tma_steps = g_steps_tma.load(std::memory_order_relaxed);
    if (generic_steps) *generic_steps = g_steps_generic.load(std::memory_order_relaxed);
    if (name && len > 0) {
        std::lock_guard<std::mutex> lk(g_step_mu);
        std::snprintf(name, (size_t)len, "%s", g_step_name);
    }
}
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

int num_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

template <typename TVI, typename TVO, typename TF, bool OUT_X>
static void iterate_t(const void* vin, void* out, const void* f, float* ckpt, Geom g, const Taps& tp,
                      float inv_alpha, float p, const double* acc_in, double* acc_out, int* flags,
                      cudaStream_t s, const float* s32) {
    OpIter<TVI, TVO, TF, OUT_X> op;
    op.sm = s32;
    op.v = (const TVI*)vin;
    op.f = (const TF*)f;
    op.out = (TVO*)out;
    op.out_pitch = OUT_X ? g.W : g.pitch;
    op.ckpt = ckpt;
    op.g = g;
    op.inv_alpha = inv_alpha;
    op.p = p;
    op.s = 1.f;
    run_stencil(op, tp, 16, acc_in, acc_out, nullptr, flags, s);
}

void launch_iterate(const void* vin, int vin_type, void* out, int out_type, bool out_x, const void* f,
                    int f_type, float* ckpt, Geom g, const Taps& tp, float inv_alpha, float p,
                    const double* acc_in, double* acc_out, int* flags, cudaStream_t s, const float* s32) {
    using bf = __nv_bfloat16;
    // The TMA kernel serves the method's radii, recording steps (float32, shared maps) included.
    if (ckpt == nullptr && fast_iterate_supported(tp) &&
        launch_iterate_fast(vin, vin_type, out, out_type, out_x, f, g, tp, inv_alpha, p, acc_in, acc_out, flags, s,
                            s32)) {
        note_step(true, tp, vin_type, out_type, out_x, false, s32 != nullptr);
        return;
    }
    if (ckpt != nullptr && vin_type == kF32 && s32 == nullptr && fast_iterate_supported(tp) &&
        launch_iterate_fast_ckpt((const float*)vin, out, out_x, (const float*)f, g, tp, inv_alpha, p, acc_in, acc_out,
                                 ckpt, flags, s)) {
        note_step(true, tp, vin_type, out_type, out_x, true, false);
        return;
    }
    // Radii without a TMA kernel, or a tensor map the driver would not encode: the generic
    // streaming stencil (same results, slower); counted so that callers can tell.
    note_step(false, tp, vin_type, out_type, out_x, ckpt != nullptr, s32 != nullptr);
#define SFSEG_IT(TVI, TVO, TF, OX) \
    iterate_t<TVI, TVO, TF, OX>(vin, out, f, ckpt, g, tp, inv_alpha, p, acc_in, acc_out, flags, s, s32)
    // A step of the bf16 phase reads v and f in bf16 and writes bf16, or float32 when the next
    // step (or the caller's x) is float32; a float32 step reads and writes float32.
    (void)f_type;
    if (out_x) {   // the last step always writes float32 x~ into the caller's layout
        if (vin_type == kF32) SFSEG_IT(float, float, float, true);
        else SFSEG_IT(bf, float, bf, true);
    } else {
        if (vin_type == kF32) SFSEG_IT(float, float, float, false);
        else if (out_type == kBF16) SFSEG_IT(bf, bf, bf, false);
        else SFSEG_IT(bf, float, bf, false);
    }
#undef SFSEG_IT
}

void launch_apply(const float* x, int x_pitch, float* y, int y_pitch, const float* f32, Geom g,
                  const Taps& tp, float inv_alpha, float p, const double* acc_in, double* acc_out,
                  int* flags, cudaStream_t s, const float* s32) {
    OpApply op;
    op.sm = s32;
    op.x = x;
    op.x_pitch = x_pitch;
    op.f = f32;
    op.out = y;
    op.out_pitch = y_pitch;
    op.g = g;
    op.inv_alpha = inv_alpha;
    op.p = p;
    op.s = 1.f;
    run_stencil(op, tp, 16, acc_in, acc_out, nullptr, flags, s);
}

// v = u x from a caller-layout x into the internal layout (the state the iteration kernels read).
__global__ void to_state_kernel(const float* x, const float* f32, const float* s32, float p, Geom g, bool pairs,
                                float* v) {
    const float* sm = s32 ? s32 : f32;
    for_each_voxel_pairs(
        g, pairs,
        [&](int64_t i, int64_t j) {
            const float2 sv = ld2(sm + j), xv = ld2(x + i);
            st2(v + j, make_float2(unary_pow_fast(sv.x, p) * xv.x, unary_pow_fast(sv.y, p) * xv.y));
        },
        [&](int64_t i, int64_t j) { v[j] = unary_pow_fast(sm[j], p) * x[i]; });
}

void launch_to_state(const float* x, const float* f32, const float* s32, float p, Geom g, float* v, cudaStream_t s) {
    const RowLaunch rl = row_launch(g, num_sms());
    to_state_kernel<<<rl.blocks, rl.threads, 0, s>>>(x, f32, s32, p, g, g.W % 2 == 0 && aligned8(x), v);
    count_launches(1);
}

void launch_apply_user(const float* x, float* y, float* scratch_v, const float* f32, Geom g, const Taps& tp,
                       float inv_alpha, float p, int* flags, cudaStream_t s, const float* s32) {
    if (fast_iterate_supported(tp)) {
        const RowLaunch rl = row_launch(g, num_sms());
        to_state_kernel<<<rl.blocks, rl.threads, 0, s>>>(x, f32, s32, p, g, g.W % 2 == 0 && aligned8(x), scratch_v);
        count_launches(1);
        // one unscaled step (no norm input) that writes x~ = A x into the caller's layout
        if (launch_iterate_fast(scratch_v, kF32, y, kF32, true, f32, g, tp, inv_alpha, p, nullptr, nullptr, flags, s,
                                s32))
            return;
    }
    launch_apply(x, g.W, y, g.W, f32, g, tp, inv_alpha, p, nullptr, nullptr, flags, s, s32);
}

// -------------------------------------------------------------------------- Eq. 9 combine
template <typename TIn>
__global__ void combine_kernel(const TIn* feat, int C, Geom g, const float* w, float bias, float* f32,
                               __nv_bfloat16* fbf, int* flags, bool pairs) {
    const int64_t N = (int64_t)g.H * g.W * g.T;
    int bad = 0;
    auto one = [&](int64_t i) {
        if (C == 1) return ldf(feat + i);
        float z = bias;
        for (int c = 0; c < C; ++c) z = fmaf(w[c], ldf(feat + (int64_t)c * N + i), z);
        return 1.f / (1.f + expf(-z));
    };
    auto check = [&](float fv) {
        if (!(fv >= 0.f) || isinf(fv)) bad = 1;
    };
    for_each_voxel_pairs(
        g, pairs,
        [&](int64_t i, int64_t j) {
            float2 fv;
            if (C == 1) {
                fv = ld2(feat + i);
            } else {
                float2 z = make_float2(bias, bias);
                for (int c = 0; c < C; ++c) {
                    const float2 x = ld2(feat + (int64_t)c * N + i);
                    z.x = fmaf(w[c], x.x, z.x);
                    z.y = fmaf(w[c], x.y, z.y);
                }
                fv = make_float2(1.f / (1.f + expf(-z.x)), 1.f / (1.f + expf(-z.y)));
            }
            check(fv.x);
            check(fv.y);
            st2(f32 + j, fv);
            if (fbf) st2(fbf + j, fv);
        },
        [&](int64_t i, int64_t j) {
            const float fv = one(i);
            check(fv);
            f32[j] = fv;
            if (fbf) fbf[j] = __float2bfloat16_rn(fv);
        });
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, kFlagBadFeature);
}

void launch_combine(const void* feat, int feat_dtype, int C, Geom g, const float* w_dev, float bias,
                    float* f32, __nv_bfloat16* fbf, int* flags, cudaStream_t s) {
    const RowLaunch rl = row_launch(g, num_sms());
    // pairs of bf16 features need 4-byte alignment, of float32 8-byte, at every channel's start
    const int64_t N = (int64_t)g.H * g.W * g.T;
    const bool pairs = g.W % 2 == 0 && (feat_dtype == kF32 ? aligned8(feat) : ((uintptr_t)feat & 3) == 0) &&
                       (C == 1 || N % 2 == 0);
    if (feat_dtype == kF32)
        combine_kernel<float><<<rl.blocks, rl.threads, 0, s>>>((const float*)feat, C, g, w_dev, bias, f32, fbf,
                                                               flags, pairs);
    else
        combine_kernel<__nv_bfloat16><<<rl.blocks, rl.threads, 0, s>>>((const __nv_bfloat16*)feat, C, g, w_dev,
                                                                       bias, f32, fbf, flags, pairs);
    count_launches(1);
}

// ------------------------------------------------------------------------- start vector
template <typename TV>
__global__ void prologue_kernel(int init, const float* x_user, const float* f32, const float* s32, float p, Geom g,
                                TV* v0, float* x_copy, float* x_user_out, double* acc0, bool pairs) {
    float part = 0.f;
    const float* sm = s32 ? s32 : f32;
    for_each_voxel_pairs(
        g, pairs,
        [&](int64_t i, int64_t j) {
            const float2 sv = ld2(sm + j);
            const float2 x = init == 0 ? ld2(x_user + i) : (init == 1 ? make_float2(1.f, 1.f) : sv);
            part += x.x * x.x + x.y * x.y;
            st2(v0 + j, make_float2(unary_pow_fast(sv.x, p) * x.x, unary_pow_fast(sv.y, p) * x.y));
            if (x_copy) st2(x_copy + j, x);
            if (x_user_out) st2(x_user_out + i, x);
        },
        [&](int64_t i, int64_t j) {
            const float sv = sm[j];
            const float x = init == 0 ? x_user[i] : (init == 1 ? 1.f : sv);
            part += x * x;
            stf(v0 + j, unary_pow_fast(sv, p) * x);
            if (x_copy) x_copy[j] = x;
            if (x_user_out) x_user_out[i] = x;
        });
    const double b = block_sum((double)part);
    if (threadIdx.x == 0) atomicAdd(acc0, b);
}

void launch_prologue(int init, const float* x_user, const float* f32, float p, Geom g, void* v0, int vtype,
                     float* x_copy, float* x_user_out, double* acc0, cudaStream_t s, const float* s32) {
    const RowLaunch rl = row_launch(g, num_sms(), 8);
    const bool pairs = g.W % 2 == 0 && aligned8(init == 0 ? x_user : nullptr, x_user_out);
    if (vtype == kF32)
        prologue_kernel<float><<<rl.blocks, rl.threads, 0, s>>>(init, x_user, f32, s32, p, g, (float*)v0, x_copy,
                                                                x_user_out, acc0, pairs);
    else
        prologue_kernel<__nv_bfloat16><<<rl.blocks, rl.threads, 0, s>>>(init, x_user, f32, s32, p, g,
                                                                        (__nv_bfloat16*)v0, x_copy, x_user_out, acc0,
                                                                        pairs);
    count_launches(1);
}

__global__ void to_bf16_kernel(const float* a, __nv_bfloat16* b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = __float2bfloat16_rn(a[i]);
}

void launch_to_bf16(const float* a, __nv_bfloat16* b, int64_t n, cudaStream_t s) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 16 * num_sms()) blocks = 16 * num_sms();
    to_bf16_kernel<<<blocks, 256, 0, s>>>(a, b, n); count_launches(1);
}

// ------------------------------------------------------------------------- reductions
__global__ void scale_inv_norm_kernel(float* x, int64_t n, bool vec, const double* acc, int* flags) {
    const float s = inv_norm_from(acc, flags);
    for_each_flat(
        n, vec,
        [&](int64_t i) {
            float4 v = reinterpret_cast<float4*>(x)[i];
            v.x *= s, v.y *= s, v.z *= s, v.w *= s;
            reinterpret_cast<float4*>(x)[i] = v;
        },
        [&](int64_t i) { x[i] *= s; });
}

void launch_scale_inv_norm(float* x, int64_t n, const double* acc, int* flags, cudaStream_t s) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 8 * num_sms()) blocks = 8 * num_sms();
    scale_inv_norm_kernel<<<blocks, 256, 0, s>>>(x, n, aligned16(x), acc, flags); count_launches(1);
}

__global__ void dot2_kernel(const float* x, const float* y, int64_t n, bool vec, double* acc) {
    float a = 0.f, b = 0.f;
    for_each_flat(
        n, vec,
        [&](int64_t i) {
            const float4 p = reinterpret_cast<const float4*>(x)[i], q = reinterpret_cast<const float4*>(y)[i];
            a += p.x * q.x + p.y * q.y + p.z * q.z + p.w * q.w;
            b += p.x * p.x + p.y * p.y + p.z * p.z + p.w * p.w;
        },
        [&](int64_t i) {
            a += x[i] * y[i];
            b += x[i] * x[i];
        });
    const double sa = block_sum((double)a);
    if (threadIdx.x == 0) atomicAdd(acc, sa);
    const double sb = block_sum((double)b);
    if (threadIdx.x == 0) atomicAdd(acc + 1, sb);
}

__global__ void resid_kernel(const float* x, const float* y, int64_t n, bool vec, double* acc) {
    const float rho = (float)(acc[0] / acc[1]);
    float a = 0.f;
    for_each_flat(
        n, vec,
        [&](int64_t i) {
            const float4 p = reinterpret_cast<const float4*>(x)[i], q = reinterpret_cast<const float4*>(y)[i];
            const float d0 = q.x - rho * p.x, d1 = q.y - rho * p.y, d2 = q.z - rho * p.z, d3 = q.w - rho * p.w;
            a += d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3;
        },
        [&](int64_t i) {
            const float d = y[i] - rho * x[i];
            a += d * d;
        });
    const double sa = block_sum((double)a);
    if (threadIdx.x == 0) atomicAdd(acc + 2, sa);
}

__global__ void sumsq_kernel(const float* x, int64_t n, bool vec, double* acc) {
    float a = 0.f;
    for_each_flat(
        n, vec,
        [&](int64_t i) {
            const float4 p = reinterpret_cast<const float4*>(x)[i];
            a = fmaf(p.x, p.x, fmaf(p.y, p.y, fmaf(p.z, p.z, fmaf(p.w, p.w, a))));
        },
        [&](int64_t i) { a = fmaf(x[i], x[i], a); });
    const double sa = block_sum((double)a);
    if (threadIdx.x == 0) atomicAdd(acc, sa);
}

void launch_sumsq(const float* x, int64_t n, double* acc, cudaStream_t s) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 8 * num_sms()) blocks = 8 * num_sms();
    if (blocks < 1) blocks = 1;
    sumsq_kernel<<<blocks, 256, 0, s>>>(x, n, aligned16(x), acc); count_launches(1);
}

void launch_dot2(const float* x, const float* y, int64_t n, double* acc, cudaStream_t s) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 8 * num_sms()) blocks = 8 * num_sms();
    dot2_kernel<<<blocks, 256, 0, s>>>(x, y, n, aligned16(x, y), acc); count_launches(1);
}

void launch_resid(const float* x, const float* y, int64_t n, double* acc, cudaStream_t s) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 8 * num_sms()) blocks = 8 * num_sms();
    resid_kernel<<<blocks, 256, 0, s>>>(x, y, n, aligned16(x, y), acc); count_launches(1);
}

}  // namespace sfseg
