// launch.h -- host-side launchers of the sfseg kernels (internal to libsfseg.so).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

struct sfseg_handle;
struct sfseg_neighborhood;

namespace sfseg {

enum StoreType { kF32 = 0, kBF16 = 1 };

// Eq. 9 / Alg. 1 lines 1-2: features [C][T][H][W] (caller layout) -> f (internal pitch), in
// float32 and, when fbf != nullptr, also in bf16.
void launch_combine(const void* feat, int feat_dtype, int C, Geom g, const float* w_dev, float bias,
                    float* f32, __nv_bfloat16* fbf, int* flags, cudaStream_t s);

// Start vector (Alg. 1 line 3 or uniform or the caller's x): writes v0 = u x0 (internal, in
// `vtype`), acc[0] = ||x0||^2, and optionally an FP32 copy of x0 (internal pitch) and x0 into
// the caller's layout.
// With separate unary maps (s32 != nullptr, internal layout) u = s^p and the S_m start is s.
void launch_prologue(int init, const float* x_user, const float* f32, float p, Geom g, void* v0,
                     int vtype, float* x_copy, float* x_user_out, double* acc0, cudaStream_t s,
                     const float* s32 = nullptr);

// One Eq. 7 power-iteration step in the scaled, u-weighted form (see kernels_generic.cu):
// input v_k = u x~_k (internal), output v_{k+1} = u x~_{k+1} or, when `out_x`, x~_{k+1} itself
// in the caller's layout (pitch W).  acc_in = ||x~_k||^2, acc_out += ||x~_{k+1}||^2.
// `ckpt` (nullable) receives an FP32 copy of x~_{k+1} in internal layout.
void launch_iterate(const void* vin, int vin_type, void* out, int out_type, bool out_x,
                    const void* f, int f_type, float* ckpt, Geom g, const Taps& tp,
                    float inv_alpha, float p, const double* acc_in, double* acc_out, int* flags,
                    cudaStream_t s, const float* s32 = nullptr);

// TMA-staged step for the radii with a compiled kernel (kernels_fast.cu).  s32
// (nullable): a separate unary map (float32 storage only).  Returns false when the radius has no
// compiled kernel or a tensor map cannot be encoded; nothing is launched then.
bool fast_iterate_supported(const Taps& tp);
bool launch_iterate_fast(const void* vin, int vin_type, void* out, int out_type, bool out_x, const void* f,
                         const Geom& g, const Taps& tp, float inv_alpha, float p, const double* acc_in,
                         double* acc_out, int* flags, cudaStream_t s, const float* s32 = nullptr);

// The TMA step from the state vin (internal layout, float32) to y = A x in the caller layout that
// also adds the order key of its largest output to *maxkey (atomicMax; zero it first): a
// soft-binarisation step's maximum without a pass of its own.  No norm scaling.  False (nothing
// launched) for a radius without a compiled kernel.
bool launch_iterate_fast_max(const float* vin, float* y, const float* f, const Geom& g, const Taps& tp,
                             float inv_alpha, float p, unsigned* maxkey, int* flags, cudaStream_t s);

// v = u x (internal layout) for a caller-layout x, u = s^p with s the unary map (s32, or f32).
void launch_to_state(const float* x, const float* f32, const float* s32, float p, Geom g, float* v, cudaStream_t s);

// The TMA step that also records x~_{k+1} (internal layout) into ckpt, float32 storage; false
// (nothing launched) for a radius without a compiled kernel.
bool launch_iterate_fast_ckpt(const float* vin, void* out, bool out_x, const float* f, const Geom& g, const Taps& tp,
                              float inv_alpha, float p, const double* acc_in, double* acc_out, float* ckpt, int* flags,
                              cudaStream_t s);

// The adjoint's Q-pass on the TMA kernel (kernels_fast.cu, mode 1), float32, internal layout:
// for the signals c0, c1, c2 of v (G*v, G*(f^2 v), G*(f v)), writes Q = s (a1 c0 - p c1 + a3 c2)
// to out, s = 1/sqrt(*acc_in) (or 1).  Returns false (nothing launched) for another mode or a
// radius without a compiled kernel.
bool launch_filter_fast(const float* vin, int mode, float* out, float* out2, const float* f, const Geom& g,
                        const Taps& tp, float inv_alpha, float p, const double* acc_in, int* flags, cudaStream_t s);

// One term j of the exact (Eq. 1) kernel's series on the TMA kernel (kernels_fast.cu, mode 7):
// for the input v = f^{3j} w (internal layout), adds the terms n = 3j, 3j+1, 3j+2 of
// sum_n c_n f^n G*(f^n w) to y (writes them when j = 0); on the last term multiplies the sum by
// u e^{-alpha f^2} / alpha and adds ||y||^2 to *acc_out (nullable).  Returns false for a radius
// without a compiled kernel.
struct ExactTerm {
    int j, last;
    float c[3];     // c_{3j}, c_{3j+1}, c_{3j+2}, c_n = (2 alpha)^n / n! (0 beyond the last term)
    float alpha;
};
bool launch_exact_term_fast(const float* v, float* y, const float* f, const Geom& g, const Taps& tp, float inv_alpha,
                            float p, const ExactTerm& ex, double* acc_out, int* flags, cudaStream_t s);

// The exact kernel's element-wise parts (kernels_exact.cu, internal layout unless noted): x~ from
// the caller's x (or 1 everywhere for a null x_user) with acc += ||x~||^2 (nullable); the input
// of term group j, v = f^{3j} s u e^{-alpha f^2} x~ with s = 1/sqrt(*acc) (or 1); and the
// caller's x = s y.
void launch_exact_in(const float* x_user, Geom g, float* xt, double* acc, cudaStream_t s);
void launch_exact_prep(const float* xt, const double* acc, const float* f32, float alpha, float p, int jt, Geom g,
                       float* v, int* flags, cudaStream_t s);
void launch_exact_out(const float* y, const double* acc, Geom g, float* x_user, int* flags, cudaStream_t s);

// The adjoint's recomputing step with its Q-pass (kernels_fast.cu, mode 6): from the state V_k
// (internal layout, s = 1/sqrt(*acc_in)) writes the next state to vout exactly as the plain step
// does, and Q = s (a1 c0 - p c1 + a3 c2) of the same filtered signals to Q.  Returns false for a
// radius without a compiled kernel.
bool launch_step_q_fast(const float* vin, float* vout, float* Q, const float* f, const Geom& g, const Taps& tp,
                        float inv_alpha, float p, const double* acc_in, int* flags, cudaStream_t s);

// The adjoint's g-pass in state form (kernels_fast.cu, mode 5): for v_g = u g_y, writes
// G = u A g_y = u^2 B to G and Q (unscaled) to Qg, and adds sum V_k B to *dot (V_k = u x~_k,
// internal layout; <x_k, A g_y> = dot / ||x~_k||).  Returns false for a radius without a
// compiled kernel.
bool launch_adjoint_gpass_fast(const float* vg, float* G, float* Qg, const float* Vk, const float* f, const Geom& g,
                               const Taps& tp, float inv_alpha, float p, double* dot, int* flags, cudaStream_t s);

// y = s * A x in the plain (x-space) form: x with pitch x_pitch, y with pitch y_pitch, FP32
// features; s = 1/sqrt(*acc_in) (or 1 if acc_in is null); acc_out += ||y||^2 (nullable).
void launch_apply(const float* x, int x_pitch, float* y, int y_pitch, const float* f32, Geom g,
                  const Taps& tp, float inv_alpha, float p, const double* acc_in, double* acc_out,
                  int* flags, cudaStream_t s, const float* s32 = nullptr);

// bf16 copy of a float32 array (n elements).
void launch_to_bf16(const float* a, __nv_bfloat16* b, int64_t n, cudaStream_t s);

// y = A x for caller-layout x and y (FP32); scratch_v holds one internal-layout volume.  Uses
// the TMA kernel for the radii it serves, the generic stencil otherwise.
void launch_apply_user(const float* x, float* y, float* scratch_v, const float* f32, Geom g, const Taps& tp,
                       float inv_alpha, float p, int* flags, cudaStream_t s, const float* s32 = nullptr);

// Restriction of f (internal layout) by (pt, ph, pw) into a caller-layout coarse volume, and
// trilinear prolongation of a caller-layout coarse x (kernels_multilevel.cu).
void launch_pool_f(const float* f, Geom g, int pt, int ph, int pw, int Tc, int Hc, int Wc, float* out, cudaStream_t s);
void launch_upsample(const float* xc, int Tc, int Hc, int Wc, int pt, int ph, int pw, int T, int H, int W, float* x,
                     cudaStream_t s);
// x /= max(x) over n caller-layout values (key: one unsigned of scratch).
void launch_scale_by_max(float* x, int64_t n, unsigned* key, cudaStream_t s);

// Soft-binarisation step pieces (kernels_tail.cu): *key = order-preserving key of max(y) over
// n caller-layout values (the key is reset first); x = sigmoid(gain (y / max y - center)) with
// optional v = u * x (internal layout) and mask = (x > 1/2).
void launch_max_key(const float* y, int64_t n, unsigned* key, cudaStream_t s);
void launch_sigmoid_step(const float* y, const unsigned* key, float gain, float center, const float* f32, float p,
                         Geom g, float* x, float* v, unsigned char* mask, int* flags, cudaStream_t s,
                         const float* s32 = nullptr);

// Online stream support (api.cu): shift the handle's combined features one frame towards t = 0
// and combine a caller-layout frame [C][H][W] into the last frame.
int handle_push_frame(sfseg_handle* h, const void* frame, int dtype, const float* weights, float bias,
                      cudaStream_t s);

// Bounded-wait self-test (selftest.cu): waits `spins` times on an mbarrier nothing completes,
// then raises kFlagTimeout.
void launch_wait_probe(long long spins, int* flags, cudaStream_t s);

// x *= 1/sqrt(*acc) over a caller-layout volume.
void launch_scale_inv_norm(float* x, int64_t n, const double* acc, int* flags, cudaStream_t s);

// acc[0] += sum x*x over n elements (FP64 block sums)
void launch_sumsq(const float* x, int64_t n, double* acc, cudaStream_t s);
// acc[0] += sum x*y, acc[1] += sum x*x  (x, y caller layout, n elements)
void launch_dot2(const float* x, const float* y, int64_t n, double* acc, cudaStream_t s);
// acc[2] += sum (y - rho x)^2 with rho = acc[0] / acc[1]
void launch_resid(const float* x, const float* y, int64_t n, double* acc, cudaStream_t s);

// Backward (adjoint) pieces, see kernels_bwd.cu.
void launch_grad_in(const float* gx_user, const float* xK, const double* accK, float* g_out, Geom g,
                    double* dot_out, cudaStream_t s);
void launch_adjoint_step(const float* xk, const double* acc_k, const float* xn, const double* acc_n,
                         const float* gn, const double* dot_n, float* gk_out, double* dot_k,
                         float* gz, const float* f32, Geom g, const Taps& tp, float inv_alpha,
                         float p, cudaStream_t s);
// The reverse step in the stencil's state form (kernels_bwd.cu; V_k = u x~_k, G_k = u g_k,
// v_g = u g_y, all internal layout): the first step's v_g from x~_K, g_K and <x_K, g_K>; the
// element-wise pass after the g-pass (gz += (1 - f)(v_g Q_x + s_k V_k Q_g), and the next v_g
// when vg_next is not null); and V = u x~ for a recomputed segment's checkpoint.
void launch_adjoint_first(const float* xK, const double* accK, const float* gK, const double* dotK,
                          const float* f32, float p, Geom g, float* vg, cudaStream_t s);
void launch_adjoint_combine_state(const float* f32, const float* vg, const float* qx, const float* Vk,
                                  const float* qg, const float* Gk, const double* acc_k, const double* dsum, Geom g,
                                  float* gz, float* vg_next, cudaStream_t s);
void launch_state_internal(const float* x, const float* f32, float p, Geom g, float* v, cudaStream_t s);
void launch_weight_grad(const void* feat, int feat_dtype, int C, Geom g, const float* gz,
                        double* acc_c_plus_1, cudaStream_t s);
void launch_soft_iou(const float* x, const float* tgt, int64_t n, float* grad, double* acc,
                     unsigned long long* amax, cudaStream_t s);

int num_sms();

// Bit of the current device in a per-call-site mask: kernel attributes (the dynamic shared-memory
// size) are set per device, so a process that drives several GPUs sets them on each.
inline unsigned long long device_bit() {
    int dev = 0;
    cudaGetDevice(&dev);
    return 1ull << (dev & 63);
}

// Validates a neighbourhood (radius limits; sigma finite and > 0 where its radius is > 0) and
// fills the three 1D Gaussian tap arrays exp(-d^2 / (2 sigma^2)), d = -r..r (all 1 at r = 0).
// Returns SFSEG_OK, or INVALID_ARG / SHAPE with the thread's last-error message set (api.cu).
int make_taps(const sfseg_neighborhood* nb, Taps* tp);

// Records `msg` as the thread's sfseg_last_error() text and returns `code`.
int set_last_error(int code, const char* msg);

// Process-wide counts of power-iteration steps issued on the TMA kernel and on the generic
// stencil, and the kernel name of the last one (sfseg_iterate_kernel_stats).
void iterate_kernel_stats(int64_t* tma_steps, int64_t* generic_steps, char* name, int len);

// Process-wide count of kernels launched by the library (sfseg_kernel_launches).
void count_launches(int n);
int64_t launches_so_far();

}  // namespace sfseg
