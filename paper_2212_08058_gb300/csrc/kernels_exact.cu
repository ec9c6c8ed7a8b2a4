// kernels_exact.cu -- the element-wise parts of the exact (Eq. 1) kernel's operator, the
// diagnostic of the first-order approximation (Sec. 4.3): M_ij = u_i u_j exp(-a (f_i - f_j)^2) G_ij
// written as the series e^{-a f_i^2} e^{-a f_j^2} sum_n c_n f_i^n f_j^n, c_n = (2a)^n / n!, whose
// terms are separable and go through the TMA stencil three at a time (kernels_fast.cu, mode 7).
// Here: the iterate into the internal layout, the input v = f^{3j} w of term group j with
// w = s u e^{-a f^2} x~, and the result back into the caller's layout.
#include "launch.h"
#include "voxels.cuh"

namespace sfseg {

// x~ (internal) = the caller's x, or 1 everywhere (x_user null); acc += ||x~||^2.
__global__ void exact_in_kernel(const float* x_user, Geom g, float* xt, double* acc) {
    float part = 0.f;
    for_each_voxel(g, [&](int64_t i, int64_t j) {
        const float v = x_user ? x_user[i] : 1.f;
        xt[j] = v;
        part += v * v;
    });
    const double b = block_sum((double)part);
    if (threadIdx.x == 0 && acc) atomicAdd(acc, b);
}

// v = f^{3j} s u e^{-a f^2} x~, s = 1/sqrt(*acc) (1 if acc is null).
__global__ void exact_prep_kernel(const float* xt, const double* acc, const float* f, float alpha, float p, int jt,
                                  Geom g, float* v, int* flags) {
    const float s = inv_norm_from(acc, flags);
    for_each_voxel(g, [&](int64_t, int64_t j) {
        const float fv = f[j];
        const float f3 = fv * fv * fv;
        float F = 1.f;
        for (int i = 0; i < jt; ++i) F *= f3;
        v[j] = F * (s * unary_pow_fast(fv, p) * expf(-alpha * fv * fv) * xt[j]);
    });
}

// The caller's x = s y (y internal), s = 1/sqrt(*acc) (1 if acc is null).
__global__ void exact_out_kernel(const float* y, const double* acc, Geom g, float* x_user, int* flags) {
    const float s = inv_norm_from(acc, flags);
    for_each_voxel(g, [&](int64_t i, int64_t j) { x_user[i] = s * y[j]; });
}

void launch_exact_in(const float* x_user, Geom g, float* xt, double* acc, cudaStream_t s) {
    const RowLaunch rl = row_launch(g, num_sms());
    exact_in_kernel<<<rl.blocks, rl.threads, 0, s>>>(x_user, g, xt, acc);
    count_launches(1);
}

void launch_exact_prep(const float* xt, const double* acc, const float* f32, float alpha, float p, int jt, Geom g,
                       float* v, int* flags, cudaStream_t s) {
    const RowLaunch rl = row_launch(g, num_sms());
    exact_prep_kernel<<<rl.blocks, rl.threads, 0, s>>>(xt, acc, f32, alpha, p, jt, g, v, flags);
    count_launches(1);
}

void launch_exact_out(const float* y, const double* acc, Geom g, float* x_user, int* flags, cudaStream_t s) {
    const RowLaunch rl = row_launch(g, num_sms());
    exact_out_kernel<<<rl.blocks, rl.threads, 0, s>>>(y, acc, g, x_user, flags);
    count_launches(1);
}

}  // namespace sfseg
