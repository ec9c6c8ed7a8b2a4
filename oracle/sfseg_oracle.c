/*
 * sfseg_oracle.c -- plain FP64 CPU oracle for the SFSeg / SFSeg++ power iteration
 * (Burceanu & Leordeanu, arXiv 2212.08058).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call this file:
 * only the test suite, the smoke check and the benchmark's CPU-baseline leg use it.  It shares
 * no code, header, table or constant with the CUDA library.
 *
 * Conventions
 *   - A volume has T frames of H x W pixels; node i = (t*H + h)*W + w  (w fastest).
 *   - Everything is double precision.  Summations that decide a norm use pairwise summation.
 *   - The neighbourhood of node i is the box |dt|<=rt, |dh|<=rh, |dw|<=rw that lies inside the
 *     volume, i itself included (zero padding: a missing neighbour is a missing edge).
 *   - The spatial Gaussian is exp(-beta * dist^2) with beta*dist^2 = 0.5*(dt^2/st^2 + dh^2/sh^2
 *     + dw^2/sw^2): the isotropic beta = 1/(2 sigma^2) of Eq. 1 when st = sh = sw = sigma,
 *     unnormalised (value 1 at distance 0).  An axis with radius 0 contributes a factor 1.
 *   - Unary term u_i = s_i^p with 0^p := 0.
 *
 * Functions follow the paper's definitions in order:
 *   orc_combine          Eq. 9 (sigmoid channel combination; single channel passes through)
 *   orc_build_affinity   Eq. 2 (first-order Taylor affinity; Eq. 1 with exact != 0), as CSR
 *   orc_spmv / orc_power_csr   Eq. 4 power iteration with the Eq. 8 renormalisation
 *   orc_filter_apply / orc_power_filter   Eq. 7 (three separable Gaussian filterings)
 *   orc_grad_csr         reverse-mode derivative of the loss through K steps of Eq. 4 + Eq. 8
 *                        with respect to the Eq. 9 channel weights (Sec. 3.4 learning)
 *   orc_conv3d_fwd/bwd   plain 3x3x3 convolution loops for the warm-start network
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Pairwise (cascade) summation of a[0..n): error O(log n * eps) instead of O(n * eps). */
static double pairwise_sum(const double* a, int64_t n) {
    if (n <= 64) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += a[i];
        return s;
    }
    int64_t m = n / 2;
    return pairwise_sum(a, m) + pairwise_sum(a + m, n - m);
}

/* Sum of squares, pairwise; the squares are formed into a temporary. */
double orc_sumsq(const double* x, int64_t n) {
    double* tmp = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    for (int64_t i = 0; i < n; ++i) tmp[i] = x[i] * x[i];
    double s = pairwise_sum(tmp, n);
    free(tmp);
    return s;
}

double orc_dot(const double* x, const double* y, int64_t n) {
    double* tmp = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    for (int64_t i = 0; i < n; ++i) tmp[i] = x[i] * y[i];
    double s = pairwise_sum(tmp, n);
    free(tmp);
    return s;
}

/* Eq. 9: S_m = F_m = sigma(sum_c w_c V_c + b) with the standard logistic sigma(z) = 1/(1+e^-z).
 * Alg. 1 (initialisation note): with a single channel the map is used directly, no sigmoid. */
void orc_combine(int64_t C, int64_t N, const double* V, const double* w, double b, double* f) {
    if (C == 1) {
        memcpy(f, V, (size_t)N * sizeof(double));
        return;
    }
    for (int64_t i = 0; i < N; ++i) {
        double z = b;
        for (int64_t c = 0; c < C; ++c) z += w[c] * V[c * N + i];
        f[i] = 1.0 / (1.0 + exp(-z));
    }
}

/* 1D factor of the Gaussian: g[d + r] = exp(-d^2 / (2 sigma^2)), d in [-r, r]. */
void orc_taps(int r, double sigma, double* g) {
    for (int d = -r; d <= r; ++d) g[d + r] = (r == 0) ? 1.0 : exp(-(double)(d * d) / (2.0 * sigma * sigma));
}

static double unary(double s, double p) { return s > 0.0 ? pow(s, p) : 0.0; }

/* Eq. 2 (exact == 0) or Eq. 1 (exact != 0): explicit sparse adjacency in CSR form.
 *   M_ij = u_i u_j [1 - alpha (f_i - f_j)^2] G_ij          (Eq. 2)
 *   M_ij = u_i u_j exp(-alpha (f_i - f_j)^2)  G_ij          (Eq. 1)
 * with G_ij = exp(-0.5 (dt^2/st^2 + dh^2/sh^2 + dw^2/sw^2)) evaluated from the distance itself
 * (not from the product of 1D factors, so that this is an independent writing of the definition).
 * Columns of a row are ascending.  rowptr has N+1 entries; col/val must hold
 * N * (2rt+1)(2rh+1)(2rw+1) entries.  Returns nnz. */
int64_t orc_build_affinity(int T, int H, int W, const double* s, const double* f, double p, double alpha,
                           int rt, int rh, int rw, double st, double sh, double sw, int exact,
                           int64_t* rowptr, int64_t* col, double* val) {
    int64_t N = (int64_t)T * H * W;
    int64_t nnz = 0;
    rowptr[0] = 0;
    for (int64_t i = 0; i < N; ++i) {
        int t = (int)(i / ((int64_t)H * W));
        int h = (int)((i / W) % H);
        int w = (int)(i % W);
        double ui = unary(s[i], p);
        for (int dt = -rt; dt <= rt; ++dt) {
            int tj = t + dt;
            if (tj < 0 || tj >= T) continue;
            for (int dh = -rh; dh <= rh; ++dh) {
                int hj = h + dh;
                if (hj < 0 || hj >= H) continue;
                for (int dw = -rw; dw <= rw; ++dw) {
                    int wj = w + dw;
                    if (wj < 0 || wj >= W) continue;
                    int64_t j = ((int64_t)tj * H + hj) * W + wj;
                    double q = 0.0;
                    if (rt > 0) q += (double)(dt * dt) / (st * st);
                    if (rh > 0) q += (double)(dh * dh) / (sh * sh);
                    if (rw > 0) q += (double)(dw * dw) / (sw * sw);
                    double G = exp(-0.5 * q);
                    double df = f[i] - f[j];
                    double pair = exact ? exp(-alpha * df * df) : (1.0 - alpha * df * df);
                    col[nnz] = j;
                    val[nnz] = ui * unary(s[j], p) * pair * G;
                    ++nnz;
                }
            }
        }
        rowptr[i + 1] = nnz;
    }
    return nnz;
}

/* y = M x (Eq. 4 right-hand side). */
void orc_spmv(int64_t N, const int64_t* rowptr, const int64_t* col, const double* val,
              const double* x, double* y) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double acc = 0.0;
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) acc += val[e] * x[col[e]];
        y[i] = acc;
    }
}

/* Eq. 4 + Eq. 8: K steps x <- M x / ||M x||_2, from x0 / ||x0||_2.
 * nu_out[k] = ||M x_k|| for k = 0..K-1 (may be NULL).  Returns 0, or -1 on a zero norm. */
int orc_power_csr(int64_t N, const int64_t* rowptr, const int64_t* col, const double* val,
                  const double* x0, int K, double* x_out, double* nu_out) {
    double* y = (double*)malloc((size_t)N * sizeof(double));
    double n0 = sqrt(orc_sumsq(x0, N));
    if (!(n0 > 0.0)) { free(y); return -1; }
    for (int64_t i = 0; i < N; ++i) x_out[i] = x0[i] / n0;
    for (int k = 0; k < K; ++k) {
        orc_spmv(N, rowptr, col, val, x_out, y);
        double nu = sqrt(orc_sumsq(y, N));
        if (nu_out) nu_out[k] = nu;
        if (!(nu > 0.0)) { free(y); return -1; }
        for (int64_t i = 0; i < N; ++i) x_out[i] = y[i] / nu;
    }
    free(y);
    return 0;
}

/* One 1D zero-padded correlation along an axis of a T x H x W volume.
 * axis 0 = t, 1 = h, 2 = w.  The Gaussian factor is even, so correlation == convolution.
 * Taps that fall outside the volume are skipped (zero padding); the valid tap range of each
 * output is computed once, and the taps are summed in increasing offset order. */
static void filter_axis(int T, int H, int W, int axis, int r, const double* g, const double* in, double* out) {
    int64_t HW = (int64_t)H * W;
    int64_t step = axis == 0 ? HW : (axis == 1 ? W : 1);
    int n = axis == 0 ? T : (axis == 1 ? H : W);
#pragma omp parallel for collapse(2) schedule(static)
    for (int t = 0; t < T; ++t) {
        for (int h = 0; h < H; ++h) {
            for (int w = 0; w < W; ++w) {
                int pos = axis == 0 ? t : (axis == 1 ? h : w);
                int lo = pos - r < 0 ? -pos : -r;
                int hi = pos + r > n - 1 ? n - 1 - pos : r;
                const double* src = in + (int64_t)t * HW + (int64_t)h * W + w;
                double acc = 0.0;
                for (int d = lo; d <= hi; ++d) acc += g[d + r] * src[d * step];
                out[(int64_t)t * HW + (int64_t)h * W + w] = acc;
            }
        }
    }
}

/* G_3D * v for the separable box-truncated Gaussian: three 1D passes (Sec. 4.2). */
static void gauss3d(int T, int H, int W, int rt, int rh, int rw, double st, double sh, double sw,
                    const double* in, double* out, double* tmp) {
    double gt[64], gh[64], gw[64];
    orc_taps(rt, st, gt);
    orc_taps(rh, sh, gh);
    orc_taps(rw, sw, gw);
    filter_axis(T, H, W, 2, rw, gw, in, out);
    filter_axis(T, H, W, 1, rh, gh, out, tmp);
    filter_axis(T, H, W, 0, rt, gt, tmp, out);
}

/* Eq. 7: y = S^p (1/alpha - F^2) G*(S^p X) - S^p G*(F^2 S^p X) + 2 S^p F G*(F S^p X).
 * This equals M x / alpha for the Eq. 2 matrix (Eq. 6 carries a leading alpha that Eq. 7 drops).
 * Radii must be < 32. */
void orc_filter_apply(int T, int H, int W, const double* s, const double* f, double p, double alpha,
                      int rt, int rh, int rw, double st, double sh, double sw,
                      const double* x, double* y) {
    int64_t N = (int64_t)T * H * W;
    double* u = (double*)malloc((size_t)N * sizeof(double));
    double* z = (double*)malloc((size_t)N * sizeof(double));
    double* c1 = (double*)malloc((size_t)N * sizeof(double));
    double* c2 = (double*)malloc((size_t)N * sizeof(double));
    double* c3 = (double*)malloc((size_t)N * sizeof(double));
    double* tmp = (double*)malloc((size_t)N * sizeof(double));
    for (int64_t i = 0; i < N; ++i) u[i] = unary(s[i], p);
    /* c1 = G * (S^p X) */
    for (int64_t i = 0; i < N; ++i) z[i] = u[i] * x[i];
    gauss3d(T, H, W, rt, rh, rw, st, sh, sw, z, c1, tmp);
    /* c2 = G * (F^2 S^p X) */
    for (int64_t i = 0; i < N; ++i) z[i] = f[i] * f[i] * u[i] * x[i];
    gauss3d(T, H, W, rt, rh, rw, st, sh, sw, z, c2, tmp);
    /* c3 = G * (F S^p X) */
    for (int64_t i = 0; i < N; ++i) z[i] = f[i] * u[i] * x[i];
    gauss3d(T, H, W, rt, rh, rw, st, sh, sw, z, c3, tmp);
    for (int64_t i = 0; i < N; ++i)
        y[i] = u[i] * (1.0 / alpha - f[i] * f[i]) * c1[i] - u[i] * c2[i] + 2.0 * u[i] * f[i] * c3[i];
    free(u); free(z); free(c1); free(c2); free(c3); free(tmp);
}

/* Eq. 7 + Eq. 8 iterated K times from x0 / ||x0||.  nu_out[k] = ||A x_k|| (A = M / alpha). */
int orc_power_filter(int T, int H, int W, const double* s, const double* f, double p, double alpha,
                     int rt, int rh, int rw, double st, double sh, double sw,
                     const double* x0, int K, double* x_out, double* nu_out) {
    int64_t N = (int64_t)T * H * W;
    double* y = (double*)malloc((size_t)N * sizeof(double));
    double n0 = sqrt(orc_sumsq(x0, N));
    if (!(n0 > 0.0)) { free(y); return -1; }
    for (int64_t i = 0; i < N; ++i) x_out[i] = x0[i] / n0;
    for (int k = 0; k < K; ++k) {
        orc_filter_apply(T, H, W, s, f, p, alpha, rt, rh, rw, st, sh, sw, x_out, y);
        double nu = sqrt(orc_sumsq(y, N));
        if (nu_out) nu_out[k] = nu;
        if (!(nu > 0.0)) { free(y); return -1; }
        for (int64_t i = 0; i < N; ++i) x_out[i] = y[i] / nu;
    }
    free(y);
    return 0;
}

/* Soft-binarisation iterations (Alg. 1 step 3, Sec. 4.1): after the continuous iterations,
 * each further step applies the Eq. 7 operator and then a sigmoid that pushes the solution
 * towards {0, 1}.  Reading taken here (the paper names only "a sigmoid controlled by a
 * parameter"): the new vector is first scaled to maximum 1, then
 *     x <- 1 / (1 + exp(-gain (y / max(y) - center))),   y = A x,
 * so the gain and the centre act on a [0, 1] scale whatever the size of the volume.  K steps
 * from x0 (any positive scale).  Returns 0, or -1 if max(y) <= 0 in some step. */
int orc_soft_binarize(int T, int H, int W, const double* s, const double* f, double p, double alpha,
                      int rt, int rh, int rw, double st, double sh, double sw,
                      const double* x0, int K, double gain, double center, double* x_out) {
    int64_t N = (int64_t)T * H * W;
    double* y = (double*)malloc((size_t)N * sizeof(double));
    for (int64_t i = 0; i < N; ++i) x_out[i] = x0[i];
    for (int k = 0; k < K; ++k) {
        orc_filter_apply(T, H, W, s, f, p, alpha, rt, rh, rw, st, sh, sw, x_out, y);
        double m = y[0];
        for (int64_t i = 1; i < N; ++i) m = y[i] > m ? y[i] : m;
        if (!(m > 0.0)) { free(y); return -1; }
        for (int64_t i = 0; i < N; ++i) x_out[i] = 1.0 / (1.0 + exp(-gain * (y[i] / m - center)));
    }
    free(y);
    return 0;
}

/* Partial derivative of the Eq. 2 pair kernel k(a, b) = a^p b^p (1 - alpha (a - b)^2) with
 * respect to its first argument (a > 0 required when p < 1). */
static double dk_da(double a, double b, double p, double alpha) {
    double ua = pow(a, p), ub = b > 0.0 ? pow(b, p) : 0.0;
    double d = a - b;
    return p * pow(a, p - 1.0) * ub * (1.0 - alpha * d * d) - 2.0 * alpha * ua * ub * d;
}

/* Reverse-mode gradient of a loss L(x_K) with respect to the Eq. 9 weights w[0..C) and bias b,
 * where f = sigma(sum_c w_c V_c + b), M = M(f) from Eq. 2 (S = F shared, Sec. 5 setup), and
 * x_{k+1} = M x_k / ||M x_k||, x_0 = x0/||x0|| independent of w.  gK = dL/dx_K.
 * Recurrence (per step, A symmetric):
 *   g_y  = (g_{k+1} - x_{k+1} <x_{k+1}, g_{k+1}>) / nu_{k+1}
 *   g_f += sum_ij g_y,i x_k,j dM_ij/df
 *   g_k  = M g_y
 * then dL/dz = g_f f (1-f), dL/dw_c = sum_i dL/dz_i V_c,i, dL/db = sum_i dL/dz_i.
 * C must be > 1 (the single-channel map has no weights).  Returns 0 or -1. */
int orc_grad_csr(int T, int H, int W, int C, const double* V, const double* w, double b,
                 double p, double alpha, int rt, int rh, int rw, double st, double sh, double sw,
                 const double* x0, int K, const double* gK, double* gw_out, double* gb_out) {
    if (C < 2) return -1;
    int64_t N = (int64_t)T * H * W;
    int64_t cap = N * (2 * rt + 1) * (2 * rh + 1) * (2 * rw + 1);
    double* f = (double*)malloc((size_t)N * sizeof(double));
    orc_combine(C, N, V, w, b, f);
    int64_t* rowptr = (int64_t*)malloc((size_t)(N + 1) * sizeof(int64_t));
    int64_t* col = (int64_t*)malloc((size_t)cap * sizeof(int64_t));
    double* val = (double*)malloc((size_t)cap * sizeof(double));
    orc_build_affinity(T, H, W, f, f, p, alpha, rt, rh, rw, st, sh, sw, 0, rowptr, col, val);

    double* xs = (double*)malloc((size_t)(K + 1) * N * sizeof(double));
    double* nus = (double*)malloc((size_t)(K + 1) * sizeof(double));
    double n0 = sqrt(orc_sumsq(x0, N));
    for (int64_t i = 0; i < N; ++i) xs[i] = x0[i] / n0;
    for (int k = 0; k < K; ++k) {
        double* xk = xs + (int64_t)k * N;
        double* xn = xs + (int64_t)(k + 1) * N;
        orc_spmv(N, rowptr, col, val, xk, xn);
        double nu = sqrt(orc_sumsq(xn, N));
        nus[k + 1] = nu;
        for (int64_t i = 0; i < N; ++i) xn[i] /= nu;
    }

    double* g = (double*)malloc((size_t)N * sizeof(double));
    double* gy = (double*)malloc((size_t)N * sizeof(double));
    double* gf = (double*)calloc((size_t)N, sizeof(double));
    memcpy(g, gK, (size_t)N * sizeof(double));
    for (int k = K - 1; k >= 0; --k) {
        const double* xk = xs + (int64_t)k * N;
        const double* xn = xs + (int64_t)(k + 1) * N;
        double proj = orc_dot(xn, g, N);
        for (int64_t i = 0; i < N; ++i) gy[i] = (g[i] - xn[i] * proj) / nus[k + 1];
        for (int64_t i = 0; i < N; ++i) {
            for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
                int64_t j = col[e];
                /* M_ij = k(f_i, f_j) G_ij with G_ij recomputed from the offsets of i and j. */
                int64_t HW = (int64_t)H * W;
                int dt = (int)(j / HW - i / HW);
                int dh = (int)((j / W) % H - (i / W) % H);
                int dw = (int)(j % W - i % W);
                double q = 0.0;
                if (rt > 0) q += (double)(dt * dt) / (st * st);
                if (rh > 0) q += (double)(dh * dh) / (sh * sh);
                if (rw > 0) q += (double)(dw * dw) / (sw * sw);
                double G = exp(-0.5 * q);
                double wgt = gy[i] * xk[j] * G;
                gf[i] += wgt * dk_da(f[i], f[j], p, alpha);
                gf[j] += wgt * dk_da(f[j], f[i], p, alpha);
            }
        }
        orc_spmv(N, rowptr, col, val, gy, g);
    }
    for (int c = 0; c < C; ++c) gw_out[c] = 0.0;
    double gb = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double gz = gf[i] * f[i] * (1.0 - f[i]);
        gb += gz;
        for (int c = 0; c < C; ++c) gw_out[c] += gz * V[(int64_t)c * N + i];
    }
    *gb_out = gb;
    free(f); free(rowptr); free(col); free(val); free(xs); free(nus); free(g); free(gy); free(gf);
    return 0;
}

/* Plain 3x3x3 convolution (cross-correlation), zero padding 1, stride 1, channels-last:
 *   x[T][H][W][Cin], wt[Cout][3][3][3][Cin], bias[Cout], y[T][H][W][Cout]. */
void orc_conv3d_fwd(int T, int H, int W, int Cin, int Cout, const double* x, const double* wt,
                    const double* bias, double* y) {
#pragma omp parallel for collapse(2) schedule(static)
    for (int t = 0; t < T; ++t)
        for (int h = 0; h < H; ++h)
            for (int w = 0; w < W; ++w)
                for (int co = 0; co < Cout; ++co) {
                    double acc = bias ? bias[co] : 0.0;
                    for (int a = 0; a < 3; ++a)
                        for (int bb = 0; bb < 3; ++bb)
                            for (int c = 0; c < 3; ++c) {
                                int ti = t + a - 1, hi = h + bb - 1, wi = w + c - 1;
                                if (ti < 0 || ti >= T || hi < 0 || hi >= H || wi < 0 || wi >= W) continue;
                                const double* xp = x + (((int64_t)ti * H + hi) * W + wi) * Cin;
                                const double* wp = wt + ((((int64_t)co * 3 + a) * 3 + bb) * 3 + c) * Cin;
                                for (int ci = 0; ci < Cin; ++ci) acc += wp[ci] * xp[ci];
                            }
                    y[(((int64_t)t * H + h) * W + w) * Cout + co] = acc;
                }
}

/* Gradients of orc_conv3d_fwd: dx (may be NULL), dw, db from dy. */
void orc_conv3d_bwd(int T, int H, int W, int Cin, int Cout, const double* x, const double* wt,
                    const double* dy, double* dx, double* dw, double* db) {
    int64_t nw = (int64_t)Cout * 27 * Cin;
    memset(dw, 0, (size_t)nw * sizeof(double));
    memset(db, 0, (size_t)Cout * sizeof(double));
    if (dx) memset(dx, 0, (size_t)T * H * W * Cin * sizeof(double));
    for (int t = 0; t < T; ++t)
        for (int h = 0; h < H; ++h)
            for (int w = 0; w < W; ++w)
                for (int co = 0; co < Cout; ++co) {
                    double g = dy[(((int64_t)t * H + h) * W + w) * Cout + co];
                    db[co] += g;
                    for (int a = 0; a < 3; ++a)
                        for (int bb = 0; bb < 3; ++bb)
                            for (int c = 0; c < 3; ++c) {
                                int ti = t + a - 1, hi = h + bb - 1, wi = w + c - 1;
                                if (ti < 0 || ti >= T || hi < 0 || hi >= H || wi < 0 || wi >= W) continue;
                                int64_t xo = (((int64_t)ti * H + hi) * W + wi) * Cin;
                                int64_t wo = ((((int64_t)co * 3 + a) * 3 + bb) * 3 + c) * Cin;
                                for (int ci = 0; ci < Cin; ++ci) {
                                    dw[wo + ci] += g * x[xo + ci];
                                    if (dx) dx[xo + ci] += g * wt[wo + ci];
                                }
                            }
                }
}
