/*
 * sfseg.h -- C ABI of the GB300 (sm_103a) SFSeg / SFSeg++ power-iteration library.
 *
 * Method: Burceanu & Leordeanu, "SFSeg / SFSeg++" (arXiv 2212.08058).  The library computes
 * the principal eigenvector of the pixel-level space-time affinity matrix M of Eq. 2,
 *     M_ij = u_i u_j [1 - alpha (f_i - f_j)^2] G_ij,   u = s^p,  (0^p := 0)
 * without forming M, by power iteration (Eq. 4, Eq. 8) in the three-filter form of Eq. 7 / Eq. 10:
 *     A x = u (1/alpha - f^2) G*(u x) - u G*(f^2 u x) + 2 u f G*(f u x),      A = M / alpha,
 *     x_{k+1} = A x_k / ||A x_k||_2.
 * Features are combined first with Eq. 9 (SFSeg++): s = f = sigmoid(sum_c w_c V_c + b); with a
 * single channel s = f = V_0 (Alg. 1, initialisation note).  G is the unnormalised Gaussian
 * exp(-0.5 (dt^2/st^2 + dh^2/sh^2 + dw^2/sw^2)) truncated to the box |dt|<=rt, |dh|<=rh,
 * |dw|<=rw, with zero padding at the volume border (Sec. 4.2: separable, three 1D passes).
 *
 * Conventions for every call
 *   - Volumes are row-major [T][H][W] (w fastest); feature tensors are [C][T][H][W].
 *   - "device" pointers are CUDA global-memory pointers owned by the caller; the library never
 *     frees or keeps them beyond the call.  "host" pointers are ordinary CPU memory.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are asynchronous on it
 *     unless they return host scalars, which they document as synchronising.
 *   - Every call returns an sfseg_status; on failure sfseg_last_error() gives a message
 *     (thread-local, valid until the next call on the same thread).  No exception crosses the ABI.
 *   - A handle is not thread-safe and its calls must not overlap on different streams.
 */
#ifndef SFSEG_H
#define SFSEG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sfseg_status {
    SFSEG_OK = 0,
    SFSEG_ERR_INVALID_ARG = 1, /* null pointer, parameter out of range */
    SFSEG_ERR_SHAPE = 2,       /* empty volume, radius beyond the supported maximum, size mismatch */
    SFSEG_ERR_DTYPE = 3,       /* unknown dtype code */
    SFSEG_ERR_CUDA = 4,        /* a CUDA runtime call failed (message holds the CUDA error) */
    SFSEG_ERR_OOM = 5,         /* device allocation failed */
    SFSEG_ERR_TIMEOUT = 6,     /* a bounded device-side wait (for a TMA copy or an MMA) gave up;
                                  reported by the next synchronising call */
    SFSEG_ERR_NONFINITE = 7,   /* a feature is negative, NaN or Inf, or a norm became non-finite */
    SFSEG_ERR_ZERO_NORM = 8,   /* an iterate became exactly zero (e.g. u = 0 everywhere) */
    SFSEG_ERR_STATE = 9,       /* call order violated (no features set, no recorded forward, ...) */
    SFSEG_ERR_UNSUPPORTED = 10 /* valid request the library does not implement */
} sfseg_status;

typedef enum sfseg_dtype {
    SFSEG_F32 = 0,  /* IEEE float32 */
    SFSEG_BF16 = 1  /* bfloat16 (1-8-7), round to nearest even when the library writes it */
} sfseg_dtype;

typedef enum sfseg_init {
    SFSEG_INIT_USER = 0,    /* start from the caller's x (any non-negative, non-zero vector) */
    SFSEG_INIT_UNIFORM = 1, /* x_0 = 1/sqrt(N) (Sec. 4: "a uniform vector") */
    SFSEG_INIT_SMAP = 2     /* x_0 = S_m / ||S_m|| (Alg. 1: X_m <- S_m) */
} sfseg_init;

/* Method hyper-parameters (Eq. 2): alpha > 0 weights the pairwise term, p > 0 the unary term.
 * The paper uses alpha = 1, p = 0.1 (unsupervised) or 0.2 (semi-supervised) (Sec. 5.1.1). */
typedef struct sfseg_params {
    double alpha;
    double p;
} sfseg_params;

/* Space-time neighbourhood (Eq. 1 distance term; Sec. 4.2 separable 3D Gaussian).
 * 0 <= rt <= 4, 0 <= rh, rw <= 8; sigma_* > 0 wherever the matching radius is > 0. */
typedef struct sfseg_neighborhood {
    int rt, rh, rw;
    float sigma_t, sigma_h, sigma_w;
} sfseg_neighborhood;

typedef struct sfseg_handle sfseg_handle;

/* Library version (major*10000 + minor*100 + patch). */
int sfseg_version(void);

/* Message of the last failed call on this thread ("" if none).  Never NULL. */
const char* sfseg_last_error(void);

/* Create a handle for C-channel feature volumes of T x H x W voxels and allocate its device
 * workspace (combined features, two iterate buffers, FP64 accumulators): about 12 N bytes plus
 * 2 N more once bf16 storage is used, N = T*H*W.  `out` receives the handle (host pointer).
 * Errors: INVALID_ARG (null, alpha <= 0, p <= 0, C < 1 or C > 64), SHAPE (T, H or W < 1,
 * N >= 2^31), OOM, CUDA. */
int sfseg_create(const sfseg_params* prm, int C, int T, int H, int W, sfseg_handle** out);

/* Free the handle and its workspace (synchronises the device).  NULL is a no-op. */
int sfseg_destroy(sfseg_handle* h);

/* Eq. 9 / Alg. 1 lines 1-2: combine the C channels of `features` (device, [C][T][H][W],
 * `dtype`) into f = s inside the handle.  `weights` (host, C floats) and `bias` are ignored when
 * C == 1.  Features must be finite and >= 0 (checked on the device; reported by the next
 * synchronising call as NONFINITE).  Asynchronous. */
int sfseg_set_features(sfseg_handle* h, const void* features, int dtype, const float* weights,
                       float bias, void* stream);

/* Separate unary and pairwise maps (Eq. 9 with its two channel sets; Alg. 1 lines 1-2):
 * S_m = sigmoid(sum_i ws_i S_i + bs) from Cs channels (Cs = 1: S_m = S_1, no sigmoid) and F_m
 * likewise from the handle's C channels (as sfseg_set_features).  Until the next
 * sfseg_set_features, the iterations use the unary term u = S_m^p and the pairwise term on F_m
 * (Eq. 7 with s != f), and the S_m start (SFSEG_INIT_SMAP) is S_m.
 *   s_features: device [Cs][T][H][W] in s_dtype; f_features: device [C][T][H][W] in f_dtype.
 * Allocates one more float32 volume on first use.  The adjoint (recording) and the coarse start
 * are for shared maps and return UNSUPPORTED while separate maps are set.  Asynchronous. */
int sfseg_set_features_sf(sfseg_handle* h, const void* s_features, int s_dtype, int Cs,
                          const float* s_weights, float s_bias, const void* f_features, int f_dtype,
                          const float* f_weights, float f_bias, void* stream);

/* Eq. 7 + Eq. 8 (Alg. 1 main loop, continuous iterations): `iters` >= 0 power iterations.
 *   features      device [C][T][H][W] in `dtype`, or NULL to reuse the features already set.
 *   weights/bias  as for sfseg_set_features (used only when features != NULL).
 *   nb            neighbourhood (host struct).
 *   iters_bf16    the first min(iters_bf16, iters) iterations keep the iterate and f in bf16
 *                 (FP32 arithmetic); the remaining ones run with FP32 storage.
 *   x_inout       device [T][H][W] float32.  Read as the start vector when init ==
 *                 SFSEG_INIT_USER; always overwritten with the unit-norm x_iters.
 *   init          sfseg_init.
 *   record_every  > 0 keeps checkpoints every `record_every` iterations for sfseg_backward
 *                 (about N*4*(iters/record_every + 1) bytes); 0 records nothing.
 *   norms_out     host array of `iters` doubles or NULL.  When given, the call synchronises and
 *                 writes nu_k = ||A x_{k-1}||_2 (k = 1..iters), which converges to lambda_max(A);
 *                 it then also reports ZERO_NORM / NONFINITE found on the device.
 * Errors: INVALID_ARG, SHAPE (radius limits), STATE (no features), OOM, CUDA, and with
 * norms_out ZERO_NORM / NONFINITE. */
int sfseg_power_iterate(sfseg_handle* h, const void* features, int dtype, const float* weights,
                        float bias, const sfseg_neighborhood* nb, int iters, int iters_bf16,
                        float* x_inout, int init, int record_every, double* norms_out,
                        void* stream);

/* One application y = A x of the Eq. 7 operator (FP32 features and storage).
 * x, y: device [T][H][W] float32 (may not alias).  Asynchronous. */
int sfseg_apply(sfseg_handle* h, const sfseg_neighborhood* nb, const float* x, float* y,
                void* stream);

/* The exact kernel (Eq. 1 instead of its first-order expansion Eq. 2), the diagnostic of the
 * approximation (Sec. 4.3, the Fig. 4 comparison): y = (1/alpha) M x with
 * M_ij = u_i u_j exp(-alpha (f_i - f_j)^2) G_ij on the same box, Gaussian and zero padding as
 * sfseg_apply (the 1/alpha matches A = M/alpha of Eq. 7, so both operators have comparable
 * eigenvalues; eigenvectors do not depend on it).  Computed without forming M, through the
 * series exp(-alpha (f_i - f_j)^2) = e^{-alpha f_i^2} e^{-alpha f_j^2} sum_n (2 alpha f_i f_j)^n / n!,
 * whose terms are separable: three terms per pass of the TMA stencil.  Shared maps only
 * (UNSUPPORTED after sfseg_set_features_sf), the radii with a TMA kernel only (UNSUPPORTED
 * otherwise), FP32 storage.
 *   n_terms   the number of series terms, 1..120; 0 chooses the smallest count whose tail
 *             bound x^(N+1)/(N+1)! e^x, x = 2 alpha max(f)^2, is below 2^-24 relative to the sum
 *             (this reads max f: the call synchronises), or returns UNSUPPORTED when 120 terms
 *             do not reach it.
 *   x, y      device [T][H][W] float32 (may not alias).
 * Errors: INVALID_ARG, SHAPE, STATE (no features), UNSUPPORTED, OOM, CUDA. */
int sfseg_apply_exact(sfseg_handle* h, const sfseg_neighborhood* nb, int n_terms, const float* x,
                      float* y, void* stream);

/* Power iteration (Eq. 4 with the Eq. 8 normalisation) on the exact kernel's operator above:
 * `iters` steps from x_inout (init SFSEG_INIT_USER) or from the uniform vector
 * (SFSEG_INIT_UNIFORM); x_inout (device [T][H][W] float32) is overwritten with the unit-norm
 * x_iters.  n_terms as for sfseg_apply_exact.  norms_out: host array of `iters` doubles or NULL
 * (as for sfseg_power_iterate; synchronises when given).  Each step costs ceil(n_terms / 3)
 * stencil passes.  Errors: those of sfseg_apply_exact, and with norms_out ZERO_NORM /
 * NONFINITE. */
int sfseg_power_iterate_exact(sfseg_handle* h, const sfseg_neighborhood* nb, int n_terms, int iters,
                              int init, float* x_inout, double* norms_out, void* stream);

/* Eq. 3: Rayleigh quotient rho = x'Ax / x'x and eigen-residual ||Ax - rho x|| / (rho ||x||)
 * of the FP32 operator (FP64 reductions).  x: device [T][H][W] float32.  rho, residual: host
 * doubles (either may be NULL).  Synchronises the stream.  Uses the handle's iterate buffer as
 * scratch. */
int sfseg_rayleigh(sfseg_handle* h, const sfseg_neighborhood* nb, const float* x, double* rho,
                   double* residual, void* stream);

/* Sec. 3.4 (learning the Eq. 9 weights through the unrolled iteration): given
 * grad_x = dL/dx_K (device [T][H][W] float32) for the x_K of the last sfseg_power_iterate call
 * on this handle (which must have used record_every > 0, C > 1, and features != NULL or set),
 * write dL/dw (host, C floats) and dL/db (host, 1 float).  The adjoint runs backwards through
 * the K normalised steps, recomputing iterates between checkpoints.  Synchronises.
 * Errors: STATE (no recorded forward), UNSUPPORTED (C == 1, or bf16 iterations recorded). */
int sfseg_backward(sfseg_handle* h, const sfseg_neighborhood* nb, const float* grad_x,
                   float* grad_weights, float* grad_bias, void* stream);

/* Coarse-to-fine start vector (the paper has no counterpart; it starts from a uniform vector
 * or from S_m, Alg. 1 line 3).  The slowly converging components of the iterate are smooth at
 * the scale of the objects, so the same Eq. 7 operator on a 2x-pooled volume (per level: f
 * averaged over 2x2x2 blocks, Gaussian widths halved, radii scaled with them and at least 1)
 * has nearly the same principal eigenvector at those scales at an eighth of the cost per
 * iteration.  The coarsest of `levels` (1..4) levels is solved from the uniform start, each
 * finer level from the trilinear upsampling of the coarser solution, each until the Eq. 3
 * residual of its own operator is <= tol (checked after `check_every` iterations, then where
 * the residual's geometric rate over the last two checks predicts tol, at most 8 check_every
 * iterations later; at most `max_iters` per level); the finest coarse solution, upsampled to the handle's volume and
 * scaled to maximum 1, is written to x0_out (device float32 [T][H][W]) for SFSEG_INIT_USER.  iters_out: host array of
 * `levels` ints (iterations per level, index 0 = finest coarse level) or NULL.  Requires the
 * features set; allocates the pyramid (about 1/7 of the handle's workspace) on first use.
 * Synchronises. */
int sfseg_coarse_start(sfseg_handle* h, const sfseg_neighborhood* nb, int levels, double tol,
                       int max_iters, int check_every, float* x0_out, int* iters_out, void* stream);

/* Soft-binarisation iterations (Alg. 1 step 3, Sec. 4.1), run after the continuous power
 * iterations.  Each of the `iters` steps computes y = A x (Eq. 7 operator, FP32) and then
 *     x <- 1 / (1 + exp(-gain (y / max(y) - center)))
 * (reading: the paper's "sigmoid controlled by a parameter" acts on the new vector scaled to
 * maximum 1, so gain and center are independent of the volume size; gain 0 gives 1/2
 * everywhere, large gains approach the indicator of y > center * max y).
 *   x_inout: device float32 [T][H][W]; on input the continuous solution (any positive scale,
 *            e.g. the output of sfseg_power_iterate), on output the soft segmentation in (0, 1).
 *   mask_out: device uint8 [T][H][W] or NULL; receives the hard segmentation x > 1/2 (0 or 1).
 *   iters >= 1; gain >= 0 and center finite.
 * Requires the features set.  Errors: ZERO_NORM if max(y) <= 0 in a step (x then stays as the
 * previous step left it).  Synchronises (reads the status flags). */
int sfseg_soft_binarize(sfseg_handle* h, const sfseg_neighborhood* nb, int iters, float gain,
                        float center, float* x_inout, unsigned char* mask_out, void* stream);

/* ------------------------------------------------------------------------------------------
 * Online form (Sec. 4.5, partial iterations): instead of iterating on the whole video, run a
 * few iterations on a sub-window of the q most recent frames each time a frame arrives, each
 * window starting from the previous window's final solution where they overlap.  Reading
 * taken: the window ends at the newest frame (frames before the first have zero features and
 * take no part); the overlap starts from the previous solution shifted by one frame, the new
 * frame from the previous newest frame's solution (uniform for the very first frame).
 * ---------------------------------------------------------------------------------------- */
typedef struct sfseg_online sfseg_online;

/* A stream of C-channel frames of H x W with a sub-window of q >= 1 frames.  Allocates a handle
 * of q frames plus two window solutions (about 7 q H W floats); the window's iterations run as
 * replayed CUDA graphs (sfseg_enable_graphs). */
int sfseg_online_create(const sfseg_params* params, int C, int q, int H, int W, sfseg_online** out);
int sfseg_online_destroy(sfseg_online* stream_handle);

/* Push the next frame: frame = device [C][H][W] in `dtype`, combined with weights / bias as
 * sfseg_set_features (Eq. 9); then `iters` power iterations (the first iters_bf16 of them with
 * bf16 storage) on the window.  x_frame_out: device float32 [H][W] or NULL; receives the
 * window solution's slice of frame k - lag (lag in [0, q); lag 0 is the frame just pushed, a
 * larger lag gives a frame that also saw lag later frames).  The slice is part of the
 * window's unit-norm vector.  Asynchronous. */
int sfseg_online_push(sfseg_online* stream_handle, const void* frame, int dtype, const float* weights,
                      float bias, const sfseg_neighborhood* nb, int iters, int iters_bf16, int lag,
                      float* x_frame_out, void* stream);

/* Copy the current window solution (device float32 [q][H][W], oldest frame first). */
int sfseg_online_window(sfseg_online* stream_handle, float* x_window_out, void* stream);

/* Learning loss: L = 1 - soft-IoU(xh, g), xh = x / max(x), soft-IoU = sum(xh g) /
 * sum(xh + g - xh g), and dL/dx (the max differentiated at its first argmax).
 * x, target: device [T][H][W] float32 of this handle's size; grad_x: device float32 or NULL;
 * loss: host double.  Synchronises. */
int sfseg_soft_iou_loss(sfseg_handle* h, const float* x, const float* target, double* loss,
                        float* grad_x, void* stream);

/* ------------------------------------------------------------------------------------------
 * Learned warm start (no counterpart in the paper, which starts from a uniform vector or from
 * S_m, Alg. 1 line 3).  A 4-layer 3x3x3 convolutional network, C_in -> 32 -> 32 -> 32 -> 1, ReLU
 * between layers and softplus at the end, predicts a start vector x0 > 0 from the raw input
 * channels.  Forward and data-gradient convolutions run on the tensor cores (bf16 in, fp32
 * accumulation); parameters are fp32 with AdamW.  Parameter order in the flat host vectors:
 * W1[32][3][3][3][C_in], b1[32], W2[32][3][3][3][32], b2[32], W3 (same), b3, W4[1][3][3][3][32], b4[1]
 * (weights as [out][kt][kh][kw][in], cross-correlation, zero padding 1).
 * ---------------------------------------------------------------------------------------- */
typedef struct sfseg_net sfseg_net;

/* Create a network for 1 <= c_in <= 16 input channels with He-normal weights drawn from a
 * counter-based generator seeded by `seed`, zero biases.  Allocates its parameters, gradients
 * and AdamW moments on the current device; activation workspace grows with the largest volume
 * seen (about 240 bytes per voxel). */
int sfseg_net_create(int c_in, uint64_t seed, sfseg_net** out);
int sfseg_net_destroy(sfseg_net* net);
int sfseg_net_num_params(sfseg_net* net, int64_t* count);
/* Copy all parameters to / from a host float array of sfseg_net_num_params entries. */
int sfseg_net_get_params(sfseg_net* net, float* host, int64_t count);
int sfseg_net_set_params(sfseg_net* net, const float* host, int64_t count);

/* x0_out (device float32 [T][H][W]) = network(features, extra), features device [C][T][H][W] in
 * `dtype`; extra: NULL, or a device float32 [T][H][W] volume given to the network as channel C
 * (e.g. the upsampled coarse solution of sfseg_coarse_start); C (+1 with extra) <= c_in.
 * Asynchronous. */
int sfseg_net_forward(sfseg_net* net, const void* features, int dtype, int C, const float* extra,
                      int T, int H, int W, float* x0_out, void* stream);

/* Training loss and gradients: L = 1 - <x0, target> / (||x0|| ||target||) for the network's x0
 * (the direction of the start vector is what power iteration uses).  target: device float32
 * [T][H][W]; features and extra as for sfseg_net_forward.  Writes L to *loss (host) and, if
 * grads_out is not NULL, the parameter gradients to it (host, sfseg_net_num_params floats);
 * keeps them for sfseg_net_adamw.  Synchronises. */
int sfseg_net_backward(sfseg_net* net, const void* features, int dtype, int C, const float* extra,
                       int T, int H, int W, const float* target, double* loss, float* grads_out,
                       void* stream);

/* One layer of the network alone, on a caller's activation (to run the network layer by layer,
 * or to check one layer's convolution against a reference).  layer = 0..3.
 *   in    device bf16 [T][H][W][CP] channels-last, CP = 16 for layer 0 (its c_in channels, then
 *         zeros) and 32 for layers 1..3.
 *   out   layers 0..2: device bf16 [T][H][W][32] = ReLU(conv(in) + b), rounded to nearest;
 *         layer 3: device float32 [T][H][W] z = conv(in) + b, and out2 (device float32
 *         [T][H][W], required) = softplus(z).
 * conv is the 3x3x3 cross-correlation with zero padding 1 and the layer's weights rounded to
 * bf16, accumulated in fp32 on the tensor cores.  Asynchronous; a bounded wait that gave up is
 * reported by sfseg_net_check.  Errors: INVALID_ARG, SHAPE, CUDA. */
int sfseg_net_layer_forward(sfseg_net* net, int layer, const void* in, int T, int H, int W,
                            void* out, float* out2, void* stream);

/* Gradients of one layer given the loss gradient dz at its output before the activation
 * (device bf16 [T][H][W][DP], DP = 32 for layers 0..2; 16 for layer 3, whose one output is
 * channel 0 and the other 15 channels must be 0), and the layer's input `in` (as for
 * sfseg_net_layer_forward):
 *   dW_out  device float32 [COUT][27][CIN] (overwritten): sum over voxels of dz x in(shifted);
 *   db_out  device float32 [COUT] (overwritten): sum over voxels of dz;
 *   dx_out  layers 1..3: device bf16 [T][H][W][32] or NULL: the gradient at the pre-activation
 *           of the layer below, conv^T(dz) * [in > 0] (flipped taps, bf16 weights, fp32
 *           accumulation on the tensor cores); must be NULL for layer 0.
 * COUT = 32 (1 for layer 3), CIN = the network's c_in for layer 0, else 32.  Asynchronous.
 * Errors: INVALID_ARG, SHAPE, CUDA. */
int sfseg_net_layer_backward(sfseg_net* net, int layer, const void* in, const void* dz, int T,
                             int H, int W, void* dx_out, float* dW_out, float* db_out,
                             void* stream);

/* Synchronises `stream` and returns TIMEOUT if a bounded wait inside one of the network's
 * kernels gave up since the last check (then clears the flag), else OK. */
int sfseg_net_check(sfseg_net* net, void* stream);

/* Launch shape of the network's convolutions (instrumentation; no counterpart in the paper).
 * For kernel 0 (the hidden-layer kernel: the forward of layers 0..2 and the data gradients of
 * layers 1..3) or 1 (the last layer's forward), the shape of the calling thread's most recent
 * launch of it: output frames per CTA (3, 2 or 1; 4 or 1 for kernel 1), output rows per CTA
 * (64, 32 or 16) and the number of CTAs; all three 0 before the first launch.  Host outputs.
 * Errors: INVALID_ARG (kernel not 0 or 1, null output). */
int sfseg_net_launch_shape(int kernel, int* frames, int* rows, int* ctas);

/* One AdamW step (decoupled weight decay) with the gradients of the last sfseg_net_backward. */
int sfseg_net_adamw(sfseg_net* net, float lr, float beta1, float beta2, float eps,
                    float weight_decay, void* stream);

/* The start vector for this handle's volume: x0_out (device float32 [T][H][W], usable as
 * x_inout with SFSEG_INIT_USER) = network(features, x_coarse), features device [C][T][H][W] of
 * the handle's shape in `dtype`, x_coarse NULL or the device float32 [T][H][W] output of
 * sfseg_coarse_start (for a network built with one more input channel).  Asynchronous. */
int sfseg_warmstart(sfseg_handle* h, sfseg_net* net, const void* features, int dtype,
                    const float* x_coarse, float* x0_out, void* stream);

/* Self-test of failure reporting (no counterpart in the paper).  Every wait inside this
 * library's kernels (for a TMA copy or an MMA to complete) is bounded: on expiry the kernel
 * raises a timeout flag, lets its own copies in flight land (again bounded), releases what it
 * holds and returns, and the host call returns SFSEG_ERR_TIMEOUT.  This call runs that path on
 * purpose: a one-warp kernel waits `spins` times (1 <= spins <= 1e6) on a barrier that nothing
 * completes.  Returns SFSEG_ERR_TIMEOUT -- the expected outcome -- and leaves the handle and the
 * CUDA context usable.  Synchronises. */
int sfseg_selftest_wait(sfseg_handle* h, long long spins, void* stream);

/* CUDA graphs for launch-bound calls (no counterpart in the paper).  When enabled, a call of
 * sfseg_power_iterate that passes features == NULL (features already set), records nothing,
 * asks for no norms and is not being timed, and every sfseg_backward, run their launch
 * sequences as CUDA graphs: the first call for given pointers and parameters (x_inout or
 * grad_x, iters, iters_bf16, init, the recording, neighbourhood, the handle's buffers) captures
 * it, later ones replay it.  The graph runs on a stream of the handle,
 * ordered after the work already queued on the caller's stream and before the work queued
 * after the call; results are those of direct launches (up to the order of the FP64 atomic
 * sums of norms and dot products, as between any two runs).  Worth it for small volumes, where
 * launch latency dominates.  Off by default.  Errors: INVALID_ARG (null handle); capture
 * failures surface as CUDA from the call that captures. */
int sfseg_enable_graphs(sfseg_handle* h, int on);

/* Instrumentation (no counterpart in the paper).  When enabled, each sfseg_power_iterate call
 * records two CUDA events on its stream, before its first and after its last iteration-kernel
 * launch.  sfseg_iter_timing waits for the recorded events, returns the summed milliseconds and
 * the number of iteration launches they bracket (host outputs), and resets both.  Disabled by
 * default; enabling it adds two event records per call.  Errors: INVALID_ARG (null handle or
 * output), CUDA. */
int sfseg_enable_iter_timing(sfseg_handle* h, int on);
int sfseg_iter_timing(sfseg_handle* h, double* ms, int64_t* launches);

/* Number of CUDA kernels this library has launched in the process so far (host output).
 * Errors: INVALID_ARG (null count). */
int sfseg_kernel_launches(int64_t* count);

/* Eq. 8 for a volume split into parts (for example slabs along t, one per GPU): the squared
 * norm of the next iterate is the sum of the parts' sums, so each part accumulates its own and
 * the caller adds them across parts (an all-reduce) before every part divides by the root.
 * sfseg_sumsq:     acc_dev[0] += sum_i x_i^2 over the n float32 values at x (device), summed in
 *                  FP64 on the device (acc_dev: device double the caller zeroes first).
 * sfseg_normalize: x_i *= 1 / sqrt(acc_dev[0]) for the n values at x (device).  A zero or
 *                  non-finite acc_dev[0] leaves x multiplied by 0 and raises the handle's
 *                  ZERO_NORM / NONFINITE flag (reported by sfseg_check).
 * Both asynchronous on `stream`; h supplies the error flags only.  Errors: INVALID_ARG. */
int sfseg_sumsq(sfseg_handle* h, const float* x, int64_t n, double* acc_dev, void* stream);
int sfseg_normalize(sfseg_handle* h, float* x, int64_t n, const double* acc_dev, void* stream);

/* Synchronises `stream` and reports (then clears) the handle's device-side error flags:
 * TIMEOUT, NONFINITE (bad features or a non-finite norm), ZERO_NORM; OK if none is set. */
int sfseg_check(sfseg_handle* h, void* stream);

/* Which kernel ran the power-iteration steps (instrumentation; no counterpart in the paper).
 * The radii (1,3,3), (2,7,7), (1,4,4), (1,2,2), (1,5,5), (2,3,3), (2,5,5) and (1,7,7) run on the
 * TMA-staged stencil kernel; other
 * radii, or a volume whose tensor maps the driver does not encode, run on the generic streaming
 * stencil, which gives the same results more slowly.  Process-wide counts of steps issued on
 * each (host outputs; steps captured into a CUDA graph count once, at capture), and in
 * last_kernel (host buffer of len >= 1 chars, or NULL) the kernel name of the last step,
 * e.g. "iter_fast<2,7,7,float,float>".  Errors: INVALID_ARG (null count). */
int sfseg_iterate_kernel_stats(int64_t* tma_steps, int64_t* generic_steps, char* last_kernel,
                               int len);

/* No-allocation power iteration (the paper has no counterpart: this is a deployment aid).
 *
 * For callers that cannot allocate device memory -- a server that reserves its whole memory
 * budget at start-up and forbids later cudaMalloc calls, a latency-bound loop where cudaMalloc
 * or cudaFree would synchronise the device and stall other streams, or plug-in code that keeps
 * no handle to own a workspace.  It computes what sfseg_create + sfseg_power_iterate (float32
 * storage, no recording) + sfseg_destroy compute, with the same kernels, but allocates nothing:
 * its scratch (combined features, two iterate buffers, FP64 norms, flags, weights) is one fixed
 * array of about 24 MiB in device global memory, declared by the library, which every GPU that
 * loads libsfseg.so holds until the process exits.
 *   Limits: T * H * round_up(W, 32) <= SFSEG_NOALLOC_MAX_VOXELS and 0 <= iters <=
 *   SFSEG_NOALLOC_MAX_ITERS; larger requests return SFSEG_ERR_SHAPE / SFSEG_ERR_INVALID_ARG
 *   without touching the GPU.
 *   Arguments: as sfseg_create (prm, C, T, H, W) and sfseg_power_iterate (features, dtype,
 *   weights, bias, nb, iters, x_inout, init, norms_out, stream).  The caller owns features,
 *   x_inout and norms_out.
 *   Errors found on the device (TIMEOUT, NONFINITE for bad features or a non-finite norm,
 *   ZERO_NORM) are reported only by a call that passes norms_out: that call synchronises and
 *   reads the device's error flags.  A call without norms_out returns once its work is queued
 *   and reports only argument and launch errors; the next call clears the flags it left.
 *   Sharing: every call, from any thread, on any stream of the same device, uses the same
 *   array, which keeps the previous call's contents (the call clears what must start at
 *   zero).  Calls whose GPU work overlaps -- concurrent streams, or calls on one device from
 *   several threads without ordering -- race on it and give wrong results; order them.
 *   Set-up: the first call on each device (with that device current) looks up the array's
 *   device address with cudaGetSymbolAddress; make that first call before any stream capture
 *   begins on the device. */
#define SFSEG_NOALLOC_MAX_VOXELS 2097152
#define SFSEG_NOALLOC_MAX_ITERS 4096
int sfseg_power_iterate_noalloc(const sfseg_params* prm, int C, int T, int H, int W,
                                const void* features, int dtype, const float* weights, float bias,
                                const sfseg_neighborhood* nb, int iters, float* x_inout, int init,
                                double* norms_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SFSEG_H */
