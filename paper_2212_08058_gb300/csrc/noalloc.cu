// noalloc.cu -- sfseg_power_iterate_noalloc: the power iteration for callers that cannot
// allocate device memory.
//
// Some callers can't call cudaMalloc: a server that reserves its whole device-memory budget
// at start-up and forbids later allocations, a latency-bound loop where cudaMalloc/cudaFree
// would synchronise the device and stall every other stream, or plug-in code that keeps no
// long-lived handle to hold a workspace.  This entry point runs the same kernels as
// sfseg_power_iterate, but every scratch buffer (combined features, the two iterate buffers,
// the FP64 norm accumulators, the error flags and the channel weights) is carved out of one
// fixed array in device global memory that the library declares at file scope.  The array is
// part of the loaded module: every GPU that loads libsfseg.so holds it until the process exits.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/sfseg.h"
#include "common.cuh"
#include "launch.h"

using namespace sfseg;

namespace {

constexpr int64_t kMaxPadded = SFSEG_NOALLOC_MAX_VOXELS;   // T * H * round_up(W, 32)
constexpr int kMaxIters = SFSEG_NOALLOC_MAX_ITERS;
constexpr int kMaxC = 64;

// Layout of the scratch array, in bytes (each part 256-byte aligned).
constexpr size_t kVolBytes = (size_t)kMaxPadded * sizeof(float);
constexpr size_t kOffF = 0;
constexpr size_t kOffV0 = kOffF + kVolBytes;
constexpr size_t kOffV1 = kOffV0 + kVolBytes;
constexpr size_t kOffAcc = kOffV1 + kVolBytes;
constexpr size_t kAccBytes = ((size_t)(kMaxIters + 2) * sizeof(double) + 255) / 256 * 256;
constexpr size_t kOffFlags = kOffAcc + kAccBytes;
constexpr size_t kOffW = kOffFlags + 256;
constexpr size_t kScratchBytes = kOffW + 256;

// The scratch itself.  Host code must not use this name as a pointer: on the host it only
// stands for the symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

int fail(int code, const std::string& msg) { return set_last_error(code, msg.c_str()); }

// Device address of g_noalloc_scratch on each device, looked up once with that device current.
std::mutex g_mu;
unsigned char* g_addr[64] = {nullptr};

int scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(SFSEG_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return fail(SFSEG_ERR_UNSUPPORTED, "device ordinal >= 64");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(SFSEG_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_addr[dev] = (unsigned char*)p;
    }
    *out = g_addr[dev];
    return SFSEG_OK;
}

}  // namespace

extern "C" int sfseg_power_iterate_noalloc(const sfseg_params* prm, int C, int T, int H, int W,
                                           const void* features, int dtype, const float* weights, float bias,
                                           const sfseg_neighborhood* nb, int iters, float* x_inout, int init,
                                           double* norms_out, void* stream) {
    if (!prm || !features || !nb || !x_inout) return fail(SFSEG_ERR_INVALID_ARG, "null argument");
    if (!(prm->alpha > 0.0) || !std::isfinite(prm->alpha)) return fail(SFSEG_ERR_INVALID_ARG, "alpha must be > 0");
    if (!(prm->p > 0.0) || !std::isfinite(prm->p)) return fail(SFSEG_ERR_INVALID_ARG, "p must be > 0");
    if (C < 1 || C > kMaxC) return fail(SFSEG_ERR_INVALID_ARG, "C must be in [1, 64]");
    if (C > 1 && !weights) return fail(SFSEG_ERR_INVALID_ARG, "C > 1 needs channel weights");
    if (dtype != SFSEG_F32 && dtype != SFSEG_BF16) return fail(SFSEG_ERR_DTYPE, "dtype must be F32 or BF16");
    if (init < SFSEG_INIT_USER || init > SFSEG_INIT_SMAP) return fail(SFSEG_ERR_INVALID_ARG, "bad init");
    if (T < 1 || H < 1 || W < 1) return fail(SFSEG_ERR_SHAPE, "empty volume");
    const int pitch = (W + 31) / 32 * 32;
    const int64_t padded = (int64_t)T * H * pitch;
    if (padded > kMaxPadded)
        return fail(SFSEG_ERR_SHAPE, "volume too large for the no-allocation scratch: T*H*round_up(W,32) = " +
                                         std::to_string(padded) + " > " + std::to_string(kMaxPadded));
    if (iters < 0 || iters > kMaxIters)
        return fail(SFSEG_ERR_INVALID_ARG, "iters must be in [0, " + std::to_string(kMaxIters) + "]");
    Taps tp;
    if (int rc = make_taps(nb, &tp)) return rc;
    if (C > 1)
        for (int c = 0; c < C; ++c)
            if (!std::isfinite(weights[c])) return fail(SFSEG_ERR_INVALID_ARG, "non-finite channel weight");

    unsigned char* base = nullptr;
    if (int rc = scratch_address(&base)) return rc;
    float* f32 = (float*)(base + kOffF);
    void* vbuf[2] = {base + kOffV0, base + kOffV1};
    double* acc = (double*)(base + kOffAcc);
    int* flags = (int*)(base + kOffFlags);
    float* wdev = (float*)(base + kOffW);
    cudaStream_t s = (cudaStream_t)stream;

    Geom g;
    g.T = T;
    g.H = H;
    g.W = W;
    g.pitch = pitch;
    const int64_t N = (int64_t)T * H * W;
    cudaError_t e;
    // The array keeps whatever the previous call left: the accumulators and the flags must
    // start at zero; f and both iterate buffers are fully overwritten before they are read.
    if ((e = cudaMemsetAsync(acc, 0, sizeof(double) * (iters + 1), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(flags, 0, sizeof(int), s)) != cudaSuccess)
        return fail(SFSEG_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    if (C > 1 && (e = cudaMemcpyAsync(wdev, weights, sizeof(float) * C, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return fail(SFSEG_ERR_CUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
    const float inv_alpha = (float)(1.0 / prm->alpha), p = (float)prm->p;
    launch_combine(features, dtype, C, g, wdev, bias, f32, nullptr, flags, s);
    launch_prologue(init, x_inout, f32, p, g, vbuf[0], kF32, nullptr, iters == 0 ? x_inout : nullptr, acc, s);
    for (int k = 0; k < iters; ++k) {
        const bool last = k == iters - 1;
        launch_iterate(vbuf[k & 1], kF32, last ? (void*)x_inout : vbuf[(k + 1) & 1], kF32, last, f32, kF32, nullptr,
                       g, tp, inv_alpha, p, acc + k, acc + k + 1, flags, s);
    }
    launch_scale_inv_norm(x_inout, N, acc + iters, flags, s);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return fail(SFSEG_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    if (norms_out) {
        double a[kMaxIters + 2];
        int fl = 0;
        if ((e = cudaMemcpyAsync(a, acc, sizeof(double) * (iters + 1), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(&fl, flags, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return fail(SFSEG_ERR_CUDA, std::string("reading the norms: ") + cudaGetErrorString(e));
        if (fl & kFlagTimeout) return fail(SFSEG_ERR_TIMEOUT, "a bounded wait for a TMA copy gave up");
        if (fl & kFlagBadFeature) return fail(SFSEG_ERR_NONFINITE, "features must be finite and >= 0");
        if (fl & kFlagNonfinite) return fail(SFSEG_ERR_NONFINITE, "an iterate norm became NaN or Inf");
        if (fl & kFlagZeroNorm) return fail(SFSEG_ERR_ZERO_NORM, "an iterate became zero");
        for (int k = 0; k < iters; ++k) norms_out[k] = std::sqrt(a[k + 1]);
    }
    return SFSEG_OK;
}
