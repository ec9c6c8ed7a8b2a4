// online.cu -- partial iterations on a stream of frames (Sec. 4.5): the online form of the
// method.  A stream keeps a sub-window of the q most recent frames.  When a frame arrives, the
// window's combined features shift by one frame and the new frame is combined into the last
// slot; the window's solution shifts the same way, its new frame starting from the previous
// newest frame's solution (uniform for the first frame); then a few power iterations run on the
// window alone.  Frames before the first one have zero features, so they take no part.
#include <string>

#include "../../include/sfseg.h"
#include "common.cuh"
#include "launch.h"

using namespace sfseg;

struct sfseg_online {
    sfseg_handle* h = nullptr;   // a handle of T = q frames: the window
    int C = 0, q = 0, H = 0, W = 0;
    float* xw[2] = {nullptr, nullptr};   // window solution, caller layout [q][H][W], ping-pong
    int cur = 0;
    long long pushed = 0;
};

namespace {

__global__ void fill_kernel(float* x, int64_t n, float v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = v;
}

int check_cuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return SFSEG_OK;
    return set_last_error(e == cudaErrorMemoryAllocation ? SFSEG_ERR_OOM : SFSEG_ERR_CUDA,
                          (std::string(what) + ": " + cudaGetErrorString(e)).c_str());
}

}  // namespace

extern "C" {

int sfseg_online_create(const sfseg_params* prm, int C, int q, int H, int W, sfseg_online** out) {
    if (!out) return set_last_error(SFSEG_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    if (q < 1 || q > 4096) return set_last_error(SFSEG_ERR_INVALID_ARG, "window length q must be in [1, 4096]");
    sfseg_handle* h = nullptr;
    if (int rc = sfseg_create(prm, C, q, H, W, &h)) return rc;
    sfseg_enable_graphs(h, 1);   // the window's iterations replay as CUDA graphs (two buffer parities)
    sfseg_online* o = new sfseg_online();
    o->h = h;
    o->C = C;
    o->q = q;
    o->H = H;
    o->W = W;
    const size_t bytes = sizeof(float) * (size_t)q * H * W;
    int rc = check_cuda(cudaMalloc(&o->xw[0], bytes), "sfseg_online_create");
    if (!rc) rc = check_cuda(cudaMalloc(&o->xw[1], bytes), "sfseg_online_create");
    if (!rc) rc = check_cuda(cudaMemset(o->xw[0], 0, bytes), "sfseg_online_create");
    if (rc) {
        sfseg_online_destroy(o);
        return rc;
    }
    *out = o;
    return SFSEG_OK;
}

int sfseg_online_destroy(sfseg_online* o) {
    if (!o) return SFSEG_OK;
    cudaDeviceSynchronize();
    cudaFree(o->xw[0]);
    cudaFree(o->xw[1]);
    sfseg_destroy(o->h);
    delete o;
    return SFSEG_OK;
}

int sfseg_online_push(sfseg_online* o, const void* frame, int dtype, const float* weights, float bias,
                      const sfseg_neighborhood* nb, int iters, int iters_bf16, int lag, float* x_frame_out,
                      void* stream) {
    if (!o) return set_last_error(SFSEG_ERR_INVALID_ARG, "null stream handle");
    if (lag < 0 || lag >= o->q) return set_last_error(SFSEG_ERR_INVALID_ARG, "lag must be in [0, q)");
    if (iters < 0) return set_last_error(SFSEG_ERR_INVALID_ARG, "iters must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    if (int rc = handle_push_frame(o->h, frame, dtype, weights, bias, s)) return rc;
    // the window's solution, shifted one frame; the new frame from the previous newest one
    const int64_t fr = (int64_t)o->H * o->W;
    float* src = o->xw[o->cur];
    float* dst = o->xw[o->cur ^ 1];
    if (o->q > 1)
        if (int rc = check_cuda(cudaMemcpyAsync(dst, src + fr, sizeof(float) * (size_t)(fr * (o->q - 1)),
                                                cudaMemcpyDeviceToDevice, s), "window shift"))
            return rc;
    if (o->pushed == 0) {
        fill_kernel<<<(int)((fr + 255) / 256 < 1024 ? (fr + 255) / 256 : 1024), 256, 0, s>>>(dst + fr * (o->q - 1), fr,
                                                                                            1.f);
        count_launches(1);
        if (int rc = check_cuda(cudaGetLastError(), "fill")) return rc;
    } else if (int rc = check_cuda(cudaMemcpyAsync(dst + fr * (o->q - 1), src + fr * (o->q - 1), sizeof(float) * fr,
                                                   cudaMemcpyDeviceToDevice, s), "new frame start")) {
        return rc;
    }
    o->cur ^= 1;
    o->pushed += 1;
    if (int rc = sfseg_power_iterate(o->h, nullptr, 0, nullptr, 0.f, nb, iters, iters_bf16, dst, SFSEG_INIT_USER, 0,
                                     nullptr, stream))
        return rc;
    if (x_frame_out)
        if (int rc = check_cuda(cudaMemcpyAsync(x_frame_out, dst + fr * (o->q - 1 - lag), sizeof(float) * fr,
                                                cudaMemcpyDeviceToDevice, s), "frame output"))
            return rc;
    return SFSEG_OK;
}

int sfseg_online_window(sfseg_online* o, float* x_window_out, void* stream) {
    if (!o || !x_window_out) return set_last_error(SFSEG_ERR_INVALID_ARG, "null argument");
    return check_cuda(cudaMemcpyAsync(x_window_out, o->xw[o->cur], sizeof(float) * (size_t)o->q * o->H * o->W,
                                      cudaMemcpyDeviceToDevice, (cudaStream_t)stream),
                      "window copy");
}

}  // extern "C"
