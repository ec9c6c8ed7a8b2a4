// api.cu -- the C ABI of libsfseg.so (declared in include/sfseg.h): argument checking, the
// handle's device workspace, and the sequence of kernel launches of each call.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sfseg.h"
#include "common.cuh"
#include "launch.h"

using namespace sfseg;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

#define SFSEG_CUDA(call)                                                                     \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(e_ == cudaErrorMemoryAllocation ? SFSEG_ERR_OOM : SFSEG_ERR_CUDA,    \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                 \
    } while (0)

#define SFSEG_LAUNCHED()                                                                     \
    do {                                                                                     \
        cudaError_t e_ = cudaGetLastError();                                                 \
        if (e_ != cudaSuccess)                                                               \
            return fail(SFSEG_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t n) {
    return cudaMalloc((void**)p, n * sizeof(T) > 0 ? n * sizeof(T) : 16);
}

}  // namespace

namespace sfseg {
int set_last_error(int code, const char* msg) { return fail(code, msg); }
}  // namespace sfseg

// Layout of the handle's FP64 scratch, in doubles: one disjoint region per use.
constexpr int kScrRayleigh = 0;      // 4: x'Ax, x'x, the residual sum
constexpr int kScrApplyAcc = 8;      // 1: norm sum of the adjoint's recomputed iterates
constexpr int kScrWeightGrad = 16;   // C + 1 <= 65: dL/dw, dL/db
constexpr int kScrSoftIou = 88;      // 4: soft-IoU sums
constexpr int kScrMaxKey = 96;       // 1 (an unsigned key): a maximum
constexpr int kScrSWeights = 104;    // 32 doubles = 64 floats: separate-map unary weights
constexpr int kScrDoubles = 136;

// A captured launch sequence of sfseg_power_iterate and what it was captured for (every pointer
// and parameter the sequence bakes in).
struct GraphKey {
    int kind;   // 0: sfseg_power_iterate, 1: sfseg_backward
    const void* x;
    const void* f32;
    const void* fbf;
    const void* v0;
    const void* v1;
    const void* s32;
    const void* acc;
    int iters, bf, init;
    Taps tp;
};
struct GraphEntry {
    GraphKey key;
    cudaGraphExec_t exec;
    int64_t launches;
};

struct sfseg_handle {
    int C = 0;
    double alpha = 1.0, p = 0.1;
    Geom g{};
    int64_t N = 0, NP = 0;            // voxels; elements of an internal (pitched) volume
    float* f32 = nullptr;             // combined features, float32
    float* s32 = nullptr;             // separate unary map S_m (sfseg_set_features_sf), float32
    bool sep = false;                 // s32 in use: u = S_m^p instead of f^p
    __nv_bfloat16* fbf = nullptr;     // bf16 copy (allocated on first bf16 use)
    bool fbf_valid = false;
    bool features_set = false;
    const void* feat_ptr = nullptr;   // caller's last feature tensor (for the weight gradient)
    int feat_dtype = 0;
    void* vbuf[2] = {nullptr, nullptr};   // iterate ping-pong, NP floats each
    double* acc = nullptr;            // per-step squared norms
    int acc_cap = 0;
    double* scratch = nullptr;        // kScrDoubles doubles for reductions (layout above)
    unsigned long long* amax = nullptr;
    int* flags = nullptr;
    float* wdev = nullptr;            // channel weights on the device
    // recorded forward (for the adjoint)
    int rec_K = 0, rec_every = 0;
    bool rec_valid = false;
    std::vector<float*> ckpt;         // x~ at k = 0, every, 2 every, ... and at K (last entry)
    double* rec_acc = nullptr;
    int rec_acc_cap = 0;
    // adjoint workspace
    float* gbuf[2] = {nullptr, nullptr};
    float* gz = nullptr;
    float* adjw[3] = {nullptr, nullptr, nullptr};   // TMA-path adjoint workspace (Q_g, v_g, v_g)
    std::vector<float*> seg;
    std::vector<float*> qxs;   // TMA path: Q_x of each step of the segment being reversed
    float* exv = nullptr;      // the exact kernel's term input (internal layout)
    double* dots = nullptr;
    int dots_cap = 0;
    // optional CUDA-event timing of the iteration kernels
    bool timing = false;
    std::vector<cudaEvent_t> ev_free;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
    int64_t timed_launches = 0;
    // CUDA graphs of sfseg_power_iterate's launch sequence (sfseg_enable_graphs)
    bool graphs = false;
    cudaStream_t gstream = nullptr;   // graphs are captured and launched here, ordered by events
    cudaEvent_t gev[2] = {nullptr, nullptr};
    std::vector<GraphEntry> gcache;
    // coarse pyramid for sfseg_coarse_start: child handles (C = 1, pooled f) and their x
    std::vector<sfseg_handle*> lvl;
    std::vector<float*> lvl_f, lvl_x;
    std::vector<int> lvl_p;           // pool factors (t, h, w) from the previous level, 3 per level
};

static cudaEvent_t take_event(sfseg_handle* h) {
    if (!h->ev_free.empty()) {
        cudaEvent_t e = h->ev_free.back();
        h->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

static bool same_key(const GraphKey& a, const GraphKey& b) {
    return a.kind == b.kind && a.x == b.x && a.f32 == b.f32 && a.fbf == b.fbf && a.v0 == b.v0 && a.v1 == b.v1 && a.s32 == b.s32 &&
           a.acc == b.acc && a.iters == b.iters && a.bf == b.bf && a.init == b.init &&
           std::memcmp(&a.tp, &b.tp, sizeof(Taps)) == 0;
}

// Runs `enqueue` (the call's launch sequence) as a CUDA graph on the handle's own stream, ordered
// after and before the caller's stream by events: replays a graph captured earlier for the same
// pointers and parameters, or captures one now (at most 8 are kept).  If capture or
// instantiation fails, the sequence runs directly on the caller's stream instead.
template <typename F>
static int run_graph(sfseg_handle* h, cudaStream_t s, const GraphKey& key, F&& enqueue) {
    if (!h->gstream) {
        SFSEG_CUDA(cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking));
        SFSEG_CUDA(cudaEventCreateWithFlags(&h->gev[0], cudaEventDisableTiming));
        SFSEG_CUDA(cudaEventCreateWithFlags(&h->gev[1], cudaEventDisableTiming));
    }
    GraphEntry* hit = nullptr;
    for (GraphEntry& e : h->gcache)
        if (same_key(e.key, key)) hit = &e;
    if (!hit) {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        const int64_t c0 = launches_so_far();
        bool ok = cudaStreamBeginCapture(h->gstream, cudaStreamCaptureModeRelaxed) == cudaSuccess;
        int rc = ok ? enqueue(h->gstream) : SFSEG_OK;
        if (ok) ok = cudaStreamEndCapture(h->gstream, &graph) == cudaSuccess && graph != nullptr;
        const int64_t n = launches_so_far() - c0;
        count_launches((int)-n);   // captured, not run
        if (ok && rc == SFSEG_OK) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
        if (graph) cudaGraphDestroy(graph);
        if (!ok || rc != SFSEG_OK) {
            cudaGetLastError();
            return enqueue(s);
        }
        if (h->gcache.size() >= 8) {
            cudaGraphExecDestroy(h->gcache.front().exec);
            h->gcache.erase(h->gcache.begin());
        }
        h->gcache.push_back(GraphEntry{key, exec, n});
        hit = &h->gcache.back();
    }
    SFSEG_CUDA(cudaEventRecord(h->gev[0], s));
    SFSEG_CUDA(cudaStreamWaitEvent(h->gstream, h->gev[0], 0));
    SFSEG_CUDA(cudaGraphLaunch(hit->exec, h->gstream));
    count_launches((int)hit->launches);
    SFSEG_CUDA(cudaEventRecord(h->gev[1], h->gstream));
    SFSEG_CUDA(cudaStreamWaitEvent(s, h->gev[1], 0));
    return SFSEG_OK;
}

static int check_handle(sfseg_handle* h) {
    if (!h) return fail(SFSEG_ERR_INVALID_ARG, "null handle");
    return SFSEG_OK;
}

int sfseg::make_taps(const sfseg_neighborhood* nb, Taps* tp) {
    if (!nb) return fail(SFSEG_ERR_INVALID_ARG, "null neighborhood");
    if (nb->rt < 0 || nb->rh < 0 || nb->rw < 0 || nb->rt > kMaxRT || nb->rh > kMaxRH || nb->rw > kMaxRW)
        return fail(SFSEG_ERR_SHAPE, "radius out of range (0 <= rt <= 4, 0 <= rh, rw <= 8)");
    const float sg[3] = {nb->sigma_t, nb->sigma_h, nb->sigma_w};
    const int rr[3] = {nb->rt, nb->rh, nb->rw};
    for (int a = 0; a < 3; ++a)
        if (rr[a] > 0 && !(sg[a] > 0.f && std::isfinite(sg[a])))
            return fail(SFSEG_ERR_INVALID_ARG, "sigma must be finite and > 0 where the radius is > 0");
    std::memset(tp, 0, sizeof(Taps));
    tp->rt = nb->rt;
    tp->rh = nb->rh;
    tp->rw = nb->rw;
    float* dst[3] = {tp->gt, tp->gh, tp->gw};
    for (int a = 0; a < 3; ++a)
        for (int d = -rr[a]; d <= rr[a]; ++d)
            dst[a][d + rr[a]] = rr[a] == 0 ? 1.f : (float)std::exp(-(double)d * d / (2.0 * (double)sg[a] * sg[a]));
    return SFSEG_OK;
}

static int ensure_acc(double** buf, int* cap, int need) {
    if (*cap >= need) return SFSEG_OK;
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
    int n = need < 1024 ? 1024 : need;
    SFSEG_CUDA(dalloc(buf, (size_t)n));
    *cap = n;
    return SFSEG_OK;
}

static int read_flags(sfseg_handle* h, cudaStream_t s) {
    int fl = 0;
    SFSEG_CUDA(cudaMemcpyAsync(&fl, h->flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    SFSEG_CUDA(cudaStreamSynchronize(s));
    if (fl) SFSEG_CUDA(cudaMemsetAsync(h->flags, 0, sizeof(int), s));
    if (fl & kFlagTimeout) return fail(SFSEG_ERR_TIMEOUT, "a bounded wait for a TMA copy gave up");
    if (fl & kFlagBadFeature) return fail(SFSEG_ERR_NONFINITE, "features must be finite and >= 0");
    if (fl & kFlagNonfinite) return fail(SFSEG_ERR_NONFINITE, "an iterate norm became NaN or Inf");
    if (fl & kFlagZeroNorm) return fail(SFSEG_ERR_ZERO_NORM, "an iterate became zero (u = 0 on its support?)");
    return SFSEG_OK;
}

namespace sfseg {

// Shift the combined features one frame towards t = 0 (frame 0 drops out) and combine `frame`
// (caller layout [C][H][W], `dtype`) into the last frame; used by the online stream.  The
// shifted copy goes into the idle iterate buffer, which then becomes the feature buffer.
int handle_push_frame(sfseg_handle* h, const void* frame, int dtype, const float* weights, float bias,
                      cudaStream_t s) {
    if (!frame) return fail(SFSEG_ERR_INVALID_ARG, "null frame");
    if (dtype != SFSEG_F32 && dtype != SFSEG_BF16) return fail(SFSEG_ERR_DTYPE, "dtype must be F32 or BF16");
    if (h->C > 1 && !weights) return fail(SFSEG_ERR_INVALID_ARG, "C > 1 needs channel weights");
    if (h->C > 1) {
        for (int c = 0; c < h->C; ++c)
            if (!std::isfinite(weights[c])) return fail(SFSEG_ERR_INVALID_ARG, "non-finite channel weight");
        SFSEG_CUDA(cudaMemcpyAsync(h->wdev, weights, sizeof(float) * h->C, cudaMemcpyHostToDevice, s));
    }
    const int64_t frame_elems = (int64_t)h->g.H * h->g.pitch;
    float* nf = (float*)h->vbuf[0];
    if (h->g.T > 1)
        SFSEG_CUDA(cudaMemcpyAsync(nf, h->f32 + frame_elems, sizeof(float) * (size_t)(frame_elems * (h->g.T - 1)),
                                   cudaMemcpyDeviceToDevice, s));
    Geom g1 = h->g;
    g1.T = 1;
    launch_combine(frame, dtype, h->C, g1, h->wdev, bias, nf + frame_elems * (h->g.T - 1), nullptr, h->flags, s);
    SFSEG_LAUNCHED();
    h->vbuf[0] = h->f32;
    h->f32 = nf;
    h->fbf_valid = false;
    h->features_set = true;
    h->sep = false;
    h->feat_ptr = nullptr;
    h->rec_valid = false;
    return SFSEG_OK;
}

}  // namespace sfseg

extern "C" {

int sfseg_version(void) { return 100; }

const char* sfseg_last_error(void) { return g_err.c_str(); }

int sfseg_create(const sfseg_params* prm, int C, int T, int H, int W, sfseg_handle** out) {
    if (!prm || !out) return fail(SFSEG_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (!(prm->alpha > 0.0) || !std::isfinite(prm->alpha)) return fail(SFSEG_ERR_INVALID_ARG, "alpha must be > 0");
    if (!(prm->p > 0.0) || !std::isfinite(prm->p)) return fail(SFSEG_ERR_INVALID_ARG, "p must be > 0");
    if (C < 1 || C > 64) return fail(SFSEG_ERR_INVALID_ARG, "C must be in [1, 64]");
    if (T < 1 || H < 1 || W < 1) return fail(SFSEG_ERR_SHAPE, "empty volume");
    const int64_t N = (int64_t)T * H * W;
    if (N >= (int64_t(1) << 31)) return fail(SFSEG_ERR_SHAPE, "volume must have fewer than 2^31 voxels");
    sfseg_handle* h = new sfseg_handle();
    h->C = C;
    h->alpha = prm->alpha;
    h->p = prm->p;
    h->g.T = T;
    h->g.H = H;
    h->g.W = W;
    h->g.pitch = (W + 31) / 32 * 32;
    h->N = N;
    h->NP = (int64_t)T * H * h->g.pitch;
    int rc = SFSEG_OK;
    auto chk = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == SFSEG_OK)
            rc = fail(e == cudaErrorMemoryAllocation ? SFSEG_ERR_OOM : SFSEG_ERR_CUDA,
                      std::string("sfseg_create: ") + cudaGetErrorString(e));
    };
    chk(dalloc(&h->f32, (size_t)h->NP));
    chk(dalloc((float**)&h->vbuf[0], (size_t)h->NP));
    chk(dalloc((float**)&h->vbuf[1], (size_t)h->NP));
    chk(dalloc(&h->scratch, kScrDoubles));
    chk(dalloc(&h->amax, 1));
    chk(dalloc(&h->flags, 1));
    chk(dalloc(&h->wdev, 64));
    if (rc == SFSEG_OK) chk(cudaMemset(h->flags, 0, sizeof(int)));
    if (rc == SFSEG_OK) chk(cudaMemset(h->f32, 0, (size_t)h->NP * sizeof(float)));
    if (rc == SFSEG_OK) rc = ensure_acc(&h->acc, &h->acc_cap, 1024);
    if (rc != SFSEG_OK) {
        sfseg_destroy(h);
        return rc;
    }
    *out = h;
    return SFSEG_OK;
}

int sfseg_destroy(sfseg_handle* h) {
    if (!h) return SFSEG_OK;
    cudaDeviceSynchronize();
    cudaFree(h->f32);
    cudaFree(h->s32);
    cudaFree(h->fbf);
    cudaFree(h->vbuf[0]);
    cudaFree(h->vbuf[1]);
    cudaFree(h->acc);
    cudaFree(h->scratch);
    for (GraphEntry& e : h->gcache) cudaGraphExecDestroy(e.exec);
    if (h->gev[0]) cudaEventDestroy(h->gev[0]);
    if (h->gev[1]) cudaEventDestroy(h->gev[1]);
    if (h->gstream) cudaStreamDestroy(h->gstream);
    for (float* q : h->adjw) cudaFree(q);
    cudaFree(h->amax);
    cudaFree(h->flags);
    cudaFree(h->wdev);
    for (float* p : h->ckpt) cudaFree(p);
    cudaFree(h->rec_acc);
    cudaFree(h->gbuf[0]);
    cudaFree(h->gbuf[1]);
    cudaFree(h->gz);
    for (float* p : h->seg) cudaFree(p);
    for (float* p : h->qxs) cudaFree(p);
    cudaFree(h->exv);
    cudaFree(h->dots);
    for (sfseg_handle* c : h->lvl) sfseg_destroy(c);
    for (float* p : h->lvl_f) cudaFree(p);
    for (float* p : h->lvl_x) cudaFree(p);
    for (cudaEvent_t e : h->ev_free) cudaEventDestroy(e);
    for (auto& pr : h->ev_pending) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    delete h;
    return SFSEG_OK;
}

int sfseg_set_features(sfseg_handle* h, const void* features, int dtype, const float* weights, float bias,
                       void* stream) {
    if (int rc = check_handle(h)) return rc;
    if (!features) return fail(SFSEG_ERR_INVALID_ARG, "null features");
    if (dtype != SFSEG_F32 && dtype != SFSEG_BF16) return fail(SFSEG_ERR_DTYPE, "dtype must be F32 or BF16");
    if (h->C > 1 && !weights) return fail(SFSEG_ERR_INVALID_ARG, "C > 1 needs channel weights");
    cudaStream_t s = (cudaStream_t)stream;
    if (h->C > 1) {
        for (int c = 0; c < h->C; ++c)
            if (!std::isfinite(weights[c])) return fail(SFSEG_ERR_INVALID_ARG, "non-finite channel weight");
        SFSEG_CUDA(cudaMemcpyAsync(h->wdev, weights, sizeof(float) * h->C, cudaMemcpyHostToDevice, s));
    }
    launch_combine(features, dtype, h->C, h->g, h->wdev, bias, h->f32, h->fbf, h->flags, s);
    SFSEG_LAUNCHED();
    h->fbf_valid = h->fbf != nullptr;
    h->features_set = true;
    h->sep = false;
    h->feat_ptr = features;
    h->feat_dtype = dtype;
    h->rec_valid = false;
    return SFSEG_OK;
}

int sfseg_set_features_sf(sfseg_handle* h, const void* s_features, int s_dtype, int Cs, const float* s_weights,
                          float s_bias, const void* f_features, int f_dtype, const float* f_weights, float f_bias,
                          void* stream) {
    if (int rc = check_handle(h)) return rc;
    if (!s_features) return fail(SFSEG_ERR_INVALID_ARG, "null s_features");
    if (s_dtype != SFSEG_F32 && s_dtype != SFSEG_BF16) return fail(SFSEG_ERR_DTYPE, "s_dtype must be F32 or BF16");
    if (Cs < 1 || Cs > 64) return fail(SFSEG_ERR_INVALID_ARG, "Cs must be in [1, 64]");
    if (Cs > 1 && !s_weights) return fail(SFSEG_ERR_INVALID_ARG, "Cs > 1 needs unary channel weights");
    if (Cs > 1)
        for (int c = 0; c < Cs; ++c)
            if (!std::isfinite(s_weights[c])) return fail(SFSEG_ERR_INVALID_ARG, "non-finite unary channel weight");
    cudaStream_t s = (cudaStream_t)stream;
    if (!h->s32) {
        SFSEG_CUDA(dalloc(&h->s32, (size_t)h->NP));
        SFSEG_CUDA(cudaMemsetAsync(h->s32, 0, (size_t)h->NP * sizeof(float), s));
    }
    if (int rc = sfseg_set_features(h, f_features, f_dtype, f_weights, f_bias, stream)) return rc;
    float* swdev = reinterpret_cast<float*>(h->scratch + kScrSWeights);   // 64 floats
    if (Cs > 1) SFSEG_CUDA(cudaMemcpyAsync(swdev, s_weights, sizeof(float) * Cs, cudaMemcpyHostToDevice, s));
    launch_combine(s_features, s_dtype, Cs, h->g, swdev, s_bias, h->s32, nullptr, h->flags, s);
    SFSEG_LAUNCHED();
    h->sep = true;
    return SFSEG_OK;
}

int sfseg_power_iterate(sfseg_handle* h, const void* features, int dtype, const float* weights, float bias,
                        const sfseg_neighborhood* nb, int iters, int iters_bf16, float* x_inout, int init,
                        int record_every, double* norms_out, void* stream) {
    if (int rc = check_handle(h)) return rc;
    Taps tp;
    if (int rc = make_taps(nb, &tp)) return rc;
    if (iters < 0 || iters > (1 << 20)) return fail(SFSEG_ERR_INVALID_ARG, "iters must be in [0, 2^20]");
    if (!x_inout) return fail(SFSEG_ERR_INVALID_ARG, "null x_inout");
    if (init < SFSEG_INIT_USER || init > SFSEG_INIT_SMAP) return fail(SFSEG_ERR_INVALID_ARG, "bad init");
    if (record_every < 0) return fail(SFSEG_ERR_INVALID_ARG, "record_every must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    const int bf = iters_bf16 < 0 ? 0 : (iters_bf16 > iters ? iters : iters_bf16);
    if (record_every > 0 && bf > 0)
        return fail(SFSEG_ERR_UNSUPPORTED, "recording for the adjoint needs float32 iterations");
    if (record_every > 0 && h->sep && !features)
        return fail(SFSEG_ERR_UNSUPPORTED, "the adjoint is for shared maps (S = F), not separate ones");
    if (bf > 0 && !h->fbf) {
        SFSEG_CUDA(dalloc(&h->fbf, (size_t)h->NP));
        SFSEG_CUDA(cudaMemsetAsync(h->fbf, 0, (size_t)h->NP * sizeof(__nv_bfloat16), s));
        h->fbf_valid = false;
    }
    if (features) {
        if (int rc = sfseg_set_features(h, features, dtype, weights, bias, stream)) return rc;
    } else if (!h->features_set) {
        return fail(SFSEG_ERR_STATE, "no features: pass them or call sfseg_set_features first");
    }
    if (bf > 0 && !h->fbf_valid) {
        launch_to_bf16(h->f32, h->fbf, h->NP, s);
        SFSEG_LAUNCHED();
        h->fbf_valid = true;
    }
    const bool record = record_every > 0;
    double* acc = nullptr;
    if (record) {
        if (int rc = ensure_acc(&h->rec_acc, &h->rec_acc_cap, iters + 2)) return rc;
        acc = h->rec_acc;
        const int need = (iters > 0 ? (iters - 1) / record_every + 1 : 1) + 1;
        while ((int)h->ckpt.size() < need) {
            float* p = nullptr;
            SFSEG_CUDA(dalloc(&p, (size_t)h->NP));
            h->ckpt.push_back(p);
        }
        h->rec_valid = false;
    } else {
        if (int rc = ensure_acc(&h->acc, &h->acc_cap, iters + 2)) return rc;
        acc = h->acc;
    }
    // The launch sequence of the call (capturable: no allocation, no host synchronisation).
    auto enqueue = [&](cudaStream_t st) -> int {
        SFSEG_CUDA(cudaMemsetAsync(acc, 0, sizeof(double) * (iters + 1), st));
        const float inv_alpha = (float)(1.0 / h->alpha), p = (float)h->p;
        const int vt0 = bf > 0 ? kBF16 : kF32;
        float* last_ckpt = record ? h->ckpt.back() : nullptr;
        const float* s32 = h->sep ? h->s32 : nullptr;
        launch_prologue(init, x_inout, h->f32, p, h->g, h->vbuf[0], vt0, record ? h->ckpt[0] : nullptr,
                        iters == 0 ? x_inout : nullptr, acc, st, s32);
        SFSEG_LAUNCHED();
        cudaEvent_t ev0 = nullptr, ev1 = nullptr;
        if (h->timing && iters > 0) {
            ev0 = take_event(h);
            ev1 = take_event(h);
            SFSEG_CUDA(cudaEventRecord(ev0, st));
        }
        for (int k = 0; k < iters; ++k) {
            const bool last = k == iters - 1;
            const int vin_t = k < bf ? kBF16 : kF32;
            const int out_t = (k + 1 < bf) ? kBF16 : kF32;
            const void* fptr = k < bf ? (const void*)h->fbf : (const void*)h->f32;
            float* ck = nullptr;
            if (record) {
                if (last) ck = last_ckpt;
                else if ((k + 1) % record_every == 0) ck = h->ckpt[(k + 1) / record_every];
            }
            launch_iterate(h->vbuf[k & 1], vin_t, last ? (void*)x_inout : h->vbuf[(k + 1) & 1], out_t, last, fptr,
                           vin_t, ck, h->g, tp, inv_alpha, p, acc + k, acc + k + 1, h->flags, st, s32);
            SFSEG_LAUNCHED();
        }
        if (ev1) {
            SFSEG_CUDA(cudaEventRecord(ev1, st));
            h->ev_pending.emplace_back(ev0, ev1);
            h->timed_launches += iters;
        }
        launch_scale_inv_norm(x_inout, h->N, acc + iters, h->flags, st);
        SFSEG_LAUNCHED();
        return SFSEG_OK;
    };
    const bool graphable = h->graphs && !record && !norms_out && !h->timing && features == nullptr;
    if (graphable) {
        GraphKey key;
        std::memset(&key, 0, sizeof(key));
        key.kind = 0;
        key.x = x_inout;
        key.f32 = h->f32;
        key.fbf = bf > 0 ? (const void*)h->fbf : nullptr;
        key.v0 = h->vbuf[0];
        key.v1 = h->vbuf[1];
        key.s32 = h->sep ? h->s32 : nullptr;
        key.acc = acc;
        key.iters = iters;
        key.bf = bf;
        key.init = init;
        key.tp = tp;
        if (int rc = run_graph(h, s, key, enqueue)) return rc;
    } else if (int rc = enqueue(s)) {
        return rc;
    }
    if (record) {
        h->rec_K = iters;
        h->rec_every = record_every;
        h->rec_valid = iters > 0;
    }
    if (norms_out) {
        std::vector<double> a((size_t)iters + 1);
        SFSEG_CUDA(cudaMemcpyAsync(a.data(), acc, sizeof(double) * (iters + 1), cudaMemcpyDeviceToHost, s));
        if (int rc = read_flags(h, s)) return rc;
        for (int k = 0; k < iters; ++k) norms_out[k] = std::sqrt(a[k + 1]);
    }
    return SFSEG_OK;
}

int sfseg_enable_graphs(sfseg_handle* h, int on) {
    if (int rc = check_handle(h)) return rc;
    h->graphs = on != 0;
    return SFSEG_OK;
}

int sfseg_enable_iter_timing(sfseg_handle* h, int on) {
    if (int rc = check_handle(h)) return rc;
    h->timing = on != 0;
    return SFSEG_OK;
}

int sfseg_iter_timing(sfseg_handle* h, double* ms, int64_t* launches) {
    if (int rc = check_handle(h)) return rc;
    if (!ms || !launches) return fail(SFSEG_ERR_INVALID_ARG, "null argument");
    double total = 0.0;
    for (auto& pr : h->ev_pending) {
        SFSEG_CUDA(cudaEventSynchronize(pr.second));
        float t = 0.f;
        SFSEG_CUDA(cudaEventElapsedTime(&t, pr.first, pr.second));
        total += t;
        h->ev_free.push_back(pr.first);
        h->ev_free.push_back(pr.second);
    }
    h->ev_pending.clear();
    *ms = total;
    *launches = h->timed_launches;
    h->timed_launches = 0;
    return SFSEG_OK;
}

int sfseg_warmstart(sfseg_handle* h, sfseg_net* net, const void* features, int dtype, const float* x_coarse,
                    float* x0_out, void* stream) {
    if (int rc = check_handle(h)) return rc;
    return sfseg_net_forward(net, features, dtype, h->C, x_coarse, h->g.T, h->g.H, h->g.W, x0_out, stream);
}

int sfseg_kernel_launches(int64_t* count) {
    if (!count) return fail(SFSEG_ERR_INVALID_ARG, "null argument");
    *count = launches_so_far();
    return SFSEG_OK;
}

int sfseg_sumsq(sfseg_handle* h, const float* x, int64_t n, double* acc_dev, void* stream) {
    if (int rc = check_handle(h)) return rc;
    if (!x || !acc_dev) return fail(SFSEG_ERR_INVALID_ARG, "null argument");
    if (n < 0) return fail(SFSEG_ERR_INVALID_ARG, "n must be >= 0");
    if (n == 0) return SFSEG_OK;
    launch_sumsq(x, n, acc_dev, (cudaStream_t)stream);
    SFSEG_LAUNCHED();
    return SFSEG_OK;
}

int sfseg_normalize(sfseg_handle* h, float* x, int64_t n, const double* acc_dev, void* stream) {
    if (int rc = check_handle(h)) return rc;
    if (!x || !acc_dev) return fail(SFSEG_ERR_INVALID_ARG, "null argument");
    if (n < 0) return fail(SFSEG_ERR_INVALID_ARG, "n must be >= 0");
    if (n == 0) return SFSEG_OK;
    launch_scale_inv_norm(x, n, acc_dev, h->flags, (cudaStream_t)stream);
    SFSEG_LAUNCHED();
    return SFSEG_OK;
}

int sfseg_check(sfseg_handle* h, void* stream) {
    if (int rc = check_handle(h)) return rc;
    return read_flags(h, (cudaStream_t)stream);
}

int sfseg_iterate_kernel_stats(int64_t* tma_steps, int64_t* generic_steps, char* last_kernel, int len) {
    if (!tma_steps || !generic_steps) return fail(SFSEG_ERR_INVALID_ARG, "null argument");
    if (last_kernel && len < 1) return fail(SFSEG_ERR_INVALID_ARG, "len must be >= 1");
    iterate_kernel_stats(tma_steps, generic_steps, last_kernel, len);
    return SFSEG_OK;
}

int sfseg_apply(sfseg_handle* h, const sfseg_neighborhood* nb, const float* x, float* y, void* stream) {
    if (int rc = check_handle(h)) return rc;
    Taps tp;
    if (int rc = make_taps(nb, &tp)) return rc;
    if (!x || !y) return fail(SFSEG_ERR_INVALID_ARG, "null x or y");
    if (x == y) return fail(SFSEG_ERR_INVALID_ARG, "x and y must not alias");
    if (!h->features_set) return fail(SFSEG_ERR_STATE, "no features set");
    launch_apply_user(x, y, (float*)h->vbuf[1], h->f32, h->g, tp, (float)(1.0 / h->alpha), (float)h->p, h->flags,
                      (cudaStream_t)stream, h->sep ? h->s32 : nullptr);
    SFSEG_LAUNCHED();
    return SFSEG_OK;
}

// ------------------------------------------------------------- the exact (Eq. 1) kernel
namespace {
constexpr int kExactMaxTerms = 120;   // 40 launches of three terms

// The series length N + 1: n_terms if given, else the smallest N whose tail bound
// x^(N+1)/(N+1)! e^x (x = 2 alpha max(f)^2, relative to the series' sum >= 1) is below 2^-24.
int exact_terms(sfseg_handle* h, int n_terms, cudaStream_t s, int* terms_out) {
    if (n_terms < 0 || n_terms > kExactMaxTerms)
        return fail(SFSEG_ERR_INVALID_ARG, "n_terms must be in [0, 120] (0: chosen from alpha and max f)");
    if (n_terms > 0) {
        *terms_out = n_terms;
        return SFSEG_OK;
    }
    unsigned* key = reinterpret_cast<unsigned*>(h->scratch + kScrMaxKey);
    SFSEG_CUDA(cudaMemsetAsync(key, 0, sizeof(unsigned), s));
    launch_max_key(h->f32, h->NP, key, s);
    SFSEG_LAUNCHED();
    unsigned k = 0;
    SFSEG_CUDA(cudaMemcpyAsync(&k, key, sizeof(k), cudaMemcpyDeviceToHost, s));
    SFSEG_CUDA(cudaStreamSynchronize(s));
    uint32_t b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    float fmax;
    std::memcpy(&fmax, &b, sizeof(fmax));
    const double x = 2.0 * h->alpha * (double)fmax * fmax;
    double tail = x * std::exp(x);   // x^(N+1)/(N+1)! e^x for N = 0
    for (int n = 1; n <= kExactMaxTerms; ++n) {
        if (tail <= std::ldexp(1.0, -24)) {
            *terms_out = n;
            return SFSEG_OK;
        }
        tail *= x / (n + 1);
    }
    return fail(SFSEG_ERR_UNSUPPORTED, "alpha * max(f)^2 too large for the series form of the exact kernel");
}

// y = (1/alpha) M x~ s (s = 1/sqrt(*acc_in), or 1), internal layout; acc_out += ||y||^2.
int exact_apply(sfseg_handle* h, const Taps& tp, int terms, const float* xt, const double* acc_in, float* y,
                double* acc_out, cudaStream_t s) {
    const double a = h->alpha;
    std::vector<double> c((size_t)terms + 2, 0.0);
    c[0] = 1.0;
    for (int n = 1; n < terms; ++n) c[n] = c[n - 1] * 2.0 * a / n;
    const int groups = (terms + 2) / 3;
    for (int j = 0; j < groups; ++j) {
        launch_exact_prep(xt, acc_in, h->f32, (float)a, (float)h->p, j, h->g, h->exv, h->flags, s);
        SFSEG_LAUNCHED();
        ExactTerm ex;
        ex.j = j;
        ex.last = j == groups - 1;
        for (int i = 0; i < 3; ++i) ex.c[i] = 3 * j + i < terms ? (float)c[3 * j + i] : 0.f;
        ex.alpha = (float)a;
        if (!launch_exact_term_fast(h->exv, y, h->f32, h->g, tp, (float)(1.0 / a), (float)h->p, ex,
                                    ex.last ? acc_out : nullptr, h->flags, s))
            return fail(SFSEG_ERR_CUDA, "the TMA stencil could not be launched");
        SFSEG_LAUNCHED();
    }
    return SFSEG_OK;
}

int exact_checks(sfseg_handle* h, const Taps& tp) {
    if (!h->features_set) return fail(SFSEG_ERR_STATE, "no features set");
    if (h->sep) return fail(SFSEG_ERR_UNSUPPORTED, "the exact kernel is for shared maps (S = F)");
    if (!fast_iterate_supported(tp))
        return fail(SFSEG_ERR_UNSUPPORTED, "the exact kernel runs on the radii with a TMA kernel only");
    if (!h->exv) SFSEG_CUDA(dalloc(&h->exv, (size_t)h->NP));
    return SFSEG_OK;
}
}  // namespace

int sfseg_apply_exact(sfseg_handle* h, const sfseg_neighborhood* nb, int n_terms, const float* x, float* y,
                      void* stream) {
    if (int rc = check_handle(h)) return rc;
    Taps tp;
    if (int rc = make_taps(nb, &tp)) return rc;
    if (!x || !y) return fail(SFSEG_ERR_INVALID_ARG, "null x or y");
    if (x == y) return fail(SFSEG_ERR_INVALID_ARG, "x and y must not alias");
    if (int rc = exact_checks(h, tp)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    int terms = 0;
    if (int rc = exact_terms(h, n_terms, s, &terms)) return rc;
    float* xt = (float*)h->vbuf[0];
    float* yt = (float*)h->vbuf[1];
    launch_exact_in(x, h->g, xt, nullptr, s);
    SFSEG_LAUNCHED();
    if (int rc = exact_apply(h, tp, terms, xt, nullptr, yt, nullptr, s)) return rc;
    launch_exact_out(yt, nullptr, h->g, y, h->flags, s);
    SFSEG_LAUNCHED();
    return SFSEG_OK;
}

int sfseg_power_iterate_exact(sfseg_handle* h, const sfseg_neighborhood* nb, int n_terms, int iters, int init,
                              float* x_inout, double* norms_out, void* stream) {
    if (int rc = check_handle(h)) return rc;
    Taps tp;
    if (int rc = make_taps(nb, &tp)) return rc;
    if (!x_inout) return fail(SFSEG_ERR_INVALID_ARG, "null x_inout");
    if (iters < 0) return fail(SFSEG_ERR_INVALID_ARG, "iters must be >= 0");
    if (init != SFSEG_INIT_USER && init != SFSEG_INIT_UNIFORM)
        return fail(SFSEG_ERR_INVALID_ARG, "init must be SFSEG_INIT_USER or SFSEG_INIT_UNIFORM");
    if (int rc = exact_checks(h, tp)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    int terms = 0;
    if (int rc = exact_terms(h, n_terms, s, &terms)) return rc;
    if (int rc = ensure_acc(&h->acc, &h->acc_cap, iters + 2)) return rc;
    double* acc = h->acc;
    SFSEG_CUDA(cudaMemsetAsync(acc, 0, sizeof(double) * (iters + 1), s));
    float* buf[2] = {(float*)h->vbuf[0], (float*)h->vbuf[1]};
    launch_exact_in(init == SFSEG_INIT_USER ? x_inout : nullptr, h->g, buf[0], acc, s);
    SFSEG_LAUNCHED();
    for (int k = 0; k < iters; ++k)
        if (int rc = exact_apply(h, tp, terms, buf[k & 1], acc + k, buf[(k + 1) & 1], acc + k + 1, s)) return rc;
    launch_exact_out(buf[iters & 1], acc + iters, h->g, x_inout, h->flags, s);
    SFSEG_LAUNCHED();
    if (norms_out) {
        std::vector<double> a((size_t)iters + 1);
        SFSEG_CUDA(cudaMemcpyAsync(a.data(), acc, sizeof(double) * (iters + 1), cudaMemcpyDeviceToHost, s));
        if (int rc = read_flags(h, s)) return rc;
        for (int k = 0; k < iters; ++k) norms_out[k] = std::sqrt(a[k + 1]);
    }
    return SFSEG_OK;
}

int sfseg_rayleigh(sfseg_handle* h, const sfseg_neighborhood* nb, const float* x, double* rho, double* residual,
                   void* stream) {
    if (int rc = check_handle(h)) return rc;
    Taps tp;
    if (int rc = make_taps(nb, &tp)) return rc;
    if (!x) return fail(SFSEG_ERR_INVALID_ARG, "null x");
    if (!h->features_set) return fail(SFSEG_ERR_STATE, "no features set");
    cudaStream_t s = (cudaStream_t)stream;
    float* y = (float*)h->vbuf[0];
    double* a = h->scratch + kScrRayleigh;
    SFSEG_CUDA(cudaMemsetAsync(a, 0, sizeof(double) * 4, s));
    launch_apply_user(x, y, (float*)h->vbuf[1], h->f32, h->g, tp, (float)(1.0 / h->alpha), (float)h->p, h->flags, s,
                      h->sep ? h->s32 : nullptr);
    launch_dot2(x, y, h->N, a, s);
    launch_resid(x, y, h->N, a, s);
    SFSEG_LAUNCHED();
    double hv[3];
    SFSEG_CUDA(cudaMemcpyAsync(hv, a, sizeof(hv), cudaMemcpyDeviceToHost, s));
    if (int rc = read_flags(h, s)) return rc;
    if (!(hv[1] > 0.0)) return fail(SFSEG_ERR_ZERO_NORM, "x is zero");
    const double r = hv[0] / hv[1];
    if (rho) *rho = r;
    if (residual) *residual = std::sqrt(hv[2] / hv[1]) / r;
    return SFSEG_OK;
}

int sfseg_backward(sfseg_handle* h, const sfseg_neighborhood* nb, const float* grad_x, float* grad_weights,
                   float* grad_bias, void* stream) {
    if (int rc = check_handle(h)) return rc;
    Taps tp;
    if (int rc = make_taps(nb, &tp)) return rc;
    if (!grad_x || !grad_weights || !grad_bias) return fail(SFSEG_ERR_INVALID_ARG, "null argument");
    if (h->C < 2) return fail(SFSEG_ERR_UNSUPPORTED, "the single-channel map has no weights to learn");
    if (!h->rec_valid || h->rec_K < 1 || h->rec_every < 1 || h->ckpt.empty())
        return fail(SFSEG_ERR_STATE, "no recorded forward pass (power_iterate with record_every > 0)");
    cudaStream_t s = (cudaStream_t)stream;
    const int K = h->rec_K, c = h->rec_every;
    const float inv_alpha = (float)(1.0 / h->alpha), p = (float)h->p;
    for (int i = 0; i < 2; ++i)
        if (!h->gbuf[i]) SFSEG_CUDA(dalloc(&h->gbuf[i], (size_t)h->NP));
    if (!h->gz) SFSEG_CUDA(dalloc(&h->gz, (size_t)h->NP));
    const bool fast_adj = fast_iterate_supported(tp);
    if (fast_adj)
        for (float*& q : h->adjw)
            if (!q) SFSEG_CUDA(dalloc(&q, (size_t)h->NP));
    while ((int)h->seg.size() < c + 1) {
        float* q = nullptr;
        SFSEG_CUDA(dalloc(&q, (size_t)h->NP));
        h->seg.push_back(q);
    }
    while (fast_adj && (int)h->qxs.size() < c) {
        float* q = nullptr;
        SFSEG_CUDA(dalloc(&q, (size_t)h->NP));
        h->qxs.push_back(q);
    }
    if (int rc = ensure_acc(&h->dots, &h->dots_cap, K + 2)) return rc;
    // The launch sequence of the reverse pass (capturable: no allocation, no host synchronisation).
    auto enqueue = [&](cudaStream_t st) -> int {
        SFSEG_CUDA(cudaMemsetAsync(h->gz, 0, sizeof(float) * h->NP, st));
        SFSEG_CUDA(cudaMemsetAsync(h->dots, 0, sizeof(double) * (K + 1), st));
        SFSEG_CUDA(cudaMemsetAsync(h->scratch, 0, sizeof(double) * kScrDoubles, st));
        float* xK = h->ckpt.back();
        launch_grad_in(grad_x, xK, h->rec_acc + K, h->gbuf[0], h->g, h->dots + K, st);
        SFSEG_LAUNCHED();
        const int nseg = (K + c - 1) / c;
        if (fast_adj) {
            // State form on the TMA kernel: V_k in seg[k - k0], Q_x(k) in qxs[k - k0], Q_g in adjw[0],
            // v_g alternating between adjw[1] and adjw[2], G_k in gbuf[1]; dots[k] = sum V_k B (k < K).
            float* vg_cur = h->adjw[1];
            float* vg_nxt = h->adjw[2];
            launch_adjoint_first(xK, h->rec_acc + K, h->gbuf[0], h->dots + K, h->f32, p, h->g, vg_cur, st);
            SFSEG_LAUNCHED();
            for (int sgi = nseg - 1; sgi >= 0; --sgi) {
                const int k0 = sgi * c, k1 = (k0 + c < K) ? k0 + c : K, n = k1 - k0;
                launch_state_internal(h->ckpt[sgi], h->f32, p, h->g, h->seg[0], st);
                SFSEG_LAUNCHED();
                // V_{k0+i} by the plain step from the recorded norm, with Q_x(k0+i-1) of the same
                // filtering; the segment's last Q_x by the Q-pass alone
                for (int i = 1; i < n; ++i) {
                    if (!launch_step_q_fast(h->seg[i - 1], h->seg[i], h->qxs[i - 1], h->f32, h->g, tp, inv_alpha, p,
                                            h->rec_acc + k0 + i - 1, h->flags, st))
                        return fail(SFSEG_ERR_CUDA, "the TMA stencil could not be launched");
                    SFSEG_LAUNCHED();
                }
                if (!launch_filter_fast(h->seg[n - 1], 1, h->qxs[n - 1], nullptr, h->f32, h->g, tp, inv_alpha, p,
                                        h->rec_acc + k1 - 1, h->flags, st))
                    return fail(SFSEG_ERR_CUDA, "the TMA stencil could not be launched");
                SFSEG_LAUNCHED();
                for (int k = k1 - 1; k >= k0; --k) {
                    const float* Vk = h->seg[k - k0];
                    if (!launch_adjoint_gpass_fast(vg_cur, h->gbuf[1], h->adjw[0], Vk, h->f32, h->g, tp, inv_alpha, p,
                                                   h->dots + k, h->flags, st))
                        return fail(SFSEG_ERR_CUDA, "the TMA stencil could not be launched");
                    launch_adjoint_combine_state(h->f32, vg_cur, h->qxs[k - k0], Vk, h->adjw[0], h->gbuf[1],
                                                 h->rec_acc + k, h->dots + k, h->g, h->gz, k > 0 ? vg_nxt : nullptr, st);
                    SFSEG_LAUNCHED();
                    std::swap(vg_cur, vg_nxt);
                }
            }
            launch_weight_grad(h->feat_ptr, h->feat_dtype, h->C, h->g, h->gz, h->scratch + kScrWeightGrad, st);
            SFSEG_LAUNCHED();
            return SFSEG_OK;
        }
        int gi = 0;   // gbuf[gi] holds g_{k+1}
        for (int sgi = nseg - 1; sgi >= 0; --sgi) {
            const int k0 = sgi * c, k1 = (k0 + c < K) ? k0 + c : K;
            std::vector<const float*> xs((size_t)(k1 - k0 + 1));
            xs[0] = h->ckpt[sgi];
            for (int i = 1; i <= k1 - k0; ++i) {
                if (k0 + i == K) {
                    xs[i] = xK;
                } else {   // recompute x~_{k0+i} = A x_{k0+i-1} from the recorded norm
                    launch_apply(xs[i - 1], h->g.pitch, h->seg[i], h->g.pitch, h->f32, h->g, tp, inv_alpha, p,
                                 h->rec_acc + k0 + i - 1, h->scratch + kScrApplyAcc, h->flags, st);
                    SFSEG_LAUNCHED();
                    xs[i] = h->seg[i];
                }
            }
            for (int k = k1 - 1; k >= k0; --k) {
                float* gnext = k > 0 ? h->gbuf[gi ^ 1] : nullptr;
                launch_adjoint_step(xs[k - k0], h->rec_acc + k, xs[k + 1 - k0], h->rec_acc + k + 1, h->gbuf[gi],
                                    h->dots + k + 1, gnext, h->dots + k, h->gz, h->f32, h->g, tp, inv_alpha, p, st);
                SFSEG_LAUNCHED();
                gi ^= 1;
            }
        }
        launch_weight_grad(h->feat_ptr, h->feat_dtype, h->C, h->g, h->gz, h->scratch + kScrWeightGrad, st);
        SFSEG_LAUNCHED();
        return SFSEG_OK;
    };
    if (h->graphs) {
        GraphKey key;
        std::memset(&key, 0, sizeof(key));
        key.kind = 1;
        key.x = grad_x;
        key.f32 = h->f32;
        key.fbf = h->feat_ptr;
        key.v0 = h->ckpt[0];
        key.v1 = h->gz;
        key.acc = h->rec_acc;
        key.iters = K;
        key.bf = c;
        key.init = h->feat_dtype;
        key.tp = tp;
        if (int rc = run_graph(h, s, key, enqueue)) return rc;
    } else if (int rc = enqueue(s)) {
        return rc;
    }
    std::vector<double> wacc((size_t)h->C + 1);
    SFSEG_CUDA(cudaMemcpyAsync(wacc.data(), h->scratch + kScrWeightGrad, sizeof(double) * (h->C + 1),
                               cudaMemcpyDeviceToHost, s));
    if (int rc = read_flags(h, s)) return rc;
    for (int ch = 0; ch < h->C; ++ch) grad_weights[ch] = (float)wacc[ch];
    *grad_bias = (float)wacc[h->C];
    return SFSEG_OK;
}

int sfseg_coarse_start(sfseg_handle* h, const sfseg_neighborhood* nb, int levels, double tol, int max_iters,
                       int check_every, float* x0_out, int* iters_out, void* stream) {
    if (int rc = check_handle(h)) return rc;
    Taps tp;
    if (int rc = make_taps(nb, &tp)) return rc;
    if (!x0_out) return fail(SFSEG_ERR_INVALID_ARG, "null x0_out");
    if (levels < 1 || levels > 4) return fail(SFSEG_ERR_INVALID_ARG, "levels must be in [1, 4]");
    if (!(tol > 0.0) || max_iters < 1 || check_every < 1)
        return fail(SFSEG_ERR_INVALID_ARG, "tol > 0, max_iters >= 1 and check_every >= 1 are required");
    if (!h->features_set) return fail(SFSEG_ERR_STATE, "no features set");
    if (h->sep) return fail(SFSEG_ERR_UNSUPPORTED, "the coarse start is for shared maps (S = F)");
    cudaStream_t s = (cudaStream_t)stream;
    // (re)build the pyramid when its depth or shape does not match
    if ((int)h->lvl.size() != levels) {
        for (sfseg_handle* c : h->lvl) sfseg_destroy(c);
        for (float* p : h->lvl_f) cudaFree(p);
        for (float* p : h->lvl_x) cudaFree(p);
        h->lvl.clear();
        h->lvl_f.clear();
        h->lvl_x.clear();
        h->lvl_p.clear();
        int T = h->g.T, H = h->g.H, W = h->g.W;
        sfseg_params prm{h->alpha, h->p};
        for (int l = 0; l < levels; ++l) {
            const int pt = T > 1 ? 2 : 1, ph = H > 1 ? 2 : 1, pw = W > 1 ? 2 : 1;
            T = (T + pt - 1) / pt;
            H = (H + ph - 1) / ph;
            W = (W + pw - 1) / pw;
            sfseg_handle* c = nullptr;
            if (int rc = sfseg_create(&prm, 1, T, H, W, &c)) return rc;
            h->lvl.push_back(c);
            float *fb = nullptr, *xb = nullptr;
            SFSEG_CUDA(cudaMalloc(&fb, sizeof(float) * (size_t)T * H * W));
            SFSEG_CUDA(cudaMalloc(&xb, sizeof(float) * (size_t)T * H * W));
            h->lvl_f.push_back(fb);
            h->lvl_x.push_back(xb);
            h->lvl_p.insert(h->lvl_p.end(), {pt, ph, pw});
        }
    }
    // restriction of f, level by level
    std::vector<sfseg_neighborhood> nbs((size_t)levels);
    double scale[3] = {1.0, 1.0, 1.0};
    for (int l = 0; l < levels; ++l) {
        const sfseg_handle* fine = l == 0 ? h : h->lvl[l - 1];
        sfseg_handle* c = h->lvl[l];
        const int* pf = &h->lvl_p[3 * l];
        launch_pool_f(fine->f32, fine->g, pf[0], pf[1], pf[2], c->g.T, c->g.H, c->g.W, h->lvl_f[l], s);
        SFSEG_LAUNCHED();
        if (int rc = sfseg_set_features(c, h->lvl_f[l], SFSEG_F32, nullptr, 0.f, s)) return rc;
        // the same Gaussian in physical units: widths in coarse pixels, truncated at the same
        // multiple of the width
        const int r[3] = {nb->rt, nb->rh, nb->rw};
        const float sg[3] = {nb->sigma_t, nb->sigma_h, nb->sigma_w};
        int rl[3];
        float sl[3];
        for (int a = 0; a < 3; ++a) {
            scale[a] *= pf[a];
            sl[a] = (float)(sg[a] / scale[a]);
            rl[a] = r[a] == 0 ? 0 : (int)std::max(1.0, std::floor(r[a] / scale[a] + 0.5));
        }
        nbs[(size_t)l] = sfseg_neighborhood{rl[0], rl[1], rl[2], sl[0], sl[1], sl[2]};
    }
    // coarsest level from the uniform start, then each finer level from the upsampled solution
    for (int l = levels - 1; l >= 0; --l) {
        sfseg_handle* c = h->lvl[l];
        int init = SFSEG_INIT_UNIFORM;
        if (l < levels - 1) {
            const sfseg_handle* cc = h->lvl[l + 1];
            const int* pf = &h->lvl_p[3 * (l + 1)];
            launch_upsample(h->lvl_x[l + 1], cc->g.T, cc->g.H, cc->g.W, pf[0], pf[1], pf[2], c->g.T, c->g.H, c->g.W,
                            h->lvl_x[l], s);
            SFSEG_LAUNCHED();
            init = SFSEG_INIT_USER;
        }
        int its = 0, step = check_every, last_its = -1;
        double res = 1e300, last_res = 0.0;
        while (its < max_iters && res > tol) {
            const int k = std::min(step, max_iters - its);
            if (int rc = sfseg_power_iterate(c, nullptr, 0, nullptr, 0.f, &nbs[(size_t)l], k, 0, h->lvl_x[l], init, 0,
                                             nullptr, stream))
                return rc;
            init = SFSEG_INIT_USER;
            its += k;
            if (int rc = sfseg_rayleigh(c, &nbs[(size_t)l], h->lvl_x[l], nullptr, &res, stream)) return rc;
            // next check where the residual's geometric rate over the last two checks predicts
            // tol (a multiple of 10 iterations, between check_every and 8 check_every away)
            step = check_every;
            if (last_its >= 0 && res > tol && res > 0.0 && res < last_res) {
                const double rate = std::log(res / last_res) / (double)(its - last_its);
                const double need = std::log(tol / res) / rate;
                const double r10 = std::ceil(need / 10.0) * 10.0;
                step = (int)std::min(std::max(r10, (double)check_every), 8.0 * check_every);
            }
            last_its = its;
            last_res = res;
        }
        if (iters_out) iters_out[l] = its;
    }
    const int* pf = &h->lvl_p[0];
    const sfseg_handle* c0 = h->lvl[0];
    launch_upsample(h->lvl_x[0], c0->g.T, c0->g.H, c0->g.W, pf[0], pf[1], pf[2], h->g.T, h->g.H, h->g.W, x0_out, s);
    // maximum 1, so that the start vector's scale does not depend on the volume size (it is an
    // input channel of the warm-start network)
    launch_scale_by_max(x0_out, h->N, reinterpret_cast<unsigned*>(h->scratch + kScrMaxKey), s);
    SFSEG_LAUNCHED();
    return SFSEG_OK;
}

int sfseg_soft_binarize(sfseg_handle* h, const sfseg_neighborhood* nb, int iters, float gain, float center,
                        float* x_inout, unsigned char* mask_out, void* stream) {
    if (int rc = check_handle(h)) return rc;
    Taps tp;
    if (int rc = make_taps(nb, &tp)) return rc;
    if (!x_inout) return fail(SFSEG_ERR_INVALID_ARG, "null x_inout");
    if (iters < 1 || iters > (1 << 20)) return fail(SFSEG_ERR_INVALID_ARG, "iters must be in [1, 2^20]");
    if (!(gain >= 0.f) || !std::isfinite(gain) || !std::isfinite(center))
        return fail(SFSEG_ERR_INVALID_ARG, "gain must be finite and >= 0, center finite");
    if (!h->features_set) return fail(SFSEG_ERR_STATE, "no features set");
    cudaStream_t s = (cudaStream_t)stream;
    const float inv_alpha = (float)(1.0 / h->alpha), p = (float)h->p;
    float* y = (float*)h->vbuf[0];                     // A x, caller layout
    float* v = (float*)h->vbuf[1];                     // u * x, internal layout
    unsigned* key = reinterpret_cast<unsigned*>(h->scratch + kScrMaxKey);
    const bool fast = fast_iterate_supported(tp);
    const float* s32 = h->sep ? h->s32 : nullptr;
    for (int k = 0; k < iters; ++k) {
        const bool last = k == iters - 1;
        bool fused = false;   // the stencil took max(y) itself (shared maps, a compiled radius)
        if (fast && !s32) {
            SFSEG_CUDA(cudaMemsetAsync(key, 0, sizeof(unsigned), s));
            if (k == 0) launch_to_state(x_inout, h->f32, nullptr, p, h->g, v, s);
            fused = launch_iterate_fast_max(v, y, h->f32, h->g, tp, inv_alpha, p, key, h->flags, s);
            if (!fused && k > 0) return fail(SFSEG_ERR_CUDA, "stencil launch failed");
        }
        if (!fused) {
            if (k == 0 || !fast)
                launch_apply_user(x_inout, y, v, h->f32, h->g, tp, inv_alpha, p, h->flags, s, s32);
            else if (!launch_iterate_fast(v, kF32, y, kF32, true, h->f32, h->g, tp, inv_alpha, p, nullptr, nullptr,
                                          h->flags, s, s32))
                return fail(SFSEG_ERR_CUDA, "stencil launch failed");
            launch_max_key(y, h->N, key, s);
        }
        launch_sigmoid_step(y, key, gain, center, h->f32, p, h->g, x_inout, (fast && !last) ? v : nullptr,
                            last ? mask_out : nullptr, h->flags, s, s32);
        SFSEG_LAUNCHED();
    }
    return read_flags(h, s);
}

int sfseg_selftest_wait(sfseg_handle* h, long long spins, void* stream) {
    if (int rc = check_handle(h)) return rc;
    if (spins < 1 || spins > 1000000) return fail(SFSEG_ERR_INVALID_ARG, "spins must be in [1, 1e6]");
    cudaStream_t s = (cudaStream_t)stream;
    launch_wait_probe(spins, h->flags, s);
    SFSEG_LAUNCHED();
    return read_flags(h, s);
}

int sfseg_soft_iou_loss(sfseg_handle* h, const float* x, const float* target, double* loss, float* grad_x,
                        void* stream) {
    if (int rc = check_handle(h)) return rc;
    if (!x || !target || !loss) return fail(SFSEG_ERR_INVALID_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    double* a = h->scratch + kScrSoftIou;
    SFSEG_CUDA(cudaMemsetAsync(a, 0, sizeof(double) * 4, s));
    SFSEG_CUDA(cudaMemsetAsync(h->amax, 0, sizeof(unsigned long long), s));
    launch_soft_iou(x, target, h->N, grad_x, a, h->amax, s);
    SFSEG_LAUNCHED();
    double hv[2];
    SFSEG_CUDA(cudaMemcpyAsync(hv, a, sizeof(hv), cudaMemcpyDeviceToHost, s));
    SFSEG_CUDA(cudaStreamSynchronize(s));
    *loss = 1.0 - hv[0] / hv[1];
    return SFSEG_OK;
}

}  // extern "C"
