// api.cu -- the C ABI of libzncc.so (declared in include/zncc.h): argument checks, the
// context's device scratch, and the launch sequence of each call.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "zncc.h"

using namespace zncc;

namespace {

std::atomic<uint64_t> g_launches{0};
thread_local std::string g_create_error;

// Kernel kinds for per-kernel timing (zncc_profile_*).
enum Kind {
    K_STATS = 0, K_COEF, K_ZNCC_RAW, K_ZNCC_HPAIR, K_ZNCC_WTA, K_DT_HPAIR, K_DT_VPAIR,
    K_DT_VPAIR_WTA, K_WTA_VOLUME, K_NKINDS
};
const char* const kKindNames[K_NKINDS] = {
    "window_stats", "dt_coef", "zncc_cost", "zncc_cost_hpair", "zncc_cost_wta",
    "dt_hpair", "dt_vpair", "dt_vpair_wta", "wta_volume"};

struct ProfRecord {
    int kind, ev0, ev1;
};

constexpr int kTargetBlocks = 1216;   // about eight blocks per SM on a 152-SM GB300

}  // namespace

struct zncc_ctx {
    int W = 0, H = 0, D = 0, win = 0, r = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    float4* coefH = nullptr;      // [H][W]       horizontal DT coefficients
    float4* coefV = nullptr;      // [W][H]       vertical DT coefficients
    void* vol = nullptr;          // the fused path's intermediate volume (on first use)
    size_t vol_bytes = 0;
    float* bestv = nullptr;       // [H][W] running WTA best across launches (on first use)
    int* bestd = nullptr;         // [H][W]
    int smem_max = 0;             // opt-in shared memory per block of the device
    uint8_t* img = nullptr;       // device copies for zncc_run_host: 2 x [H][W]
    uint16_t* disp = nullptr;     // [H][W]
    bool profiling = false;
    std::vector<cudaEvent_t> events;
    int events_used = 0;
    std::vector<ProfRecord> records;
};

namespace {

zncc_status fail(zncc_ctx* c, zncc_status s, const std::string& msg) {
    if (c) c->err = msg;
    else g_create_error = msg;
    return s;
}

zncc_status cuda_fail(zncc_ctx* c, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(c, ZNCC_ECUDA, m);
}

#define ZNCC_CUDA(c, call, what)                                  \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what);     \
    } while (0)

#define ZNCC_TRY(expr)                   \
    do {                                 \
        zncc_status s_ = (expr);         \
        if (s_ != ZNCC_OK) return s_;    \
    } while (0)

// An event of the context's pool (grown on demand), or -1 if one cannot be created.
int prof_event(zncc_ctx* c) {
    if (c->events_used == (int)c->events.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        c->events.push_back(e);
    }
    return c->events_used++;
}

#define ZNCC_LAUNCH(c, kind, call, what)                                      \
    do {                                                                      \
        g_launches.fetch_add(1, std::memory_order_relaxed);                   \
        int ev0_ = -1;                                                        \
        if ((c)->profiling && (ev0_ = prof_event(c)) >= 0)                    \
            cudaEventRecord((c)->events[ev0_], (c)->stream);                  \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what);                 \
        int ev1_ = ev0_ >= 0 ? prof_event(c) : -1;                            \
        if (ev1_ >= 0) {                                                      \
            cudaEventRecord((c)->events[ev1_], (c)->stream);                  \
            (c)->records.push_back(ProfRecord{(kind), ev0_, ev1_});           \
        }                                                                     \
    } while (0)

// The chunk count is padded so that a line's threads fill whole warps (every warp-wide
// shuffle then has all 32 lanes); padded chunks lie past the line end and hold zeros.
int padded_chunks(int n, int tq) {
    const int per_warp = 32 / tq;
    const int nch = (n + kL - 1) / kL;
    return (nch + per_warp - 1) / per_warp * per_warp;
}

// Disparity slices per block: about kTargetBlocks blocks in all, equal runs per block.
int slices_per_block(int nslices, int blocks_x) {
    const int per = std::max(1, blocks_x * nslices / kTargetBlocks);
    const int groups = std::max(1, (nslices + per - 1) / per);
    return (nslices + groups - 1) / groups;
}

zncc_status check_images(zncc_ctx* c, const void* a, const void* b, int pitch) {
    if (!a || !b) return fail(c, ZNCC_EINVAL, "image pointer is NULL");
    if (pitch < c->W) return fail(c, ZNCC_EINVAL, "pitch is smaller than the width");
    return ZNCC_OK;
}

zncc_status check_dt(zncc_ctx* c, float sigma_s, float sigma_r, int iters) {
    if (!(sigma_s > 0.0f) || !isfinite(sigma_s)) return fail(c, ZNCC_EINVAL, "sigma_s must be > 0");
    if (!(sigma_r > 0.0f) || !isfinite(sigma_r)) return fail(c, ZNCC_EINVAL, "sigma_r must be > 0");
    if (iters < 0 || iters > 64) return fail(c, ZNCC_EINVAL, "iters must be in [0, 64]");
    return ZNCC_OK;
}

float scale_s2(float sigma_s) {
    const double s = 1.0 - exp(-1.0 / (double)sigma_s);
    return (float)(s * s);
}

zncc_status run_coef(zncc_ctx* c, const uint8_t* guide, int pitch, float sigma_s, float sigma_r) {
    const float K = (float)exp(-1.0 / (double)sigma_s);
    const float inv = (float)(1.0 / (255.0 * (double)sigma_r));
    ZNCC_LAUNCH(c, K_COEF, launch_dt_coef(guide, pitch, c->W, c->H, K, inv, c->coefH, c->coefV, c->stream),
                "DT coefficients");
    return ZNCC_OK;
}

void free_dev_f(float*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

zncc_status ensure_best(zncc_ctx* c) {
    if (c->bestv) return ZNCC_OK;
    const size_t npix = (size_t)c->W * c->H;
    cudaError_t e = cudaMalloc(&c->bestv, npix * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c->bestd, npix * sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_dev_f(c->bestv);
        return fail(c, ZNCC_ENOMEM, std::string("WTA buffers: ") + cudaGetErrorString(e));
    }
    return ZNCC_OK;
}

// ZNCC row launches over the disparities [0, D): the band of a block covers its disparity
// slices, so the slices per block shrink until the block fits in shared memory. In Wta
// mode a block must see every disparity of its launch, so the disparity range is split
// into several launches chained through the running best when it does not fit.
zncc_status run_rows(zncc_ctx* c, const uint8_t* left, const uint8_t* right, int pitch, int mode, int dtype,
                     void* vol, long long dstride, float s2, uint16_t* disp, int kind, const char* what) {
    RowArgs a;
    memset(&a, 0, sizeof(a));
    a.left = left;
    a.right = right;
    a.pitch = pitch;
    a.W = c->W;
    a.H = c->H;
    a.D = c->D;
    a.tq = c->W <= 1024 ? 8 : (c->W <= 2048 ? 4 : 2);
    a.nch = padded_chunks(c->W, a.tq);
    a.vol = vol;
    a.dstride = dstride;
    a.d_out0 = 0;
    a.vec = vol && (dstride % 4 == 0) && ((uintptr_t)vol % (dtype == 0 ? 16 : 8) == 0) ? 1 : 0;
    a.coef = c->coefH;
    a.s2 = s2;
    const int threads = a.nch * a.tq;
    const int ds = kG * a.tq;
    const int nslices = (c->D + ds - 1) / ds;
    if (mode != kModeWta) {
        a.d_lo = 0;
        a.d_hi = c->D;
        a.spb = slices_per_block(nslices, c->H);
        while (a.spb > 1 && zncc_row_smem_bytes(c->r, mode, a, threads) > (size_t)c->smem_max) --a.spb;
        if (zncc_row_smem_bytes(c->r, mode, a, threads) > (size_t)c->smem_max)
            return fail(c, ZNCC_EUNSUPPORTED, "image too wide for the cost kernel's shared memory");
        ZNCC_LAUNCH(c, kind, launch_zncc_row(c->r, a, mode, dtype, c->stream), what);
        return ZNCC_OK;
    }
    int per_launch = nslices;   // slices of one Wta launch
    for (;;) {
        a.d_lo = 0;
        a.d_hi = std::min(c->D, per_launch * ds);
        a.spb = per_launch;
        if (zncc_row_smem_bytes(c->r, mode, a, threads) <= (size_t)c->smem_max) break;
        if (per_launch == 1) return fail(c, ZNCC_EUNSUPPORTED, "image too wide for the cost kernel's shared memory");
        per_launch = (per_launch + 1) / 2;
    }
    const int nlaunch = (nslices + per_launch - 1) / per_launch;
    if (nlaunch > 1) ZNCC_TRY(ensure_best(c));
    for (int g = 0; g < nlaunch; ++g) {
        a.d_lo = g * per_launch * ds;
        a.d_hi = std::min(c->D, (g + 1) * per_launch * ds);
        a.spb = per_launch;
        a.wta.bestv = c->bestv;
        a.wta.bestd = c->bestd;
        a.wta.disp = disp;
        a.wta.first = g == 0;
        a.wta.last = g == nlaunch - 1;
        ZNCC_LAUNCH(c, kind, launch_zncc_row(c->r, a, mode, dtype, c->stream), what);
    }
    return ZNCC_OK;
}

// One DT pair along rows (horiz) or columns of a [H][W][dstride] volume. The block shape is
// the widest lane count per chunk whose block fits, streaming the next slices through shared
// memory (async) where that fits too.
zncc_status run_line_pair(zncc_ctx* c, void* vol, int dtype, long long dstride, bool horiz, float s2,
                          int mode, uint16_t* disp) {
    LineArgs a;
    memset(&a, 0, sizeof(a));
    const int n = horiz ? c->W : c->H;
    a.vol = vol;
    a.elem_stride = horiz ? dstride : (long long)c->W * dstride;
    a.line_stride = horiz ? (long long)c->W * dstride : dstride;
    a.n = n;
    a.nlines = horiz ? c->H : c->W;
    a.dcount = c->D;
    a.d_base = 0;
    a.coef = horiz ? c->coefH : c->coefV;
    a.coef_line_stride = horiz ? c->W : c->H;
    a.s2 = s2;
    a.vec = (dstride % 4 == 0) && ((uintptr_t)vol % (dtype == 0 ? 16 : 8) == 0) ? 1 : 0;
    a.wta.disp = disp;
    a.wta.first = 1;
    a.wta.last = 1;
    a.pix_line = horiz ? c->W : 1;
    a.pix_pos = horiz ? 1 : c->W;
    bool found = false;
    for (int pass = 0; pass < 2 && !found; ++pass) {          // with, then without, async
        for (int tq = 8; tq >= 2 && !found; tq >>= 1) {
            a.tq = tq;
            a.nch = padded_chunks(n, tq);
            const int per_line = a.nch * tq;
            if (per_line > 512) continue;
            a.async = pass == 0 ? a.vec : 0;
            if (pass == 0 && !a.vec) continue;
            for (a.lpc = std::max(1, std::min(8, 256 / per_line)); a.lpc >= 1; --a.lpc)
                if (line_pair_smem_bytes(mode, dtype, a) <= (size_t)c->smem_max) {
                    found = true;
                    break;
                }
        }
    }
    if (!found) return fail(c, ZNCC_EUNSUPPORTED, "line too long for the DT kernel's shared memory");
    const int nslices = (c->D + kG * a.tq - 1) / (kG * a.tq);
    a.spb = mode == kLineWta ? nslices : slices_per_block(nslices, (a.nlines + a.lpc - 1) / a.lpc);
    const int kind = horiz ? K_DT_HPAIR : (mode == kLineWta ? K_DT_VPAIR_WTA : K_DT_VPAIR);
    ZNCC_LAUNCH(c, kind, launch_line_pair(a, mode, dtype, c->stream), horiz ? "DT horizontal pair" : "DT vertical pair");
    return ZNCC_OK;
}

template <typename T>
void free_dev(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

void release(zncc_ctx* c) {
    free_dev(c->coefH);
    free_dev(c->coefV);
    free_dev(c->vol);
    free_dev(c->bestv);
    free_dev(c->bestd);
    free_dev(c->img);
    free_dev(c->disp);
    for (cudaEvent_t e : c->events) cudaEventDestroy(e);
    c->events.clear();
    c->records.clear();
    c->events_used = 0;
}

}  // namespace

extern "C" {

zncc_status zncc_create(int width, int height, int max_disp, int win, zncc_ctx** out) {
    g_create_error.clear();
    if (!out) return fail(nullptr, ZNCC_EINVAL, "out is NULL");
    *out = nullptr;
    if (width < 1 || height < 1) return fail(nullptr, ZNCC_EINVAL, "width and height must be >= 1");
    if (width > 4096 || height > 4096)
        return fail(nullptr, ZNCC_EUNSUPPORTED, "width and height must be <= 4096");
    if (max_disp < 1) return fail(nullptr, ZNCC_EINVAL, "max_disp must be >= 1");
    if (max_disp > 1024) return fail(nullptr, ZNCC_EUNSUPPORTED, "max_disp must be <= 1024");
    if (win < 3 || win > 15 || win % 2 == 0)
        return fail(nullptr, ZNCC_EINVAL, "win must be odd and in [3, 15]");
    zncc_ctx* c = new (std::nothrow) zncc_ctx();
    if (!c) return fail(nullptr, ZNCC_ENOMEM, "host allocation failed");
    c->W = width;
    c->H = height;
    c->D = max_disp;
    c->win = win;
    c->r = win / 2;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    const size_t npix = (size_t)width * height;
    if (e == cudaSuccess) e = cudaMalloc(&c->coefH, npix * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&c->coefV, npix * sizeof(float4));
    if (e != cudaSuccess) {
        zncc_status s = e == cudaErrorMemoryAllocation ? ZNCC_ENOMEM : ZNCC_ECUDA;
        std::string m = std::string("zncc_create: ") + cudaGetErrorString(e);
        cudaGetLastError();
        release(c);
        delete c;
        return fail(nullptr, s, m);
    }
    *out = c;
    return ZNCC_OK;
}

zncc_status zncc_destroy(zncc_ctx* c) {
    if (!c) return ZNCC_EINVAL;
    cudaStreamSynchronize(c->stream);
    release(c);
    delete c;
    return ZNCC_OK;
}

zncc_status zncc_set_stream(zncc_ctx* c, void* stream) {
    if (!c) return ZNCC_EINVAL;
    c->stream = (cudaStream_t)stream;
    return ZNCC_OK;
}

size_t zncc_volume_bytes(const zncc_ctx* c, zncc_dtype dtype) {
    if (!c || (dtype != ZNCC_F32 && dtype != ZNCC_F16)) return 0;
    return (size_t)c->W * c->H * c->D * (dtype == ZNCC_F32 ? 4 : 2);
}

zncc_status zncc_window_stats(zncc_ctx* c, const uint8_t* img, int pitch, int32_t* S, int32_t* Q,
                              float* inv_sigma) {
    if (!c) return ZNCC_EINVAL;
    c->err.clear();
    if (!img) return fail(c, ZNCC_EINVAL, "image pointer is NULL");
    if (pitch < c->W) return fail(c, ZNCC_EINVAL, "pitch is smaller than the width");
    if (!S && !Q && !inv_sigma) return ZNCC_OK;
    ZNCC_LAUNCH(c, K_STATS, launch_window_stats(img, pitch, c->W, c->H, c->r, 0, c->W, S, Q, inv_sigma,
                                                nullptr, c->stream), "window statistics");
    return ZNCC_OK;
}

zncc_status zncc_cost_volume(zncc_ctx* c, const uint8_t* left, const uint8_t* right, int pitch,
                             void* cost, zncc_dtype dtype) {
    if (!c) return ZNCC_EINVAL;
    c->err.clear();
    ZNCC_TRY(check_images(c, left, right, pitch));
    if (!cost) return fail(c, ZNCC_EINVAL, "cost pointer is NULL");
    if (dtype != ZNCC_F32 && dtype != ZNCC_F16) return fail(c, ZNCC_EINVAL, "unknown dtype");
    return run_rows(c, left, right, pitch, kModeRaw, dtype, cost, c->D, 0.0f, nullptr, K_ZNCC_RAW, "ZNCC cost");
}

zncc_status dt_aggregate(zncc_ctx* c, const uint8_t* guide, int pitch, void* cost, zncc_dtype dtype,
                         float sigma_s, float sigma_r, int iters) {
    if (!c) return ZNCC_EINVAL;
    c->err.clear();
    if (!guide) return fail(c, ZNCC_EINVAL, "guide pointer is NULL");
    if (pitch < c->W) return fail(c, ZNCC_EINVAL, "pitch is smaller than the width");
    if (!cost) return fail(c, ZNCC_EINVAL, "cost pointer is NULL");
    if (dtype != ZNCC_F32 && dtype != ZNCC_F16) return fail(c, ZNCC_EINVAL, "unknown dtype");
    ZNCC_TRY(check_dt(c, sigma_s, sigma_r, iters));
    if (iters == 0) return ZNCC_OK;
    ZNCC_TRY(run_coef(c, guide, pitch, sigma_s, sigma_r));
    const float s2 = scale_s2(sigma_s);
    for (int it = 0; it < iters; ++it) {
        ZNCC_TRY(run_line_pair(c, cost, dtype, c->D, true, s2, kLineStore, nullptr));
        ZNCC_TRY(run_line_pair(c, cost, dtype, c->D, false, s2, kLineStore, nullptr));
    }
    return ZNCC_OK;
}

zncc_status wta_disparity(zncc_ctx* c, const void* cost, zncc_dtype dtype, uint16_t* disp) {
    if (!c) return ZNCC_EINVAL;
    c->err.clear();
    if (!cost || !disp) return fail(c, ZNCC_EINVAL, "cost or disp pointer is NULL");
    if (dtype != ZNCC_F32 && dtype != ZNCC_F16) return fail(c, ZNCC_EINVAL, "unknown dtype");
    ZNCC_LAUNCH(c, K_WTA_VOLUME, launch_wta_volume(cost, dtype, c->W, c->H, c->D, disp, c->stream), "WTA");
    return ZNCC_OK;
}

zncc_status zncc_run(zncc_ctx* c, const uint8_t* left, const uint8_t* right, int pitch, float sigma_s,
                     float sigma_r, int iters, zncc_dtype storage, uint16_t* disp) {
    if (!c) return ZNCC_EINVAL;
    c->err.clear();
    ZNCC_TRY(check_images(c, left, right, pitch));
    if (!disp) return fail(c, ZNCC_EINVAL, "disp pointer is NULL");
    if (storage != ZNCC_F32 && storage != ZNCC_F16) return fail(c, ZNCC_EINVAL, "unknown dtype");
    ZNCC_TRY(check_dt(c, sigma_s, sigma_r, iters));
    const size_t npix = (size_t)c->W * c->H;

    if (iters == 0) return run_rows(c, left, right, pitch, kModeWta, 0, nullptr, 0, 0.0f, disp, K_ZNCC_WTA, "ZNCC + WTA");
    const int dt = storage == ZNCC_F32 ? 0 : 1;
    const long long dstride = (c->D + 3) / 4 * 4;   // padded so every access is vectorised
    const size_t need = npix * (size_t)dstride * (dt == 0 ? 4 : 2);
    if (c->vol_bytes < need) {
        free_dev(c->vol);
        c->vol_bytes = 0;
        cudaError_t e = cudaMalloc(&c->vol, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, e == cudaErrorMemoryAllocation ? ZNCC_ENOMEM : ZNCC_ECUDA,
                        std::string("cost volume allocation: ") + cudaGetErrorString(e));
        }
        c->vol_bytes = need;
    }
    ZNCC_TRY(run_coef(c, left, pitch, sigma_s, sigma_r));
    const float s2 = scale_s2(sigma_s);
    ZNCC_TRY(run_rows(c, left, right, pitch, kModeHPair, dt, c->vol, dstride, s2, nullptr, K_ZNCC_HPAIR,
                      "ZNCC + horizontal DT pair"));
    for (int it = 0; it < iters; ++it) {
        const bool last = it == iters - 1;
        ZNCC_TRY(run_line_pair(c, c->vol, dt, dstride, false, s2, last ? kLineWta : kLineStore, disp));
        if (!last) ZNCC_TRY(run_line_pair(c, c->vol, dt, dstride, true, s2, kLineStore, nullptr));
    }
    return ZNCC_OK;
}

zncc_status zncc_run_host(zncc_ctx* c, const uint8_t* left_host, const uint8_t* right_host, int pitch,
                          float sigma_s, float sigma_r, int iters, zncc_dtype storage,
                          uint16_t* disp_host) {
    if (!c) return ZNCC_EINVAL;
    c->err.clear();
    ZNCC_TRY(check_images(c, left_host, right_host, pitch));
    if (!disp_host) return fail(c, ZNCC_EINVAL, "disp_host pointer is NULL");
    const size_t npix = (size_t)c->W * c->H;
    if (!c->img) {
        cudaError_t e = cudaMalloc(&c->img, 2 * npix);
        if (e == cudaSuccess) e = cudaMalloc(&c->disp, npix * sizeof(uint16_t));
        if (e != cudaSuccess) {
            cudaGetLastError();
            free_dev(c->img);
            free_dev(c->disp);
            return fail(c, ZNCC_ENOMEM, std::string("image buffers: ") + cudaGetErrorString(e));
        }
    }
    ZNCC_CUDA(c, cudaMemcpy2DAsync(c->img, c->W, left_host, pitch, c->W, c->H, cudaMemcpyHostToDevice, c->stream),
              "left image upload");
    ZNCC_CUDA(c, cudaMemcpy2DAsync(c->img + npix, c->W, right_host, pitch, c->W, c->H, cudaMemcpyHostToDevice,
                                   c->stream), "right image upload");
    ZNCC_TRY(zncc_run(c, c->img, c->img + npix, c->W, sigma_s, sigma_r, iters, storage, c->disp));
    ZNCC_CUDA(c, cudaMemcpyAsync(disp_host, c->disp, npix * sizeof(uint16_t), cudaMemcpyDeviceToHost, c->stream),
              "disparity download");
    ZNCC_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
    return ZNCC_OK;
}

const char* zncc_last_error(const zncc_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

const char* zncc_status_string(zncc_status s) {
    switch (s) {
        case ZNCC_OK: return "ZNCC_OK";
        case ZNCC_EINVAL: return "ZNCC_EINVAL";
        case ZNCC_ENOMEM: return "ZNCC_ENOMEM";
        case ZNCC_ECUDA: return "ZNCC_ECUDA";
        case ZNCC_EBUSY: return "ZNCC_EBUSY";
        case ZNCC_ENOTREADY: return "ZNCC_ENOTREADY";
        case ZNCC_ETIMEOUT: return "ZNCC_ETIMEOUT";
        case ZNCC_EUNSUPPORTED: return "ZNCC_EUNSUPPORTED";
    }
    return "unknown status";
}

uint64_t zncc_kernel_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

zncc_status zncc_profile_enable(zncc_ctx* c, int enable) {
    if (!c) return ZNCC_EINVAL;
    c->profiling = enable != 0;
    return ZNCC_OK;
}

zncc_status zncc_profile_read(zncc_ctx* c, double* total_ms, uint64_t* launches, int nkinds) {
    if (!c || nkinds < 0 || (nkinds > 0 && (!total_ms || !launches))) return ZNCC_EINVAL;
    c->err.clear();
    for (int k = 0; k < nkinds; ++k) {
        total_ms[k] = 0.0;
        launches[k] = 0;
    }
    ZNCC_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
    for (const ProfRecord& r : c->records) {
        float ms = 0.0f;
        ZNCC_CUDA(c, cudaEventElapsedTime(&ms, c->events[r.ev0], c->events[r.ev1]), "event time");
        if (r.kind < nkinds) {
            total_ms[r.kind] += ms;
            launches[r.kind] += 1;
        }
    }
    c->records.clear();
    c->events_used = 0;
    return ZNCC_OK;
}

int zncc_profile_nkinds(void) { return K_NKINDS; }

const char* zncc_profile_kind_name(int kind) {
    return kind >= 0 && kind < K_NKINDS ? kKindNames[kind] : nullptr;
}

}  // extern "C"
