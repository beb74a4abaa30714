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
    K_DT_VPAIR_WTA, K_WTA_VOLUME, K_AHAT, K_NKINDS
};
const char* const kKindNames[K_NKINDS] = {
    "window_stats", "dt_coef", "zncc_cost", "zncc_cost_hpair", "zncc_cost_wta",
    "dt_hpair", "dt_vpair", "dt_vpair_wta", "wta_volume", "ahat_pair"};

struct ProfRecord {
    int kind, ev0, ev1;
};

// Launch shape of one kind of line pass, chosen once per context and pass signature.
struct LinePlan {
    long long key;
    int tq, lpc, nch, async, per_block, blocks;
};

constexpr int kTargetBlocks = 1216;   // about eight blocks per SM on a 152-SM GB300

}  // namespace

struct zncc_ctx {
    int W = 0, H = 0, D = 0, win = 0, r = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cur = nullptr;       // the stream launches go to (stream, or side)
    cudaStream_t side = nullptr;      // second stream for work independent of the cost kernel
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::string err;
    float4* coefH = nullptr;      // [H][W]       horizontal DT coefficients
    float4* coefV = nullptr;      // [W][H]       vertical DT coefficients
    void* vol = nullptr;          // the fused path's intermediate volume (on first use)
    size_t vol_bytes = 0;
    float* bestv = nullptr;       // [H][W] running WTA best across launches (on first use)
    int* bestd = nullptr;         // [H][W]
    float* ahat = nullptr;        // [nahat][H][W] DT responses of an all-ones plane (F16 storage)
    int nahat = 0;
    int smem_max = 0;             // opt-in shared memory per block of the device
    int row_minb2 = 1;            // cost kernel: two-blocks-per-SM variant where it applies
    int row_spb = 0;              // cost kernel: slices per block (0 = automatic)
    int h_tq = 0, v_tq = 0;       // DT pairs: forced lanes per chunk (0 = automatic)
    int num_sms = 0;
    std::vector<LinePlan> plans;  // line-pass launch shapes, by pass signature
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
            cudaEventRecord((c)->events[ev0_], (c)->cur);                     \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what);                 \
        int ev1_ = ev0_ >= 0 ? prof_event(c) : -1;                            \
        if (ev1_ >= 0) {                                                      \
            cudaEventRecord((c)->events[ev1_], (c)->cur);                     \
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
    ZNCC_LAUNCH(c, K_COEF, launch_dt_coef(guide, pitch, c->W, c->H, K, inv, c->coefH, c->coefV, c->cur),
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
    a.minb2 = c->row_minb2;
    const int threads = a.nch * a.tq;
    const int ds = kG * a.tq;
    const int nslices = (c->D + ds - 1) / ds;
    if (mode != kModeWta) {
        a.d_lo = 0;
        a.d_hi = c->D;
        a.spb = c->row_spb > 0 ? std::min(c->row_spb, nslices) : slices_per_block(nslices, c->H);
        while (a.spb > 1 && zncc_row_smem_bytes(c->r, mode, a, threads) > (size_t)c->smem_max) --a.spb;
        if (zncc_row_smem_bytes(c->r, mode, a, threads) > (size_t)c->smem_max)
            return fail(c, ZNCC_EUNSUPPORTED, "image too wide for the cost kernel's shared memory");
        ZNCC_LAUNCH(c, kind, launch_zncc_row(c->r, a, mode, dtype, c->cur), what);
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
        ZNCC_LAUNCH(c, kind, launch_zncc_row(c->r, a, mode, dtype, c->cur), what);
    }
    return ZNCC_OK;
}

// One DT pass pair along rows (horiz) or columns of a [H][W][dstride] volume.
struct LinePass {
    void* vol = nullptr;           // output (and input unless src / ones)
    const void* src = nullptr;
    bool ones = false;
    long long dstride = 0;
    int dcount = 0;
    int dtype = 0;
    bool horiz = true;
    int mode = kLineStore;
    const float* ahat_in = nullptr;
    const float* ahat_out = nullptr;
    uint16_t* disp = nullptr;
    float s2 = 1.0f;
    int force_tq = 0;
    bool ahat = false;             // a pass of the A_hat chain (profiled separately)
};

// The launch shape: among lane counts per chunk (8, 4, 2, or the forced one) and lines per
// block that fit in shared memory, prefer whole 64-byte segments per chunk, then streaming
// through shared memory (async), then at least two resident blocks per SM, then the most
// resident warps. The grid is the resident blocks (persistent), each taking an equal run of
// items.
zncc_status plan_line_pass(zncc_ctx* c, LineArgs& a, const LinePass& p) {
    const long long key = ((((long long)p.horiz * 2 + p.mode) * 2 + p.dtype) * 2 + (a.vec ? 1 : 0)) * 16 +
                          p.force_tq + ((long long)p.dcount << 20) + ((long long)(p.horiz ? c->h_tq : c->v_tq) << 40);
    for (const LinePlan& pl : c->plans)
        if (pl.key == key) {
            a.tq = pl.tq; a.lpc = pl.lpc; a.nch = pl.nch; a.async = pl.async; a.per_block = pl.per_block;
            return ZNCC_OK;
        }
    LinePlan best{key, 0, 0, 0, 0, 0, 0};
    long long best_score = -1;
    const int tqs[4] = {8, 4, 2, 1};
    const int forced = p.force_tq ? p.force_tq : (p.horiz ? c->h_tq : c->v_tq);
    for (int ti = 0; ti < 4; ++ti) {
        const int tq = tqs[ti];
        if (forced ? tq != forced : tq == 1) continue;
        const int nch = padded_chunks(a.n, tq);
        const int per_line = nch * tq;
        if (per_line > 512) continue;
        // a chunk's lanes read tq * 4 contiguous entries per position: shapes whose segments
        // are whole 64-byte DRAM bursts come first
        const bool whole_bursts = tq * 4 * (p.dtype == 0 ? 4 : 2) >= 64;
        for (int async = a.vec ? 1 : 0; async >= 0; --async) {
            for (int lpc = std::max(1, std::min(8, 256 / per_line)); lpc >= 1; --lpc) {
                a.tq = tq; a.nch = nch; a.lpc = lpc; a.async = async;
                if (line_pair_smem_bytes(p.mode, p.dtype, a) > (size_t)c->smem_max) continue;
                int bps = 0;
                ZNCC_CUDA(c, line_pair_occupancy(a, p.mode, p.dtype, &bps), "occupancy query");
                if (bps < 1) continue;
                const long long warps = (long long)bps * lpc * per_line / 32;
                const long long score = (whole_bursts ? 10000000LL : 0) + async * 1000000LL +
                                        (bps >= 2 ? 100000LL : 0) + warps * 100 + tq;
                if (score > best_score) {
                    best_score = score;
                    best.tq = tq; best.lpc = lpc; best.nch = nch; best.async = async; best.blocks = bps;
                }
                break;                      // fewer lines per block only when this did not fit
            }
        }
    }
    if (best_score < 0) return fail(c, ZNCC_EUNSUPPORTED, "line too long for the DT kernel's shared memory");
    a.tq = best.tq; a.lpc = best.lpc; a.nch = best.nch; a.async = best.async;
    const int nslices = (p.dcount + kG * a.tq - 1) / (kG * a.tq);
    const int ngroups = (a.nlines + a.lpc - 1) / a.lpc;
    const int grid_max = std::max(1, c->num_sms * best.blocks);
    if (p.mode == kLineWta) {
        const int gpb = (ngroups + grid_max - 1) / grid_max;
        a.per_block = gpb * nslices;
    } else {
        const int total = ngroups * nslices;
        a.per_block = (total + grid_max - 1) / grid_max;
    }
    best.per_block = a.per_block;
    c->plans.push_back(best);
    return ZNCC_OK;
}

zncc_status run_line_pair(zncc_ctx* c, const LinePass& p) {
    LineArgs a;
    memset(&a, 0, sizeof(a));
    const int n = p.horiz ? c->W : c->H;
    a.vol = p.vol;
    a.src = p.src;
    a.src_ones = p.ones ? 1 : 0;
    a.elem_stride = p.horiz ? p.dstride : (long long)c->W * p.dstride;
    a.line_stride = p.horiz ? (long long)c->W * p.dstride : p.dstride;
    a.n = n;
    a.nlines = p.horiz ? c->H : c->W;
    a.dcount = p.dcount;
    a.d_base = 0;
    a.ahat_in = p.ahat_in;
    a.ahat_out = p.ahat_out;
    a.coef = p.horiz ? c->coefH : c->coefV;
    a.coef_line_stride = p.horiz ? c->W : c->H;
    a.s2 = p.s2;
    const void* in = p.src ? p.src : p.vol;
    a.vec = (p.dstride % 4 == 0) && ((uintptr_t)p.vol % (p.dtype == 0 ? 16 : 8) == 0) &&
                    ((uintptr_t)in % (p.dtype == 0 ? 16 : 8) == 0) ? 1 : 0;
    a.wta.disp = p.disp;
    a.wta.first = 1;
    a.wta.last = 1;
    a.pix_line = p.horiz ? c->W : 1;
    a.pix_pos = p.horiz ? 1 : c->W;
    ZNCC_TRY(plan_line_pass(c, a, p));
    const int kind = p.ahat ? K_AHAT
                     : (p.horiz ? K_DT_HPAIR : (p.mode == kLineWta ? K_DT_VPAIR_WTA : K_DT_VPAIR));
    ZNCC_LAUNCH(c, kind, launch_line_pair(a, p.mode, p.dtype, c->cur), p.horiz ? "DT horizontal pair" : "DT vertical pair");
    return ZNCC_OK;
}

// The scaled DT responses of an all-ones plane after pairs 1 .. n (A_hat, Eqs. (3)-(6) on a
// constant input), one [H][W] map each: the per-pixel bound of |aggregated cost|.
zncc_status run_ahat_chain(zncc_ctx* c, int n, float s2) {
    const size_t npix = (size_t)c->W * c->H;
    if (c->nahat < n) {
        free_dev_f(c->ahat);
        c->nahat = 0;
        cudaError_t e = cudaMalloc(&c->ahat, npix * n * sizeof(float));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, ZNCC_ENOMEM, std::string("A_hat maps: ") + cudaGetErrorString(e));
        }
        c->nahat = n;
    }
    for (int p = 1; p <= n; ++p) {
        LinePass lp;
        lp.vol = c->ahat + (size_t)(p - 1) * npix;
        lp.src = p == 1 ? nullptr : c->ahat + (size_t)(p - 2) * npix;
        lp.ones = p == 1;
        lp.dstride = 1;
        lp.dcount = 1;
        lp.dtype = 0;
        lp.horiz = (p % 2) == 1;
        lp.s2 = s2;
        lp.force_tq = 1;
        lp.ahat = true;
        ZNCC_TRY(run_line_pair(c, lp));
    }
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
    free_dev(c->ahat);
    c->nahat = 0;
    c->plans.clear();
    free_dev(c->img);
    free_dev(c->disp);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    c->side = nullptr;
    c->ev_fork = c->ev_join = nullptr;
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
    if (width > 3072 || height > 4096)
        return fail(nullptr, ZNCC_EUNSUPPORTED, "width must be <= 3072 and height <= 4096");
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
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
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
    c->cur = c->stream;
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
                                                nullptr, c->cur), "window statistics");
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
    LinePass lp;
    lp.vol = cost;
    lp.dstride = c->D;
    lp.dcount = c->D;
    lp.dtype = dtype;
    lp.s2 = s2;
    for (int it = 0; it < iters; ++it) {
        lp.horiz = true;
        ZNCC_TRY(run_line_pair(c, lp));
        lp.horiz = false;
        ZNCC_TRY(run_line_pair(c, lp));
    }
    return ZNCC_OK;
}

zncc_status wta_disparity(zncc_ctx* c, const void* cost, zncc_dtype dtype, uint16_t* disp) {
    if (!c) return ZNCC_EINVAL;
    c->err.clear();
    if (!cost || !disp) return fail(c, ZNCC_EINVAL, "cost or disp pointer is NULL");
    if (dtype != ZNCC_F32 && dtype != ZNCC_F16) return fail(c, ZNCC_EINVAL, "unknown dtype");
    ZNCC_LAUNCH(c, K_WTA_VOLUME, launch_wta_volume(cost, dtype, c->W, c->H, c->D, disp, c->cur), "WTA");
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
    if (dt == 1 && iters > 1) {
        // the A_hat maps of half storage depend only on the guide: computed on a second stream,
        // concurrently with the cost kernel, and joined before the first stored pair is read
        if (!c->side) {
            ZNCC_CUDA(c, cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking), "side stream");
            ZNCC_CUDA(c, cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming), "fork event");
            ZNCC_CUDA(c, cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming), "join event");
        }
        ZNCC_CUDA(c, cudaEventRecord(c->ev_fork, c->stream), "fork");
        ZNCC_CUDA(c, cudaStreamWaitEvent(c->side, c->ev_fork, 0), "fork");
        c->cur = c->side;
        const zncc_status st = run_ahat_chain(c, 2 * iters - 1, s2);
        c->cur = c->stream;
        ZNCC_TRY(st);
        ZNCC_CUDA(c, cudaEventRecord(c->ev_join, c->side), "join");
    }
    ZNCC_TRY(run_rows(c, left, right, pitch, kModeHPair, dt, c->vol, dstride, s2, nullptr, K_ZNCC_HPAIR,
                      "ZNCC + horizontal DT pair"));
    // Half storage keeps each stored pair p >= 2 divided by A_hat_p (the per-pixel bound of
    // |cost|), so that it stays inside the half range wherever the guide isolates a pixel;
    // the next pair multiplies it back. The factor is the same for every d of a pixel.
    const bool norm = dt == 1;
    const int npairs = 2 * iters;
    const size_t ahat_sz = npix;
    const bool fork = norm && npairs > 2;
    if (fork) ZNCC_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_join, 0), "join of the A_hat stream");
    (void)ahat_sz;
    LinePass lp;
    lp.vol = c->vol;
    lp.dstride = dstride;
    lp.dcount = c->D;
    lp.dtype = dt;
    lp.s2 = s2;
    for (int pair = 2; pair <= npairs; ++pair) {    // pair 1 is the cost kernel's
        lp.horiz = (pair % 2) == 1;
        lp.mode = pair == npairs ? kLineWta : kLineStore;
        lp.disp = pair == npairs ? disp : nullptr;
        lp.ahat_in = norm && pair - 1 >= 2 ? c->ahat + (size_t)(pair - 2) * ahat_sz : nullptr;
        lp.ahat_out = norm && pair < npairs ? c->ahat + (size_t)(pair - 1) * ahat_sz : nullptr;
        ZNCC_TRY(run_line_pair(c, lp));
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

zncc_status zncc_set_tuning(zncc_ctx* c, int key, int value) {
    if (!c) return ZNCC_EINVAL;
    c->err.clear();
    if (value < 0) return fail(c, ZNCC_EINVAL, "tuning values are >= 0");
    switch (key) {
        case ZNCC_TUNE_ROW_MINB2: c->row_minb2 = value ? 1 : 0; break;
        case ZNCC_TUNE_ROW_SPB: c->row_spb = value; break;
        case ZNCC_TUNE_H_TQ:
        case ZNCC_TUNE_V_TQ:
            if (value != 0 && value != 2 && value != 4 && value != 8)
                return fail(c, ZNCC_EINVAL, "lanes per chunk must be 0, 2, 4 or 8");
            (key == ZNCC_TUNE_H_TQ ? c->h_tq : c->v_tq) = value;
            break;
        default: return fail(c, ZNCC_EINVAL, "unknown tuning key");
    }
    c->plans.clear();
    return ZNCC_OK;
}

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
