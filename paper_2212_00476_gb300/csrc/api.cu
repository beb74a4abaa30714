// api.cu -- the C ABI of libzncc.so (declared in include/zncc.h): argument checks, the
// context's device scratch, and the launch sequence of each call.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "zncc.h"

using namespace zncc;

namespace {

std::atomic<uint64_t> g_launches{0};
// Error text of the last failed call without a context (zncc_create, dt_aggregate_noalloc)
// on this thread: a fixed buffer, so that recording an error allocates nothing.
thread_local char g_free_error[256];

void set_free_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_free_error, sizeof(g_free_error), fmt, ap);
    va_end(ap);
}

}  // namespace

// Every device allocation of the library goes through here. Host-side fault injection for
// tests: with the environment variable ZNCC_FAIL_DEVICE_ALLOC set to 1, each allocation
// reports cudaErrorMemoryAllocation without calling the driver (no GPU fault is involved).
cudaError_t zncc::device_alloc(void** p, size_t bytes) {
    const char* f = getenv("ZNCC_FAIL_DEVICE_ALLOC");
    if (f && f[0] == '1') {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

namespace {

// Kernel kinds for per-kernel timing (zncc_profile_*).
enum Kind {
    K_STATS = 0, K_COEF, K_ZNCC_RAW, K_ZNCC_HPAIR, K_ZNCC_WTA, K_DT_HPAIR, K_DT_VPAIR,
    K_DT_VPAIR_WTA, K_WTA_VOLUME, K_AHAT, K_WTA_FINISH, K_ZNCC_SCAN, K_PLANE, K_ZNCC_MMA, K_NKINDS
};
const char* const kKindNames[K_NKINDS] = {
    "window_stats", "dt_coef", "zncc_cost", "zncc_cost_hpair", "zncc_cost_wta",
    "dt_hpair", "dt_vpair", "dt_vpair_wta", "wta_volume", "ahat_pair", "wta_finish", "zncc_cost_scan",
    "zncc_plane", "zncc_cost_mma"};

struct ProfRecord {
    int kind, ev0, ev1;
};

// Launch shape of one kind of line pass, chosen once per context and pass signature.
struct LinePlan {
    long long key;
    int tq, lpc, nch, async, per_block, blocks, cs;
};


}  // namespace

// An occupancy answer (blocks or clusters per SM) for a kernel variant, block size and shared
// memory, kept by the context so that repeated runs make no occupancy query.
struct OccEntry {
    long long key[3];
    int value;
};

struct zncc_ctx {
    int W = 0, H = 0, D = 0, win = 0, r = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cur = nullptr;       // the stream launches go to
    cudaStream_t side = nullptr;      // (F16, I8) the A_hat chain beside the cost kernel
    cudaEvent_t ev_fork = nullptr;
    std::vector<cudaEvent_t> ev_pair; // [p-2]: the side work line pair p needs is done
    std::string err;
    float4* coefH = nullptr;      // [H][W]       horizontal DT coefficients
    float4* coefV = nullptr;      // [W][H]       vertical DT coefficients
    unsigned long long* keys = nullptr;   // [H][W] fused-WTA keys, zero between runs
    void* vol = nullptr;          // the fused path's intermediate volume (on first use)
    size_t vol_bytes = 0;
    float* ahat = nullptr;        // [nahat][H][W] DT responses of an all-ones plane (F16, I8 storage)
    float2* mulmap = nullptr;     // [nmul] maps of the pairs from 2 (F16) or 1 (I8) on:
    int nahat = 0, nmul = 0;      //        (A_hat_{p-1}, s2 / A_hat_p), line-major
    int smem_max = 0;             // opt-in shared memory per block of the device
    int row_minb2 = 0;            // cost kernel: two-blocks-per-SM variant where it applies
    int row_spb = 0;              // cost kernel: slices per block (0 = automatic)
    int row_nobulk = 0;           // cost kernel: stage the image rows with plain loads
    int line_loads = 0;           // DT pairs' staging: 0 TMA for rows, 1 cp.async only, 2 TMA for both
    int wait_drill = 0;           // (tests) DT pairs wait out an mbarrier nobody arrives on
    int ahat_sms = 0;             // SMs the cost kernel leaves to the A_hat chain (0 = automatic)
    int h_tq = 0, v_tq = 0;       // DT pairs: forced lanes per chunk (0 = automatic)
    int v_lpc = 0;                // vertical store pairs: most columns per block (0 = automatic)
    int ahat_join = 0;            // (F16) line pairs join the A_hat chain: 1 whole, 2 per pass, 0 automatic
    int plane_mode = 0;           // F32 fused runs: the plane-resident path where it applies
    int plane_force_cs = 0;       // its cluster size (0 = automatic)
    int plane_cs = -1;            // chosen cluster size (0: streaming path; -1: not chosen yet)
    int plane_cls = 0, plane_smem = 0, plane_clusters = 0;   // its size class, shared memory, clusters
    int num_sms = 0;
    std::vector<LinePlan> plans;  // line-pass launch shapes, by pass signature
    std::vector<OccEntry> occ;    // occupancy answers
    // encoded tensor maps of the DT pairs' inputs, by (volume, pixel stride, element size,
    // direction, box): a run then encodes none (the volume and strides repeat)
    struct TmapEntry {
        const void* base;
        long long dstride;
        int elem, horiz, ds, np;
        CUtensorMap map;
    };
    std::vector<TmapEntry> tmaps;
    int2* scan_stats = nullptr;   // (progressive scan) packed statistics: left [H][W], right [H][W+D-1]
    uint8_t* img = nullptr;       // device copies for zncc_run_host: 2 x [H][W]
    uint16_t* disp = nullptr;     // [H][W]
    unsigned* fault = nullptr;    // device word: faults the kernels recorded (kFault*), zero initially
    bool profiling = false;
    std::vector<cudaEvent_t> events;
    int events_used = 0;
    std::vector<ProfRecord> records;
    // zncc_run_host replayed as a CUDA graph: the arguments of the last call and of the captured
    // one, and the instantiated graph; gen counts changes of tuning and stream
    struct HostKey {
        const void *left, *right, *disp;            // host addresses
        const void *dleft, *dright, *ddisp;         // their device mappings (NULL: not page-locked)
        int pitch, iters, storage;
        float sigma_s, sigma_r;
        unsigned gen;
        bool operator==(const HostKey& o) const {
            return left == o.left && right == o.right && disp == o.disp && dleft == o.dleft &&
                   dright == o.dright && ddisp == o.ddisp && pitch == o.pitch && iters == o.iters &&
                   storage == o.storage && sigma_s == o.sigma_s && sigma_r == o.sigma_r && gen == o.gen;
        }
    };
    HostKey host_last{}, host_key{}, host_nocapture{};
    cudaGraphExec_t host_graph = nullptr;
    unsigned gen = 1;
};

namespace {

zncc_status fail(zncc_ctx* c, zncc_status s, const std::string& msg) {
    if (c) c->err = msg;
    else set_free_error("%s", msg.c_str());
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

// The context's cached occupancy answer for key, or query() (which fills *value) on a miss.
template <typename Query>
cudaError_t cached_occupancy(zncc_ctx* c, long long k0, long long k1, long long k2, Query query, int* value) {
    for (const OccEntry& o : c->occ)
        if (o.key[0] == k0 && o.key[1] == k1 && o.key[2] == k2) {
            *value = o.value;
            return cudaSuccess;
        }
    const cudaError_t e = query(value);
    if (e == cudaSuccess) c->occ.push_back(OccEntry{{k0, k1, k2}, *value});
    return e;
}

template <typename T>
void free_dev(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

void release(zncc_ctx* c) {
    free_dev(c->coefH);
    free_dev(c->coefV);
    free_dev(c->keys);
    free_dev(c->vol);
    c->vol_bytes = 0;
    free_dev(c->ahat);
    free_dev(c->mulmap);
    c->nahat = c->nmul = 0;
    free_dev(c->img);
    free_dev(c->disp);
    free_dev(c->scan_stats);
    free_dev(c->fault);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    for (cudaEvent_t e : c->ev_pair) cudaEventDestroy(e);
    c->ev_pair.clear();
    c->side = nullptr;
    c->ev_fork = nullptr;
    for (cudaEvent_t e : c->events) cudaEventDestroy(e);
    c->events.clear();
    c->records.clear();
    c->events_used = 0;
    c->plans.clear();
    if (c->host_graph) cudaGraphExecDestroy(c->host_graph);
    c->host_graph = nullptr;
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

// A pair whose volume alone fills the device: batching it with others only costs the batched
// kernels' per-pair argument indexing, so it gets launches of its own.
bool fills_device(const zncc_ctx* c) { return (long long)c->W * c->H * c->D >= (1LL << 25); }

float scale_s2(float sigma_s) {
    const double s = 1.0 - exp(-1.0 / (double)sigma_s);
    return (float)(s * s);
}

void free_dev_f(float*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

zncc_status alloc_dev(zncc_ctx* c, void** p, size_t bytes, const char* what) {
    ++c->gen;                                       // a captured host-buffer run refers to the old buffers
    c->tmaps.clear();                               // (a new buffer may reuse an old address)
    cudaError_t e = device_alloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(c, e == cudaErrorMemoryAllocation ? ZNCC_ENOMEM : ZNCC_ECUDA,
                    std::string(what) + ": " + cudaGetErrorString(e));
    }
    return ZNCC_OK;
}

// One pair of a (possibly batched) call: its context and this call's buffers. lc, the
// launching context, is the first pair's: its stream carries every launch, and errors and
// per-kernel timings are recorded on it.
struct PairIO {
    zncc_ctx* c;
    const uint8_t* left;
    const uint8_t* right;
    int pitch;
    uint16_t* disp;
    void* vol;              // the pair's cost volume [H][W][dstride]
    long long dstride;
    const float2* mulmap1 = nullptr;     // (FastDT) the multipliers of the cost kernel's pass pair
};

// DT coefficients of every pair (guide = left image), one launch.
zncc_status run_coef(zncc_ctx* lc, const PairIO* io, int n, float sigma_s, float sigma_r, bool rows = true) {
    CoefBatch b;
    memset(&b, 0, sizeof(b));
    b.npairs = n;
    const float K = (float)exp(-1.0 / (double)sigma_s);
    const float inv = (float)(1.0 / (255.0 * (double)sigma_r));
    long long t = 0;
    for (int i = 0; i < n; ++i) {
        CoefArgs& a = b.p[i];
        a.guide = io[i].left;
        a.pitch = io[i].pitch;
        a.W = io[i].c->W;
        a.H = io[i].c->H;
        a.K = K;
        a.inv_sr255 = inv;
        a.coefH = io[i].c->coefH;
        a.coefV = io[i].c->coefV;
        a.thread0 = t;
        t += rows ? dt_coef_threads(a.W, a.H) : dt_coef_col_blocks(a.W, a.H);
    }
    b.total_threads = t;
    if (rows) ZNCC_LAUNCH(lc, K_COEF, launch_dt_coef(b, lc->cur), "DT coefficients");
    else ZNCC_LAUNCH(lc, K_COEF, launch_dt_coef_cols(b, lc->cur), "DT column coefficients");
    return ZNCC_OK;
}

// Cost-kernel launches over the pairs (one per window radius among them). A block covers
// one row and a run of disparity slices (the band of a block spans its slices, so the run
// shrinks until the block fits in shared memory); in Wta mode a block covers every
// disparity of its row.
zncc_status run_rows(zncc_ctx* lc, const PairIO* io, int n, int mode, int dtype, float s2, float K,
                     float inv_sr255, int kind, int reserve_sms,
                     const char* what) {
    // pairs share a launch when they share the window radius and the block shape; a pair large
    // enough to fill the device by itself takes a launch of its own
    auto tq_of = [](int W) { return W <= 1024 ? 8 : (W <= 2048 ? 4 : 2); };
    bool done[kMaxBatch] = {false};
    for (int first = 0; first < n; ++first) {
        if (done[first]) continue;
        const int r = io[first].c->r;
        const int tq0 = tq_of(io[first].c->W), nch0 = padded_chunks(io[first].c->W, tq0);
        const bool alone = fills_device(io[first].c);
        RowBatch b;
        memset(&b, 0, sizeof(b));
        b.mode = mode;
        b.fault = lc->fault;
        int threads = 0;
        size_t smem = 0;
        bool minb2 = true;
        for (int i = first; i < n; ++i) {
            if (done[i] || io[i].c->r != r || tq_of(io[i].c->W) != tq0 || padded_chunks(io[i].c->W, tq0) != nch0 ||
                (i != first && (alone || fills_device(io[i].c))))
                continue;
            done[i] = true;
            zncc_ctx* c = io[i].c;
            RowArgs& a = b.p[b.npairs++];
            a.left = io[i].left;
            a.right = io[i].right;
            a.pitch = io[i].pitch;
            a.W = c->W;
            a.H = c->H;
            a.D = c->D;
            a.tq = tq0;
            a.nch = nch0;
            a.d_lo = 0;
            a.d_hi = c->D;
            a.vol = io[i].vol;
            a.dstride = io[i].dstride;
            a.d_out0 = 0;
            a.vec = io[i].vol && (io[i].dstride % 4 == 0) &&
                    ((uintptr_t)io[i].vol % (dtype == 0 ? 16 : (dtype == 1 ? 8 : 4)) == 0) ? 1 : 0;
            a.mulmap = io[i].mulmap1;
            a.K = K;
            a.inv_sr255 = inv_sr255;
            a.coefH_out = mode == kModeHPair ? c->coefH : nullptr;
            a.s2 = s2;
            a.minb2 = c->row_minb2;
            a.wta.disp = io[i].disp;
            a.wta.first = 1;
            a.wta.last = 1;
            const int nthr = a.nch * a.tq;
            const int nslices = (c->D + kG * a.tq - 1) / (kG * a.tq);
            // WTA keeps a row's running best in registers, FastDT codes each slice against the
            // row's d = 0: a block then visits whole rows
            const bool whole_rows = mode == kModeWta || dtype == 2;
            if (whole_rows) a.spb = nslices;
            else a.spb = c->row_spb > 0 ? std::min(c->row_spb, nslices) : nslices;
            // the image rows by bulk copies where both images and the pitch are 16-byte aligned
            // and W is a multiple of 16, while the rows fit in the region they share and the
            // guide row's buffer fits in shared memory; else plain loads
            a.bulk = mode == kModeHPair && a.W % 16 == 0 && a.pitch % 16 == 0 &&
                     (uintptr_t)a.left % 16 == 0 && (uintptr_t)a.right % 16 == 0 && !c->row_nobulk ? 1 : 0;
            while (!whole_rows && a.spb > 1 && zncc_row_smem_bytes(r, mode, dtype, a, nthr) > (size_t)lc->smem_max)
                --a.spb;
            if (a.bulk && (zncc_row_smem_bytes(r, mode, dtype, a, nthr) > (size_t)lc->smem_max ||
                           !zncc_row_bulk_fits_host(r, dtype, a, nthr)))
                a.bulk = 0;
            const size_t sm = zncc_row_smem_bytes(r, mode, dtype, a, nthr);
            if (sm > (size_t)lc->smem_max)
                return fail(lc, ZNCC_EUNSUPPORTED, "the cost kernel's row band does not fit in shared memory");
            a.item0 = b.total_items;
            a.nitems = whole_rows ? c->H : c->H * nslices;       // units: rows, or (row, slice)
            b.total_items += a.nitems;
            threads = std::max(threads, nthr);
            smem = std::max(smem, sm);
            minb2 = minb2 && a.minb2;
        }
        int bps = 0;
        const long long k0 = ((((long long)r * 4 + mode) * 4 + dtype) * 2 + (minb2 ? 1 : 0)) * 2 + (b.npairs == 1);
        ZNCC_CUDA(lc, cached_occupancy(lc, 1, k0 * 4096 + threads, (long long)smem, [&](int* v) {
                      return zncc_row_occupancy(r, mode, dtype, threads, smem, minb2, b.npairs == 1, v);
                  }, &bps), "occupancy query");
        b.grid = std::max(1, std::min(b.total_items, std::max(1, lc->num_sms - reserve_sms) * std::max(1, bps)));
        ZNCC_LAUNCH(lc, kind, launch_zncc_row(r, b, threads, smem, mode, dtype, lc->cur), what);
    }
    return ZNCC_OK;
}

// One DT pass pair along rows (horiz) or columns of a pair's [H][W][dstride] volume.
struct LinePass {
    void* vol = nullptr;           // output (and input unless src / ones)
    const void* src = nullptr;
    bool ones = false;
    long long dstride = 0;
    int dcount = 0;
    int dtype = 0;
    bool horiz = true;
    int mode = kLineStore;
    const float2* mulmap = nullptr;   // per-position (input multiplier, output scale), line-major
    unsigned long long* keys = nullptr;   // (Wta)
    float s2 = 1.0f;
    int force_tq = 0;
};

// The block shape of a pair's pass: among lane counts per chunk (8, 4, 2, or the forced
// one) and lines per block that fit in shared memory (at most 256 threads of lines, or
// max_lpc lines when that is set), prefer whole 64-byte segments per chunk, then streaming
// through shared memory (async), then at least two resident blocks per SM (unless max_lpc
// is set), then the most resident warps, then a line inside one block. Which of a cluster with
// 64-byte segments and one block with 32-byte segments is faster depends on the shape
// (half-precision rows of 1280 pixels: one block, 181 against 235 us per pair; of 1920
// pixels: the cluster, 839 against 954 us), so the autotuner settles it per shape.
// `found` is false when no shape fits; on success the shape is also left in a.
cudaError_t choose_line_plan(int smem_max, int forced, int max_lpc, LineArgs& a, const LinePass& p,
                             LinePlan& best, bool& found) {
    found = false;
    long long best_score = -1;
    const int tqs[4] = {8, 4, 2, 1};
    for (int ti = 0; ti < 4; ++ti) {
        const int tq = tqs[ti];
        if (forced ? tq != forced : tq == 1) continue;
        // chunks per CTA: the line in one block, or split over a cluster of 2 or 4 CTAs
        const int per_warp = 32 / tq, nch_line = padded_chunks(a.n, tq);
        int cs = 1, nch = nch_line;
        while (nch * tq > 512 && cs < 4) {
            cs *= 2;
            nch = ((nch_line + cs - 1) / cs + per_warp - 1) / per_warp * per_warp;
        }
        const int per_line = nch * tq;
        if (per_line > 512) continue;
        const int seg = tq * 4 * (p.dtype == 0 ? 4 : (p.dtype == 1 ? 2 : 1));   // bytes per chunk position
        const bool whole_bursts = seg >= 64;
        for (int async = a.vec ? 1 : 0; async >= 0; --async) {
            const int lpc0 = cs > 1 ? 1 : max_lpc > 0 ? std::max(1, std::min(max_lpc, 512 / per_line))
                                                      : std::max(1, std::min(8, 256 / per_line));
            for (int lpc = lpc0; lpc >= 1; --lpc) {
                a.tq = tq; a.nch = nch; a.lpc = lpc; a.async = async; a.cs = cs;
                const size_t smem = line_pair_smem_bytes(p.mode, p.dtype, a, line_coef_async(a));
                if (smem > (size_t)smem_max) continue;
                int bps = 0;
                cudaError_t e = line_pair_occupancy(p.mode, p.dtype, lpc * per_line, smem, true, cs > 1, &bps);
                if (e != cudaSuccess) return e;
                if (bps < 1) continue;
                if (cs > 1) {
                    int ncl = 0;
                    e = line_pair_max_clusters(p.mode, p.dtype, per_line, smem, true, cs, &ncl);
                    if (e != cudaSuccess) return e;
                    if (ncl < 1) continue;
                }
                const long long warps = (long long)bps * lpc * per_line / 32;
                const long long score = (whole_bursts ? 10000000LL : 0) + async * 1000000LL +
                                        (bps >= 2 && max_lpc == 0 ? 100000LL : 0) + warps * 100 +
                                        (cs == 1 ? 50 : 0) + tq;
                if (score > best_score) {
                    best_score = score;
                    best.tq = tq; best.lpc = lpc; best.nch = nch; best.async = async; best.blocks = bps;
                    best.cs = cs;
                }
                break;                      // fewer lines per block only when this did not fit
            }
        }
    }
    if (best_score < 0) return cudaSuccess;
    found = true;
    a.tq = best.tq; a.lpc = best.lpc; a.nch = best.nch; a.async = best.async; a.cs = best.cs;
    return cudaSuccess;
}

// Grid of a line-pair launch: the resident blocks (or clusters of cs CTAs), at most one per item.
// With a context the occupancy answer comes from its cache.
cudaError_t size_line_grid(LineBatch& b, int threads, size_t smem, int mode, int dtype, int num_sms,
                           zncc_ctx* c = nullptr) {
    const int cs = b.p[0].cs;
    const bool single = b.npairs == 1;
    auto query = [&](int* v) {
        return cs > 1 ? line_pair_max_clusters(mode, dtype, threads, smem, single, cs, v)
                      : line_pair_occupancy(mode, dtype, threads, smem, single, false, v);
    };
    int n = 0;
    const long long k0 = (((long long)mode * 4 + dtype) * 2 + (single ? 1 : 0)) * 8 + cs;
    const cudaError_t e = c ? cached_occupancy(c, 2, k0 * 4096 + threads, (long long)smem, query, &n) : query(&n);
    if (cs > 1) b.grid = cs * std::max(1, std::min(b.total_items, n));
    else b.grid = std::max(1, std::min(b.total_items, num_sms * std::max(1, n)));
    return e;
}

// The block shape of a pair's pass (choose_line_plan), chosen once per context and pass
// signature.
zncc_status plan_line_pass(zncc_ctx* c, LineArgs& a, const LinePass& p) {
    const int forced = p.force_tq ? p.force_tq : (p.horiz ? c->h_tq : c->v_tq);
    const int max_lpc = (!p.horiz && p.mode == kLineStore) ? c->v_lpc : 0;
    const long long key = ((((long long)p.horiz * 2 + p.mode) * 2 + p.dtype) * 2 + (a.vec ? 1 : 0)) * 16 +
                          forced + ((long long)p.dcount << 20) + ((long long)(p.mulmap ? 1 : 0) << 40) +
                          ((long long)max_lpc << 44);
    for (const LinePlan& pl : c->plans)
        if (pl.key == key) {
            a.tq = pl.tq; a.lpc = pl.lpc; a.nch = pl.nch; a.async = pl.async; a.cs = pl.cs;
            return ZNCC_OK;
        }
    LinePlan best{key, 0, 0, 0, 0, 0, 0, 1};
    bool found = false;
    ZNCC_CUDA(c, choose_line_plan(c->smem_max, forced, max_lpc, a, p, best, found), "occupancy query");
    if (!found) return fail(c, ZNCC_EUNSUPPORTED, "line too long for the DT kernel's shared memory");
    c->plans.push_back(best);
    return ZNCC_OK;
}

// The arguments of one pair's pass, before its block shape is chosen.
void fill_line_args(LineArgs& a, const LinePass& p, int W, int H, const float4* coefH, const float4* coefV) {
    memset(&a, 0, sizeof(a));
    a.vol = p.vol;
    a.src = p.src;
    a.src_ones = p.ones ? 1 : 0;
    a.elem_stride = p.horiz ? p.dstride : (long long)W * p.dstride;
    a.line_stride = p.horiz ? (long long)W * p.dstride : p.dstride;
    a.n = p.horiz ? W : H;
    a.nlines = p.horiz ? H : W;
    a.dcount = p.dcount;
    a.d_base = 0;
    a.mulmap = p.mulmap;
    a.coef = p.horiz ? coefH : coefV;
    a.coef_line_stride = p.horiz ? W : H;
    a.s2 = p.s2;
    const void* in = p.src ? p.src : p.vol;
    const size_t al = p.dtype == 0 ? 16 : (p.dtype == 1 ? 8 : 4);
    a.vec = (p.dstride % 4 == 0) && ((uintptr_t)p.vol % al == 0) && ((uintptr_t)in % al == 0) ? 1 : 0;
    a.keys = p.keys;
    a.pix_line = p.horiz ? W : 1;
    a.pix_pos = p.horiz ? 1 : W;
    a.cs = 1;
    a.horiz = p.horiz ? 1 : 0;
    a.tma = 0;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to the driver
// library), looked up once; NULL where the driver does not provide it.
using TmapEncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
TmapEncodeFn tmap_encoder() {
    static const TmapEncodeFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return (TmapEncodeFn) nullptr;
        }
        return reinterpret_cast<TmapEncodeFn>(p);
    }();
    return fn;
}

// Whether a planned pass streams its slices by TMA, with its tensor map in m: the input volume
// as {entries per pixel, W, H}, one box of kL + G - 1 positions per chunk and slice (G =
// line_tma_chunks_per_wavefront). Taken for F32 and F16 where G <= 4, the volume and the pixel
// stride are 16-byte aligned, a line stays in one CTA, and the larger slots keep the plan's
// blocks per SM within shared memory; for columns only when asked (ZNCC_TUNE_LINE_LOADS = 2):
// a column box is 16 + G - 1 rows of 64 or 128 bytes an image row of the volume apart, which
// the tensor copy fetches row by row (at 1920x1080, D = 256 the F32 V pair took 1419 us so,
// 1165 us with cp.async), while a row box reads consecutive pixels.
bool line_tma(zncc_ctx* c, const LineArgs& a, const LinePass& p, CUtensorMap& m) {
    if (c->line_loads == 1 || (c->line_loads == 0 && !p.horiz) || !a.async || a.cs != 1 || p.ones ||
        p.dtype == 2)
        return false;
    const long long elem = p.dtype == 0 ? 4 : 2;
    const int g = line_tma_chunks_per_wavefront(a.tq, (int)elem);
    if (g > 4) return false;
    LineArgs t = a;
    t.tma = 1;
    const size_t smem0 = line_pair_smem_bytes(p.mode, p.dtype, a, line_coef_async(a));
    const size_t smem1 = line_pair_smem_bytes(p.mode, p.dtype, t, line_coef_async(t));
    if (smem1 > (size_t)c->smem_max) return false;
    if (smem1 > smem0) {
        const int threads = a.lpc * a.nch * a.tq;
        auto occ = [&](size_t smem, int* v) {
            return cached_occupancy(c, 3, ((long long)p.mode * 4 + p.dtype) * 4096 + threads, (long long)smem,
                                    [&](int* r) { return line_pair_occupancy(p.mode, p.dtype, threads, smem, true,
                                                                             false, r); }, v);
        };
        int b0 = 0, b1 = 0;
        if (occ(smem0, &b0) != cudaSuccess || occ(smem1, &b1) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (b1 < b0) return false;
    }
    const void* in = p.src ? p.src : p.vol;
    if ((uintptr_t)in % 16 != 0 || (p.dstride * elem) % 16 != 0) return false;
    const cuuint32_t ds = (cuuint32_t)(kG * a.tq), np = (cuuint32_t)(kL + g - 1);
    for (const zncc_ctx::TmapEntry& t : c->tmaps)
        if (t.base == in && t.dstride == p.dstride && t.elem == (int)elem && t.horiz == (int)p.horiz &&
            t.ds == (int)ds && t.np == (int)np) {
            m = t.map;
            return true;
        }
    const TmapEncodeFn enc = tmap_encoder();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)p.dstride, (cuuint64_t)c->W, (cuuint64_t)c->H};
    const cuuint64_t strides[2] = {(cuuint64_t)(p.dstride * elem), (cuuint64_t)(p.dstride * elem * c->W)};
    const cuuint32_t box[3] = {ds, p.horiz ? np : 1u, p.horiz ? 1u : np};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    if (enc(&m, p.dtype == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3,
            const_cast<void*>(in), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    if (c->tmaps.size() >= 32) c->tmaps.clear();   // (callers' own volumes, e.g. dt_aggregate)
    c->tmaps.push_back(zncc_ctx::TmapEntry{in, p.dstride, (int)elem, (int)p.horiz, (int)ds, (int)np, m});
    return true;
}

// Appends a pair (its block shape chosen) to a launch: its items and steps, and the block's
// thread count and shared memory (staging region and the rest) grown to cover it.
void add_line_pair(LineBatch& b, const LineArgs& ai, int mode, int dtype, int& threads, size_t& stage,
                   size_t& rest) {
    b.co_async = (b.npairs == 0 || b.co_async) && line_coef_async(ai);
    LineArgs& a = b.p[b.npairs++];
    a = ai;
    const int nslices = (a.dcount + kG * a.tq - 1) / (kG * a.tq);
    const int ngroups = (a.nlines + a.lpc - 1) / a.lpc;
    a.step0 = b.total_steps;
    a.nsteps = ngroups * nslices;
    a.item0 = b.total_items;
    // FastDT stores code each slice against the line group's d = 0, which the group's first
    // slice computes: a block then takes whole line groups
    a.nitems = dtype == 2 && mode == kLineStore ? ngroups : a.nsteps;
    b.total_steps += a.nsteps;
    b.total_items += a.nitems;
    threads = std::max(threads, a.lpc * a.nch * a.tq);
    const size_t st = line_stage_bytes(dtype, a);
    stage = std::max(stage, st);
    rest = std::max(rest, line_pair_smem_bytes(mode, dtype, a, line_coef_async(a)) - st);
}

// Line-pair launches over the passes of several pairs (the same mode and storage): pairs
// whose passes have the same block shape share one launch.
zncc_status run_lines(zncc_ctx* lc, zncc_ctx* const* ctxs, const LinePass* passes, int n, int kind) {
    const int mode = passes[0].mode, dtype = passes[0].dtype;
    LineArgs args[kMaxBatch];
    CUtensorMap tmaps[kMaxBatch];
    for (int i = 0; i < n; ++i) {
        zncc_ctx* c = ctxs[i];
        const LinePass& p = passes[i];
        LineArgs& a = args[i];
        fill_line_args(a, p, c->W, c->H, c->coefH, c->coefV);
        if (plan_line_pass(c, a, p) != ZNCC_OK) return fail(lc, ZNCC_EUNSUPPORTED, c->err);
        a.tma = line_tma(c, a, p, tmaps[i]) ? 1 : 0;
    }
    bool done[kMaxBatch] = {false};
    for (int first = 0; first < n; ++first) {
        if (done[first]) continue;
        const LineArgs& a0 = args[first];
        const bool alone = fills_device(ctxs[first]);
        LineBatch b;
        memset(&b, 0, sizeof(b));
        int threads = 0;
        size_t stage = 0, rest = 0;
        for (int i = first; i < n; ++i) {
            const LineArgs& ai = args[i];
            if (done[i] || ai.tq != a0.tq || ai.nch != a0.nch || ai.lpc != a0.lpc || ai.async != a0.async ||
                ai.cs != a0.cs || ai.tma != a0.tma || (i != first && (alone || fills_device(ctxs[i]))))
                continue;
            done[i] = true;
            add_line_pair(b, ai, mode, dtype, threads, stage, rest);
            if (ai.tma) b.tmap[b.npairs - 1] = tmaps[i];
        }
        b.stage_bytes = (long long)stage;
        b.fault = lc->fault;
        b.drill = lc->wait_drill;
        const size_t smem = stage + rest;
        if (smem > (size_t)lc->smem_max) return fail(lc, ZNCC_EUNSUPPORTED, "DT pass exceeds shared memory");
        ZNCC_CUDA(lc, size_line_grid(b, threads, smem, mode, dtype, lc->num_sms, lc), "occupancy query");
        ZNCC_LAUNCH(lc, kind, launch_line_batch(b, threads, smem, mode, dtype, lc->cur), "DT pass pair");
    }
    return ZNCC_OK;
}

zncc_status ensure_volume(zncc_ctx* c, int dtype, long long dstride) {
    const size_t need = (size_t)c->W * c->H * (size_t)dstride * (dtype == 0 ? 4 : (dtype == 1 ? 2 : 1));
    if (c->vol_bytes >= need) return ZNCC_OK;
    free_dev(c->vol);
    c->vol_bytes = 0;
    ZNCC_TRY(alloc_dev(c, &c->vol, need, "cost volume"));
    c->vol_bytes = need;
    return ZNCC_OK;
}

zncc_status ensure_ahat(zncc_ctx* c, int nahat, int nmul) {
    if (c->nahat >= nahat && c->nmul >= nmul) return ZNCC_OK;
    free_dev_f(c->ahat);
    free_dev(c->mulmap);
    c->nahat = c->nmul = 0;
    ZNCC_TRY(alloc_dev(c, (void**)&c->ahat, (size_t)c->W * c->H * nahat * sizeof(float), "A_hat maps"));
    ZNCC_TRY(alloc_dev(c, (void**)&c->mulmap, (size_t)c->W * c->H * nmul * sizeof(float2), "A_hat multipliers"));
    c->nahat = nahat;
    c->nmul = nmul;
    return ZNCC_OK;
}

// SMs the cost kernel leaves to the A_hat chain by default (F16 step 0.662 -> 0.629 ms at
// 1280x384x128 with 8; 16 to 32 gave the same).
constexpr int kAhatSideSms = 8;

// Pass pair p of the A_hat chain (A_hat_p from A_hat_{p-1}, or from ones for p = 1) for every
// pair of the batch, one launch, with the multipliers of pair p when it has a map (p >= pfirst).
zncc_status run_ahat(zncc_ctx* lc, const PairIO* io, int n, int p, int pfirst, int npairs, float K,
                     float inv_sr255, float s2, bool fast) {
    AhatBatch b;
    memset(&b, 0, sizeof(b));
    b.npairs = n;
    b.horiz = (p % 2) == 1;
    b.K = K;
    b.inv_sr255 = inv_sr255;
    b.s2 = s2;
    // FastDT passes read -E (times A_hat / T) and write values scaled by T, ready to round
    b.xscale = fast ? 1.0f / kFastT : 1.0f;
    b.yscale = fast ? s2 * kFastT : s2;
    for (int i = 0; i < n; ++i) {
        zncc_ctx* c = io[i].c;
        const size_t npix = (size_t)c->W * c->H;
        AhatArgs& a = b.p[i];
        a.guide = io[i].left;
        a.pitch = io[i].pitch;
        a.W = c->W;
        a.H = c->H;
        a.ain = p == 1 ? nullptr : c->ahat + (size_t)(p - 2) * npix;
        a.aout = c->ahat + (size_t)(p - 1) * npix;
        a.mulmap = p >= pfirst && p <= npairs ? c->mulmap + (size_t)(p - pfirst) * npix : nullptr;
        a.in_mul = p - 1 >= pfirst ? 1 : 0;
        a.line0 = b.total_lines;
        b.total_lines += b.horiz ? c->H : c->W;
        b.nmax = std::max(b.nmax, b.horiz ? c->W : c->H);
    }
    ZNCC_LAUNCH(lc, K_AHAT, launch_ahat_pair(b, lc->cur), "A_hat pass pair");
    return ZNCC_OK;
}

// The fused path over n pairs that share the DT parameters and the storage type: the
// coefficients, the cost kernel with the first horizontal pair, the remaining pairs, and
// WTA in the last vertical pair; every step is one launch for all pairs (one per window
// radius for the cost kernel).
// The cluster size of the plane-resident path for a context's shape, or 0 where the pair
// takes the streaming path: the row length fits the lanes of a warp (W <= 1024) and a band of
// at most kPlaneBandMax rows per CTA with its image rows fits in shared memory; with it the
// kernel's size class (plane_class). Among the sizes that fit, the one with the least modelled
// time: waves of planes (D over the resident clusters) times the rows per CTA plus a fixed cost
// per plane (barriers, the cost rows' start).
int plane_choice(zncc_ctx* c) {
    if (c->plane_cs >= 0) return c->plane_cs;
    c->plane_cs = 0;
    if (!c->plane_mode || c->W > kPlaneMaxW || c->W + 2 * c->r > kPlaneThreads * kPlaneColsPerThread) return 0;
    double best = 0.0;
    for (int cs = 1; cs <= 8; cs *= 2) {
        if (c->plane_force_cs && cs != c->plane_force_cs) continue;
        const PlaneLayout L = plane_layout(c->W, c->H, c->r, cs);
        const int cls = plane_class(c->W, L.hb);
        if (cls < 0 || (long long)L.total > (long long)c->smem_max) continue;
        int clusters = 0;
        if (plane_max_clusters(cls, cs, L.total, &clusters) != cudaSuccess || clusters < 1) {
            cudaGetLastError();
            continue;
        }
        const double t = (double)((c->D + clusters - 1) / clusters) * (L.hb + 8);
        if (c->plane_cs == 0 || t < best) {
            best = t;
            c->plane_cs = cs;
            c->plane_cls = cls;
            c->plane_smem = (int)L.total;
            c->plane_clusters = clusters;
        }
    }
    return c->plane_cs;
}

// The plane-resident path for F32 runs of the pairs whose shape allows it: the window
// statistics of both images, one launch per cluster size among the pairs, the WTA finish.
zncc_status run_plane(zncc_ctx* lc, const PairIO* io, int n, float sigma_s, float sigma_r, int iters) {
    for (int i = 0; i < n; ++i) {
        zncc_ctx* c = io[i].c;
        const size_t nl = (size_t)c->W * c->H, nr = (size_t)(c->W + c->D - 1) * c->H;
        if (!c->scan_stats && alloc_dev(c, (void**)&c->scan_stats, (nl + nr) * sizeof(int2), "window statistics") != ZNCC_OK)
            return fail(lc, ZNCC_ENOMEM, c->err);
        ZNCC_LAUNCH(lc, K_STATS, launch_window_stats(io[i].left, io[i].pitch, c->W, c->H, c->r, 0, c->W, nullptr,
                                                     nullptr, nullptr, c->scan_stats, lc->cur),
                    "window statistics (left)");
        ZNCC_LAUNCH(lc, K_STATS, launch_window_stats(io[i].right, io[i].pitch, c->W, c->H, c->r, -(c->D - 1),
                                                     c->W + c->D - 1, nullptr, nullptr, nullptr,
                                                     c->scan_stats + nl, lc->cur),
                    "window statistics (right)");
    }
    for (int group = 0; group < 4 * kPlaneClasses; ++group) {      // one launch per (cluster size, class)
        const int cs = 1 << (group / kPlaneClasses), cls = group % kPlaneClasses;
        PlaneBatch b;
        memset(&b, 0, sizeof(b));
        size_t smem = 0;
        for (int i = 0; i < n; ++i) {
            zncc_ctx* c = io[i].c;
            if (c->plane_cs != cs || c->plane_cls != cls) continue;
            PlaneArgs& a = b.p[b.npairs++];
            a.left = io[i].left;
            a.right = io[i].right;
            a.pitch = io[i].pitch;
            a.W = c->W;
            a.H = c->H;
            a.D = c->D;
            a.r = c->r;
            a.statsL = c->scan_stats;
            a.statsR = c->scan_stats + (size_t)c->W * c->H;
            a.keys = c->keys;
            a.item0 = b.total_items;
            b.total_items += c->D;
            smem = std::max(smem, (size_t)c->plane_smem);
        }
        if (b.npairs == 0) continue;
        int clusters = 0;
        ZNCC_CUDA(lc, plane_max_clusters(cls, cs, smem, &clusters), "plane-resident path occupancy");
        if (clusters < 1) return fail(lc, ZNCC_EUNSUPPORTED, "plane-resident path: no cluster fits on the device");
        b.nclusters = std::min(clusters, b.total_items);
        b.cs = cs;
        b.iters = iters;
        b.K = (float)exp(-1.0 / (double)sigma_s);
        b.inv_sr255 = (float)(1.0 / (255.0 * (double)sigma_r));
        b.s2 = scale_s2(sigma_s);
        ZNCC_LAUNCH(lc, K_PLANE, launch_plane(b, cls, smem, lc->cur), "plane-resident ZNCC + DT + WTA");
    }
    WtaFinishBatch fb;
    memset(&fb, 0, sizeof(fb));
    fb.npairs = n;
    for (int i = 0; i < n; ++i) {
        fb.p[i].keys = io[i].c->keys;
        fb.p[i].disp = io[i].disp;
        fb.p[i].npix = (long long)io[i].c->W * io[i].c->H;
        fb.p[i].thread0 = fb.total_threads;
        fb.total_threads += fb.p[i].npix;
    }
    ZNCC_LAUNCH(lc, K_WTA_FINISH, launch_wta_finish(fb, lc->cur), "WTA finish");
    return ZNCC_OK;
}

zncc_status run_fused(zncc_ctx* lc, PairIO* io, int n, float sigma_s, float sigma_r, int iters,
                      int storage) {
    if (iters == 0) return run_rows(lc, io, n, kModeWta, 0, 0.0f, 0.0f, 0.0f, K_ZNCC_WTA, 0, "ZNCC + WTA");
    if (storage == ZNCC_F32) {      // pairs whose planes fit on chip take the plane-resident path
        PairIO plane[kMaxBatch];
        int np = 0, ns = 0;
        for (int i = 0; i < n; ++i) {
            if (plane_choice(io[i].c) > 0) plane[np++] = io[i];
            else io[ns++] = io[i];
        }
        if (np) ZNCC_TRY(run_plane(lc, plane, np, sigma_s, sigma_r, iters));
        if (ns == 0) return ZNCC_OK;
        n = ns;
    }
    const int dt = storage;                         // 0 float, 1 half, 2 FastDT codes
    zncc_ctx* ctxs[kMaxBatch];
    for (int i = 0; i < n; ++i) {
        ctxs[i] = io[i].c;
        io[i].dstride = (io[i].c->D + 3) / 4 * 4;     // padded so that every access is vectorised
        if (ensure_volume(io[i].c, dt, io[i].dstride) != ZNCC_OK) return fail(lc, ZNCC_ENOMEM, io[i].c->err);
        io[i].vol = io[i].c->vol;
    }
    const float K = (float)exp(-1.0 / (double)sigma_s);
    const float inv_sr255 = (float)(1.0 / (255.0 * (double)sigma_r));
    const int npairs = 2 * iters;
    // The scaled form multiplies every pass pair's output by s2 = (1-K)^2 so that |cost| <= 1.
    // With F32 storage only the disparity map leaves the fused path, and a positive constant
    // factor changes no argmax, so the passes run the literal chain (s2 = 1, no multiply) while
    // its values stay far inside the float range: |value| <= (1/(1-K))^(4 iters) <= 1e30.
    const bool literal = dt == 0 && 4.0 * iters * -log(1.0 - (double)K) <= log(1e30);
    const float s2 = literal ? 1.0f : scale_s2(sigma_s);
    // The DT weights of the line pairs (and the A_hat maps) depend only on the guide; they are
    // computed first, on the same stream: the persistent cost kernel fills every SM, so work
    // on a second stream would only run after it anyway. The cost kernel computes the
    // coefficients of its own rows and stores them for the later horizontal pairs, so the
    // coefficient kernel computes the columns' only.
    // Half storage keeps each stored pair p >= 2 divided by A_hat_p (the per-pixel bound of
    // |cost|), so that it stays inside the half range wherever the guide isolates a pixel;
    // the next pair multiplies it back. The factor is the same for every d of a pixel.
    // FastDT codes (Sec. IV-C) are normalised that way from the cost kernel's pair on.
    const bool norm = (dt == 1 && npairs > 2) || dt == 2;
    const int pfirst = dt == 2 ? 1 : 2;             // the first pair with a multiplier map
    if (norm)
        for (int i = 0; i < n; ++i)
            if (ensure_ahat(io[i].c, npairs - 1, npairs - pfirst + 1) != ZNCC_OK)
                return fail(lc, ZNCC_ENOMEM, io[i].c->err);
    // Side work beside the cost kernel, on a second stream: the column DT coefficients (the
    // cost kernel writes the rows') and, with F16 or I8 storage, the A_hat chain (small and
    // latency-bound, one warp per line). With F16 storage line pair p may wait for the side
    // work it reads and no more: the coefficients and the A_hat passes up to p (pass p writes
    // pair p's multipliers; the last pair's come from a separate kernel), so the later passes
    // run beside the first line pairs instead of before them. That pays where a pass's block
    // fits beside the line pairs' blocks (1280x384x128, 3 iterations: step 0.549 -> 0.535 ms)
    // and costs where it does not (1920x1080x256: 5.73 -> 6.10 ms, the passes waiting for
    // free SMs), so it is taken where the pass needs at most 64 KB of shared memory, or as
    // ZNCC_TUNE_AHAT_JOIN says. FastDT's pairs measured slower that way (1.21 -> 1.23 ms), so
    // there pair 2 waits for the whole side stream, as without multipliers. The cost kernel's
    // 128-register variant holds one block per SM and leaves registers and shared memory for
    // the side kernels' blocks on every SM; its two-blocks-per-SM variant fills the registers,
    // so with the A_hat chain `reserve` SMs are left to it. FastDT needs A_hat_1 in the cost
    // kernel itself, so that pass comes first, on the main stream.
    const int reserve = norm && lc->row_minb2 ? (lc->ahat_sms > 0 ? lc->ahat_sms : kAhatSideSms) : 0;
    int p_first_side = 1;
    if (dt == 2) {
        ZNCC_TRY(run_ahat(lc, io, n, 1, pfirst, npairs, K, inv_sr255, s2, true));
        p_first_side = 2;
    }
    {
        if (!lc->side) {
            ZNCC_CUDA(lc, cudaStreamCreateWithFlags(&lc->side, cudaStreamNonBlocking), "side stream");
            ZNCC_CUDA(lc, cudaEventCreateWithFlags(&lc->ev_fork, cudaEventDisableTiming), "fork event");
        }
        while ((int)lc->ev_pair.size() < npairs - 1) {
            cudaEvent_t e = nullptr;
            ZNCC_CUDA(lc, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "join event");
            lc->ev_pair.push_back(e);
        }
        ZNCC_CUDA(lc, cudaEventRecord(lc->ev_fork, lc->stream), "fork");
        ZNCC_CUDA(lc, cudaStreamWaitEvent(lc->side, lc->ev_fork, 0), "fork");
        lc->cur = lc->side;
    }
    // mark(q) records, after the side stream's last launch, the events of pairs pj..q (the
    // pairs that need nothing later); pj ends as the first pair with no event of its own
    int pj = 2;
    auto mark = [&](int upto) -> zncc_status {
        for (; pj <= upto; ++pj) {
            const cudaError_t e = cudaEventRecord(lc->ev_pair[pj - 2], lc->side);
            if (e != cudaSuccess) return cuda_fail(lc, e, "join");
        }
        return ZNCC_OK;
    };
    int longest = 0;
    for (int i = 0; i < n; ++i) longest = std::max(longest, std::max(io[i].c->W, io[i].c->H));
    const bool per_pair = norm && dt == 1 &&
                          (lc->ahat_join == 2 || (lc->ahat_join == 0 && ahat_pass_smem_bytes(longest) <= 65536));
    zncc_status st = run_coef(lc, io, n, sigma_s, sigma_r, false);
    if (st == ZNCC_OK && !norm) st = mark(2);       // later pairs follow pair 2 on the main stream
    for (int p = p_first_side; norm && p <= npairs - 1 && st == ZNCC_OK; ++p) {
        st = run_ahat(lc, io, n, p, pfirst, npairs, K, inv_sr255, s2, dt == 2);
        if (st == ZNCC_OK && per_pair) st = mark(p);
    }
    // the last pair's multipliers (A_hat_{npairs-1}, s2): its result is not stored
    for (int i = 0; norm && i < n && st == ZNCC_OK; ++i) {
        const int W = io[i].c->W, H = io[i].c->H;
        const size_t npix = (size_t)W * H;
        const float* ain = npairs - 1 >= pfirst ? io[i].c->ahat + (size_t)(npairs - 2) * npix : nullptr;
        g_launches.fetch_add(1, std::memory_order_relaxed);
        const cudaError_t e = launch_mulmap(ain, dt == 2 ? 1.0f / kFastT : 1.0f, s2, W, H, (npairs % 2) == 1,
                                            io[i].c->mulmap + (size_t)(npairs - pfirst) * npix, lc->cur);
        if (e != cudaSuccess) st = cuda_fail(lc, e, "A_hat multipliers");
    }
    if (st == ZNCC_OK && norm) st = mark(per_pair ? npairs : 2);
    lc->cur = lc->stream;
    ZNCC_TRY(st);
    if (dt == 2)
        for (int i = 0; i < n; ++i) io[i].mulmap1 = io[i].c->mulmap;
    ZNCC_TRY(run_rows(lc, io, n, kModeHPair, dt, s2, K, inv_sr255, K_ZNCC_HPAIR, reserve,
                      "ZNCC + horizontal DT pair"));
    for (int pair = 2; pair <= npairs; ++pair) {    // pair 1 is the cost kernel's
        // every recorded event is waited on, so that a captured graph joins the side stream
        if (pair < pj)
            ZNCC_CUDA(lc, cudaStreamWaitEvent(lc->stream, lc->ev_pair[pair - 2], 0), "join of the side stream");
        LinePass lp[kMaxBatch];
        for (int i = 0; i < n; ++i) {
            const size_t npix = (size_t)io[i].c->W * io[i].c->H;
            lp[i].vol = io[i].vol;
            lp[i].dstride = io[i].dstride;
            lp[i].dcount = io[i].c->D;
            lp[i].dtype = dt;
            lp[i].s2 = s2;
            lp[i].horiz = (pair % 2) == 1;
            lp[i].mode = pair == npairs ? kLineWta : kLineStore;
            lp[i].keys = pair == npairs ? io[i].c->keys : nullptr;
            lp[i].mulmap = norm ? io[i].c->mulmap + (size_t)(pair - pfirst) * npix : nullptr;
        }
        const int kind = pair % 2 ? K_DT_HPAIR : (pair == npairs ? K_DT_VPAIR_WTA : K_DT_VPAIR);
        ZNCC_TRY(run_lines(lc, ctxs, lp, n, kind));
    }
    WtaFinishBatch fb;                              // keys -> disparities, keys zeroed
    memset(&fb, 0, sizeof(fb));
    fb.npairs = n;
    for (int i = 0; i < n; ++i) {
        fb.p[i].keys = io[i].c->keys;
        fb.p[i].disp = io[i].disp;
        fb.p[i].npix = (long long)io[i].c->W * io[i].c->H;
        fb.p[i].thread0 = fb.total_threads;
        fb.total_threads += fb.p[i].npix;
    }
    ZNCC_LAUNCH(lc, K_WTA_FINISH, launch_wta_finish(fb, lc->cur), "WTA finish");
    return ZNCC_OK;
}

// ---- dt_aggregate_noalloc: per-device state of the static scratch --------------------
// Everything here has static storage: the device limits, read once per device, and a
// fixed-capacity cache of line-pass shapes. A mutex guards both. The scratch's address is
// not kept: it is looked up on every call, because it belongs to the device context that
// loaded the module and changes when that context is torn down and created again (after a
// cudaDeviceReset, say), where a kept address would point at memory that no longer exists.
constexpr int kNoallocDevices = 64;
constexpr int kNoallocPlans = 16;

struct NoallocPlan {
    bool used;
    int n, dcount, horiz, dtype, vec;
    LinePlan plan;
};

struct NoallocDevice {
    bool ready;
    int smem_max, num_sms;
    NoallocPlan plans[kNoallocPlans];
    int next;                       // the cache slot replaced next when it is full
};

std::mutex g_noalloc_mu;
NoallocDevice g_noalloc[kNoallocDevices];

zncc_status noalloc_cuda_fail(cudaError_t e, const char* what) {
    set_free_error("dt_aggregate_noalloc: %s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    return ZNCC_ECUDA;
}

// The device's state, set up on its first use, and the scratch's address in the current
// context of the current device (the caller holds g_noalloc_mu). cudaGetSymbolAddress is a
// host-side lookup; it allocates nothing once the module is loaded in the context.
zncc_status noalloc_device(int dev, NoallocDevice** out, unsigned char** scratch) {
    NoallocDevice& d = g_noalloc[dev];
    if (!d.ready) {
        cudaError_t e = cudaDeviceGetAttribute(&d.smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return noalloc_cuda_fail(e, "device attributes");
        d.ready = true;
    }
    void* p = nullptr;
    const cudaError_t e = noalloc_scratch_address(&p);
    if (e != cudaSuccess) return noalloc_cuda_fail(e, "scratch address (cudaGetSymbolAddress)");
    *scratch = static_cast<unsigned char*>(p);
    *out = &d;
    return ZNCC_OK;
}

// The block shape of a pass (choose_line_plan), from the device's cache (the caller holds
// g_noalloc_mu).
zncc_status noalloc_plan(NoallocDevice& d, LineArgs& a, const LinePass& p) {
    for (const NoallocPlan& c : d.plans)
        if (c.used && c.n == a.n && c.dcount == p.dcount && c.horiz == (int)p.horiz && c.dtype == p.dtype &&
            c.vec == a.vec) {
            a.tq = c.plan.tq; a.lpc = c.plan.lpc; a.nch = c.plan.nch; a.async = c.plan.async; a.cs = c.plan.cs;
            return ZNCC_OK;
        }
    LinePlan best{0, 0, 0, 0, 0, 0, 0, 1};
    bool found = false;
    cudaError_t e = choose_line_plan(d.smem_max, 0, 0, a, p, best, found);
    if (e != cudaSuccess) return noalloc_cuda_fail(e, "occupancy query");
    if (!found) {
        set_free_error("dt_aggregate_noalloc: a line of %d pixels does not fit the DT kernel's shared memory", a.n);
        return ZNCC_EUNSUPPORTED;
    }
    NoallocPlan& slot = d.plans[d.next];
    d.next = (d.next + 1) % kNoallocPlans;
    slot = NoallocPlan{true, a.n, p.dcount, (int)p.horiz, p.dtype, a.vec, best};
    return ZNCC_OK;
}

}  // namespace

extern "C" {

zncc_status zncc_create(int width, int height, int max_disp, int win, zncc_ctx** out) {
    g_free_error[0] = '\0';
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
    forget_smem_attributes();
    c->W = width;
    c->H = height;
    c->D = max_disp;
    c->win = win;
    c->r = win / 2;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    const size_t npix = (size_t)width * height;
    if (e == cudaSuccess) e = device_alloc((void**)&c->coefH, npix * sizeof(float4));
    if (e == cudaSuccess) e = device_alloc((void**)&c->coefV, npix * sizeof(float4));
    if (e == cudaSuccess) e = device_alloc((void**)&c->keys, npix * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(c->keys, 0, npix * sizeof(unsigned long long));
    if (e == cudaSuccess) e = device_alloc((void**)&c->fault, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(c->fault, 0, sizeof(unsigned));
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
    ++c->gen;
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
    PairIO io{c, left, right, pitch, nullptr, cost, c->D};
    return run_rows(c, &io, 1, kModeRaw, dtype, 0.0f, 0.0f, 0.0f, K_ZNCC_RAW, 0, "ZNCC cost");
}

}  // extern "C"

namespace {
// The cost-volume ablations (progressive scan, tensor-core banded product): the window
// statistics of both images (left centres x, right centres x - d for d < D), then the kernel.
zncc_status cost_volume_variant(zncc_ctx* c, const uint8_t* left, const uint8_t* right, int pitch, void* cost,
                                zncc_dtype dtype, bool mma) {
    if (!c) return ZNCC_EINVAL;
    c->err.clear();
    ZNCC_TRY(check_images(c, left, right, pitch));
    if (!cost) return fail(c, ZNCC_EINVAL, "cost pointer is NULL");
    if (dtype != ZNCC_F32 && dtype != ZNCC_F16) return fail(c, ZNCC_EINVAL, "unknown dtype");
    const size_t nl = (size_t)c->W * c->H, nr = (size_t)(c->W + c->D - 1) * c->H;
    if (!c->scan_stats) ZNCC_TRY(alloc_dev(c, (void**)&c->scan_stats, (nl + nr) * sizeof(int2), "scan statistics"));
    int2* pl = c->scan_stats;
    int2* pr = c->scan_stats + nl;
    ZNCC_LAUNCH(c, K_STATS, launch_window_stats(left, pitch, c->W, c->H, c->r, 0, c->W, nullptr, nullptr, nullptr,
                                                pl, c->cur), "window statistics (left)");
    ZNCC_LAUNCH(c, K_STATS, launch_window_stats(right, pitch, c->W, c->H, c->r, -(c->D - 1), c->W + c->D - 1,
                                                nullptr, nullptr, nullptr, pr, c->cur), "window statistics (right)");
    ScanArgs a;
    a.left = left;
    a.right = right;
    a.pitch = pitch;
    a.W = c->W;
    a.H = c->H;
    a.D = c->D;
    a.packL = pl;
    a.packR = pr;
    a.vol = cost;
    if (mma) ZNCC_LAUNCH(c, K_ZNCC_MMA, launch_zncc_mma(c->r, a, dtype, c->cur), "tensor-core ZNCC");
    else ZNCC_LAUNCH(c, K_ZNCC_SCAN, launch_zncc_scan(c->r, a, dtype, c->cur), "progressive-scan ZNCC");
    return ZNCC_OK;
}
}  // namespace

extern "C" {

zncc_status zncc_cost_volume_scan(zncc_ctx* c, const uint8_t* left, const uint8_t* right, int pitch,
                                  void* cost, zncc_dtype dtype) {
    return cost_volume_variant(c, left, right, pitch, cost, dtype, false);
}

zncc_status zncc_cost_volume_mma(zncc_ctx* c, const uint8_t* left, const uint8_t* right, int pitch,
                                 void* cost, zncc_dtype dtype) {
    return cost_volume_variant(c, left, right, pitch, cost, dtype, true);
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
    PairIO io{c, guide, guide, pitch, nullptr, cost, c->D};
    ZNCC_TRY(run_coef(c, &io, 1, sigma_s, sigma_r));
    LinePass lp;
    lp.vol = cost;
    lp.dstride = c->D;
    lp.dcount = c->D;
    lp.dtype = dtype;
    lp.s2 = scale_s2(sigma_s);
    for (int it = 0; it < iters; ++it) {
        lp.horiz = true;
        ZNCC_TRY(run_lines(c, &c, &lp, 1, K_DT_HPAIR));
        lp.horiz = false;
        ZNCC_TRY(run_lines(c, &c, &lp, 1, K_DT_VPAIR));
    }
    return ZNCC_OK;
}

zncc_status dt_aggregate_noalloc(const uint8_t* guide, int pitch, int width, int height, int max_disp,
                                 void* cost, zncc_dtype dtype, float sigma_s, float sigma_r, int iters,
                                 void* cuda_stream) {
    g_free_error[0] = '\0';
    if (!guide || !cost) {
        set_free_error("dt_aggregate_noalloc: guide or cost pointer is NULL");
        return ZNCC_EINVAL;
    }
    if (width < 1 || height < 1 || max_disp < 1 || pitch < width) {
        set_free_error("dt_aggregate_noalloc: width, height and max_disp must be >= 1 and pitch >= width");
        return ZNCC_EINVAL;
    }
    if (dtype != ZNCC_F32 && dtype != ZNCC_F16) {
        set_free_error("dt_aggregate_noalloc: unknown dtype");
        return ZNCC_EINVAL;
    }
    if (!(sigma_s > 0.0f) || !isfinite(sigma_s) || !(sigma_r > 0.0f) || !isfinite(sigma_r) || iters < 0 ||
        iters > 64) {
        set_free_error("dt_aggregate_noalloc: sigma_s and sigma_r must be > 0 and iters in [0, 64]");
        return ZNCC_EINVAL;
    }
    if (width > 3072 || height > 4096 || max_disp > 1024) {
        set_free_error("dt_aggregate_noalloc: width must be <= 3072, height <= 4096 and max_disp <= 1024");
        return ZNCC_EUNSUPPORTED;
    }
    const long long npix = (long long)width * height;
    if (npix > kNoallocMaxPixels) {
        set_free_error("dt_aggregate_noalloc: %d x %d needs %lld bytes of scratch (32 per pixel); the static "
                       "scratch holds %lld bytes, so width * height must be <= %lld",
                       width, height, npix * 32, (long long)kNoallocScratchBytes, kNoallocMaxPixels);
        return ZNCC_EUNSUPPORTED;
    }
    if (iters == 0) return ZNCC_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_cuda_fail(e, "current device");
    if (dev < 0 || dev >= kNoallocDevices) {
        set_free_error("dt_aggregate_noalloc: device ordinals above %d are not supported", kNoallocDevices - 1);
        return ZNCC_EUNSUPPORTED;
    }
    const cudaStream_t st = (cudaStream_t)cuda_stream;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoallocDevice* d = nullptr;
    unsigned char* scratch = nullptr;
    ZNCC_TRY(noalloc_device(dev, &d, &scratch));
    float4* coefH = reinterpret_cast<float4*>(scratch);
    float4* coefV = coefH + npix;

    CoefBatch cb;
    memset(&cb, 0, sizeof(cb));
    cb.npairs = 1;
    CoefArgs& ca = cb.p[0];
    ca.guide = guide;
    ca.pitch = pitch;
    ca.W = width;
    ca.H = height;
    ca.K = (float)exp(-1.0 / (double)sigma_s);
    ca.inv_sr255 = (float)(1.0 / (255.0 * (double)sigma_r));
    ca.coefH = coefH;
    ca.coefV = coefV;
    cb.total_threads = dt_coef_threads(width, height);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    e = launch_dt_coef(cb, st);
    if (e != cudaSuccess) return noalloc_cuda_fail(e, "DT coefficients");

    LinePass lp;
    lp.vol = cost;
    lp.dstride = max_disp;
    lp.dcount = max_disp;
    lp.dtype = dtype;
    lp.s2 = scale_s2(sigma_s);
    for (int it = 0; it < 2 * iters; ++it) {
        lp.horiz = (it % 2) == 0;
        LineArgs a;
        fill_line_args(a, lp, width, height, coefH, coefV);
        ZNCC_TRY(noalloc_plan(*d, a, lp));
        LineBatch b;
        memset(&b, 0, sizeof(b));
        int threads = 0;
        size_t stage = 0, rest = 0;
        add_line_pair(b, a, kLineStore, dtype, threads, stage, rest);
        b.stage_bytes = (long long)stage;
        const size_t smem = stage + rest;
        e = size_line_grid(b, threads, smem, kLineStore, dtype, d->num_sms);
        if (e != cudaSuccess) return noalloc_cuda_fail(e, "occupancy query");
        g_launches.fetch_add(1, std::memory_order_relaxed);
        e = launch_line_batch(b, threads, smem, kLineStore, dtype, st);
        if (e != cudaSuccess) return noalloc_cuda_fail(e, "DT pass pair");
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

zncc_status fastdt_codec(const int16_t* values, int n, uint8_t* codes, int16_t* decoded, void* cuda_stream) {
    g_free_error[0] = '\0';
    if (n < 0 || (!values && n > 0)) {
        set_free_error("fastdt_codec: n < 0, or values is NULL and n > 0");
        return ZNCC_EINVAL;
    }
    g_launches.fetch_add(n > 0 ? 1 : 0, std::memory_order_relaxed);
    const cudaError_t e = launch_fastdt_codec(values, n, codes, decoded, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) {
        set_free_error("fastdt_codec: %s (%s)", cudaGetErrorName(e), cudaGetErrorString(e));
        return ZNCC_ECUDA;
    }
    return ZNCC_OK;
}

zncc_status zncc_run(zncc_ctx* c, const uint8_t* left, const uint8_t* right, int pitch, float sigma_s,
                     float sigma_r, int iters, zncc_dtype storage, uint16_t* disp) {
    if (!c) return ZNCC_EINVAL;
    c->err.clear();
    ZNCC_TRY(check_images(c, left, right, pitch));
    if (!disp) return fail(c, ZNCC_EINVAL, "disp pointer is NULL");
    if (storage != ZNCC_F32 && storage != ZNCC_F16 && storage != ZNCC_I8) return fail(c, ZNCC_EINVAL, "unknown dtype");
    ZNCC_TRY(check_dt(c, sigma_s, sigma_r, iters));
    PairIO io{c, left, right, pitch, disp, nullptr, 0};
    return run_fused(c, &io, 1, sigma_s, sigma_r, iters, storage);
}

zncc_status zncc_run_batch(zncc_ctx* const* ctxs, const uint8_t* const* lefts, const uint8_t* const* rights,
                           const int* pitches, uint16_t* const* disps, int n, float sigma_s, float sigma_r,
                           int iters, zncc_dtype storage) {
    if (!ctxs || !ctxs[0] || n < 1) return ZNCC_EINVAL;
    zncc_ctx* lc = ctxs[0];
    lc->err.clear();
    if (n > kMaxBatch) return fail(lc, ZNCC_EINVAL, "at most 32 pairs per batch");
    if (!lefts || !rights || !pitches || !disps) return fail(lc, ZNCC_EINVAL, "a batch array is NULL");
    if (storage != ZNCC_F32 && storage != ZNCC_F16 && storage != ZNCC_I8)
        return fail(lc, ZNCC_EINVAL, "unknown dtype");
    ZNCC_TRY(check_dt(lc, sigma_s, sigma_r, iters));
    PairIO io[kMaxBatch];
    for (int i = 0; i < n; ++i) {
        zncc_ctx* c = ctxs[i];
        if (!c) return fail(lc, ZNCC_EINVAL, "a context is NULL");
        if (c->device != lc->device) return fail(lc, ZNCC_EINVAL, "the contexts of a batch share one device");
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == c) return fail(lc, ZNCC_EINVAL, "a context appears twice in the batch");
        if (check_images(c, lefts[i], rights[i], pitches[i]) != ZNCC_OK) return fail(lc, ZNCC_EINVAL, c->err);
        if (!disps[i]) return fail(lc, ZNCC_EINVAL, "disp pointer is NULL");
        io[i] = PairIO{c, lefts[i], rights[i], pitches[i], disps[i], nullptr, 0};
    }
    // a pair that fills the device by itself runs its own chain; the others share launches
    PairIO small[kMaxBatch];
    int nsmall = 0;
    for (int i = 0; i < n; ++i) {
        if (fills_device(io[i].c)) ZNCC_TRY(run_fused(lc, &io[i], 1, sigma_s, sigma_r, iters, storage));
        else small[nsmall++] = io[i];
    }
    return nsmall ? run_fused(lc, small, nsmall, sigma_s, sigma_r, iters, storage) : ZNCC_OK;
}

namespace {
// The device work of zncc_run_host on the context's stream: the uploads, the fused run, and the
// map's way back (disp_dev: the device address of a page-locked map, which the last kernel then
// stores into; NULL: a copy from the context's map).
zncc_status issue_host_run(zncc_ctx* c, const uint8_t* left_host, const uint8_t* right_host, int pitch,
                           float sigma_s, float sigma_r, int iters, zncc_dtype storage, uint16_t* disp_host,
                           uint16_t* disp_dev) {
    const size_t npix = (size_t)c->W * c->H;
    // contiguous rows go up as one linear copy each, pitched ones row by row
    if (pitch == c->W) {
        ZNCC_CUDA(c, cudaMemcpyAsync(c->img, left_host, npix, cudaMemcpyHostToDevice, c->stream), "left image upload");
        ZNCC_CUDA(c, cudaMemcpyAsync(c->img + npix, right_host, npix, cudaMemcpyHostToDevice, c->stream),
                  "right image upload");
    } else {
        ZNCC_CUDA(c, cudaMemcpy2DAsync(c->img, c->W, left_host, pitch, c->W, c->H, cudaMemcpyHostToDevice,
                                       c->stream), "left image upload");
        ZNCC_CUDA(c, cudaMemcpy2DAsync(c->img + npix, c->W, right_host, pitch, c->W, c->H, cudaMemcpyHostToDevice,
                                       c->stream), "right image upload");
    }
    ZNCC_TRY(zncc_run(c, c->img, c->img + npix, c->W, sigma_s, sigma_r, iters, storage,
                      disp_dev ? disp_dev : c->disp));
    if (!disp_dev)
        ZNCC_CUDA(c, cudaMemcpyAsync(disp_host, c->disp, npix * sizeof(uint16_t), cudaMemcpyDeviceToHost,
                                     c->stream), "disparity download");
    return ZNCC_OK;
}

// Whether p is page-locked host memory of the context's device; its device address in *dev.
bool pinned_on(const zncc_ctx* c, const void* p, void** dev) {
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, p) != cudaSuccess) {
        cudaGetLastError();                         // (a pageable pointer is not an error)
        return false;
    }
    if (pa.type != cudaMemoryTypeHost || !pa.devicePointer || pa.device != c->device) return false;
    if (dev) *dev = pa.devicePointer;
    return true;
}
}  // namespace

zncc_status zncc_run_host(zncc_ctx* c, const uint8_t* left_host, const uint8_t* right_host, int pitch,
                          float sigma_s, float sigma_r, int iters, zncc_dtype storage,
                          uint16_t* disp_host) {
    if (!c) return ZNCC_EINVAL;
    c->err.clear();
    ZNCC_TRY(check_images(c, left_host, right_host, pitch));
    if (!disp_host) return fail(c, ZNCC_EINVAL, "disp_host pointer is NULL");
    const size_t npix = (size_t)c->W * c->H;
    if (!c->img) {
        cudaError_t e = device_alloc((void**)&c->img, 2 * npix);
        if (e == cudaSuccess) e = device_alloc((void**)&c->disp, npix * sizeof(uint16_t));
        if (e != cudaSuccess) {
            cudaGetLastError();
            free_dev(c->img);
            free_dev(c->disp);
            return fail(c, ZNCC_ENOMEM, std::string("image buffers: ") + cudaGetErrorString(e));
        }
        ++c->gen;
    }
    // a page-locked map the device can address takes the last kernel's stores directly
    void *dmap = nullptr, *dleft = nullptr, *dright = nullptr;
    const bool map_pinned = pinned_on(c, disp_host, &dmap);
    const bool imgs_pinned = pinned_on(c, left_host, &dleft) && pinned_on(c, right_host, &dright);
    uint16_t* disp_dev = map_pinned ? static_cast<uint16_t*>(dmap) : nullptr;
    // A call that repeats the previous one (the same host buffers, still page-locked at the same
    // device mappings, parameters, tuning, stream and context buffers), on a stream other than
    // the legacy default one, is captured once as a CUDA graph and replayed from then on: the
    // device runs the uploads, the kernels and the map's way back without waiting for the host
    // to issue them. The buffers are looked up on every call, so a buffer freed and allocated
    // anew is never reached through an old mapping. A capture that fails leaves the call to
    // direct issue (and that argument set uncaptured).
    const zncc_ctx::HostKey key{left_host, right_host, disp_host, dleft,         dright,      dmap,
                                pitch,     iters,      (int)storage, sigma_s, sigma_r, c->gen};
    if (c->host_graph && map_pinned && imgs_pinned && key == c->host_key && !c->profiling) {
        ZNCC_CUDA(c, cudaGraphLaunch(c->host_graph, c->stream), "graph launch");
        ZNCC_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
        return ZNCC_OK;
    }
    const bool repeat = key == c->host_last && !(key == c->host_nocapture);
    c->host_last = key;
    if (repeat && !c->profiling && c->stream != nullptr && map_pinned && imgs_pinned) {
        if (c->host_graph) cudaGraphExecDestroy(c->host_graph);
        c->host_graph = nullptr;
        cudaGraph_t g = nullptr;
        cudaGraphExec_t x = nullptr;
        bool ok = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            const zncc_status s = issue_host_run(c, left_host, right_host, pitch, sigma_s, sigma_r, iters, storage,
                                                 disp_host, disp_dev);
            const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
            ok = s == ZNCC_OK && e == cudaSuccess && g != nullptr && key.gen == c->gen;
        }
        if (ok) ok = cudaGraphInstantiate(&x, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        c->err.clear();
        if (ok) {
            c->host_graph = x;
            c->host_key = key;
            ZNCC_CUDA(c, cudaGraphLaunch(x, c->stream), "graph launch");
            ZNCC_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
            return ZNCC_OK;
        }
        if (x) cudaGraphExecDestroy(x);
        c->host_nocapture = key;
    }
    ZNCC_TRY(issue_host_run(c, left_host, right_host, pitch, sigma_s, sigma_r, iters, storage, disp_host, disp_dev));
    ZNCC_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
    return ZNCC_OK;
}

const char* zncc_last_error(const zncc_ctx* c) { return c ? c->err.c_str() : g_free_error; }

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
        case ZNCC_TUNE_AHAT_SMS: c->ahat_sms = value; break;
        case ZNCC_TUNE_PLANE: c->plane_mode = value ? 1 : 0; break;
        case ZNCC_TUNE_ROW_LOADS: c->row_nobulk = value ? 1 : 0; break;
        case ZNCC_TUNE_LINE_LOADS:
            if (value > 2) return fail(c, ZNCC_EINVAL, "line staging must be 0, 1 or 2");
            c->line_loads = value;
            break;
        case ZNCC_TUNE_WAIT_DRILL: c->wait_drill = value ? 1 : 0; break;
        case ZNCC_TUNE_AHAT_JOIN:
            if (value > 2) return fail(c, ZNCC_EINVAL, "A_hat join must be 0, 1 or 2");
            c->ahat_join = value;
            break;
        case ZNCC_TUNE_V_LPC:
            if (value != 0 && value != 1 && value != 2 && value != 4)
                return fail(c, ZNCC_EINVAL, "columns per block must be 0, 1, 2 or 4");
            c->v_lpc = value;
            break;
        case ZNCC_TUNE_PLANE_CS:
            if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8)
                return fail(c, ZNCC_EINVAL, "plane cluster size must be 0, 1, 2, 4 or 8");
            c->plane_force_cs = value;
            break;
        case ZNCC_TUNE_H_TQ:
        case ZNCC_TUNE_V_TQ:
            if (value != 0 && value != 2 && value != 4 && value != 8)
                return fail(c, ZNCC_EINVAL, "lanes per chunk must be 0, 2, 4 or 8");
            (key == ZNCC_TUNE_H_TQ ? c->h_tq : c->v_tq) = value;
            break;
        default: return fail(c, ZNCC_EINVAL, "unknown tuning key");
    }
    c->plans.clear();
    c->occ.clear();
    c->plane_cs = -1;
    ++c->gen;
    return ZNCC_OK;
}

zncc_status zncc_device_faults(zncc_ctx* c, uint32_t* faults) {
    if (!c || !faults) return ZNCC_EINVAL;
    c->err.clear();
    *faults = 0;
    unsigned v = 0;
    ZNCC_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
    ZNCC_CUDA(c, cudaMemcpy(&v, c->fault, sizeof(v), cudaMemcpyDeviceToHost), "fault word read");
    if (v) ZNCC_CUDA(c, cudaMemset(c->fault, 0, sizeof(unsigned)), "fault word clear");
    *faults = v;
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
