// kernels.h -- argument blocks and launchers of the device kernels (internal to libzncc).
#pragma once

#include <cuda.h>                 // CUtensorMap (the descriptor type only; no driver calls here)
#include <cuda_runtime.h>
#include <stdint.h>

namespace zncc {

enum { kModeRaw = 0, kModeHPair = 1, kModeWta = 2 };   // k_zncc_row variants
enum { kLineStore = 0, kLineWta = 1 };                  // k_line_pair variants
constexpr int kMaxBatch = 32;                           // pairs per batched launch

// WTA output of a launch: a running best (value, d) per pixel that persists across launches
// which split the disparity range, and the disparity map written by the last one.
struct WtaOut {
    float* bestv;             // [H][W] (read unless first, written unless last)
    int* bestd;               // [H][W]
    uint16_t* disp;           // [H][W] (written by the last launch)
    int first, last;
};

struct RowArgs {
    const uint8_t* left;
    const uint8_t* right;
    int pitch, W, H, D;
    int nch, tq;              // chunks per row (padded to whole warps), lanes per chunk
    int d_lo, d_hi;           // disparity range of this launch (d_lo a multiple of 4)
    int spb;                  // disparity slices (4 * tq each) per visit of a row
    void* vol;                // output [H][W][dstride] of float or half (Raw / HPair)
    long long dstride;        // entries per pixel in the output
    int d_out0;               // disparity stored at entry 0 of a pixel
    int vec;                  // 16-byte (float) / 8-byte (half) accesses allowed
    float K, inv_sr255;       // DT weights (HPair): exp(-1/sigma_s), 1/(255 sigma_r); guide = left
    float4* coefH_out;        // (HPair) if set, the row coefficients go here too ([H][W], as k_dt_coef)
    const float2* mulmap;     // (HPair, FastDT codes) [H][W]: (unused, output scale (1-K)^2/A_hat_1)
    float s2;                 // (1 - K)^2
    WtaOut wta;               // (Wta)
    int minb2;                // use the two-blocks-per-SM variant where the block allows
    int bulk;                 // (HPair) stage the image rows by bulk asynchronous copies: both
                              // images and the pitch 16-byte aligned, W a multiple of 16
    int item0, nitems;        // this pair's units (row, slice), or rows (Wta), in a batched launch
};

// One cost-kernel launch over up to kMaxBatch pairs of the same window radius, passed by
// value. Of G blocks, block b takes the units [b * total / G, (b+1) * total / G), in order.
struct RowBatch {
    int npairs, total_items, grid, mode;
    unsigned* fault;          // device word of the launching context: bits of kFault* set by the kernel
    RowArgs p[kMaxBatch];
};

// Device-side faults a kernel records instead of waiting without end (ZNCC_FAULT_* of zncc.h).
constexpr unsigned kFaultBulkWait = 1u;      // a bulk copy of image rows did not complete in time
constexpr unsigned kFaultBulkDrain = 2u;     // ... nor after the second wait (the block then stopped)
constexpr unsigned kFaultTmaWait = 4u;       // a TMA copy of a DT pass step did not complete in time
constexpr unsigned kFaultTmaAlign = 8u;      // a TMA destination was not 128-byte aligned (not copied)
// Polls of an mbarrier before a wait counts as timed out (each poll may suspend the thread for a
// while; a copy from L2 or HBM completes within a few thousand).
constexpr unsigned kBulkWaitPolls = 1u << 24;
constexpr unsigned kDrillWaitPolls = 64;     // the wait drill's limit (ZNCC_TUNE_WAIT_DRILL)

struct LineArgs {
    void* vol;                // float or half cost volume (output, and input unless src is set)
    const void* src;          // input volume with the layout of vol (NULL: vol itself)
    int src_ones;             // the input is 1 at every element (src and vol are not read)
    long long elem_stride;    // entries between consecutive positions of a line
    long long line_stride;    // entries between consecutive lines
    int n, nlines;            // line length, number of lines
    int dcount;               // valid disparity entries per pixel
    int d_base;               // disparity of entry 0 (WTA)
    int tq, lpc, nch;         // lanes per chunk, lines per block, chunks per line and CTA
    int cs;                   // CTAs per line (a thread-block cluster; 1 = none, then lpc >= 1)
    int per_block;            // work items (line group, disparity slice) per block
    // per position of each line ([nlines][n], the pass's own line-major order): the multiplier
    // of the input and the scale of the output (NULL: 1 and s2)
    const float2* mulmap;
    const float4* coef;       // coefficients: coef[line * coef_line_stride + pos]
    long long coef_line_stride;
    float s2;
    int vec;                  // 16-byte (float) / 8-byte (half) accesses allowed
    int async;                // vec, and the next slices are streamed through shared memory
    int horiz;                // lines are rows (positions x) rather than columns (positions y)
    // the streamed slices arrive by TMA: one tensor copy per chunk and step from the pass's
    // tensor map (LineBatch::tmap) instead of 16-byte cp.async per thread and position
    int tma;
    // (Wta) per-pixel keys (ordered value << 32 | ~d), merged with atomicMax by every block that
    // saw part of a pixel's disparities; zero before the launch, turned into disparities (and
    // zeroed again) by k_wta_finish
    unsigned long long* keys;
    long long pix_line, pix_pos;  // pixel of (line, pos) is line * pix_line + pos * pix_pos
    // position of this pair in a batched launch: items and steps (line group, slice) are
    // numbered pair by pair
    int item0, nitems, step0, nsteps;
};

// One line-pair launch over up to kMaxBatch pairs, passed by value. Of G blocks (or clusters),
// block b takes the items [b * total / G, (b+1) * total / G) of all pairs, in order; an item is
// one step (line group, disparity slice) in both modes, or a whole line group for FastDT
// stores.
struct LineBatch {
    int npairs, total_items, total_steps, grid;
    int co_async;             // coefficients streamed by cp.async (two buffers; line_coef_async)
    long long stage_bytes;    // staging region (the largest pair's), before the other arrays
    unsigned* fault;          // device fault word (kFaultTmaWait), or NULL without TMA
    int drill;                // (tests) one thread per block waits out an mbarrier nobody arrives on
    LineArgs p[kMaxBatch];
    // (tma) per pair: the input volume as a 3-D tensor {entries per pixel, W, H}, box
    // {4 tq, 16, 1} (rows) or {4 tq, 1, 16} (columns): one chunk's positions of one slice
    CUtensorMap tmap[kMaxBatch];
};

// Launch configuration with programmatic stream serialization (the kernel may start while
// the previous kernel on the stream finishes; it waits for it in griddep_wait) and, for
// cluster > 1, thread-block clusters of that many CTAs along x. attr must hold 2 entries.
void launch_config(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, dim3 grid, dim3 block, size_t smem,
                   cudaStream_t st, int cluster);

size_t zncc_row_smem_bytes(int R, int mode, int dtype, const RowArgs& a, int nthreads);
// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) for a kernel on the current device, made only
// when the size exceeds what an earlier call set (a launch pays for it once, not every time);
// forget_smem_attributes() drops the record (zncc_create calls it, so that contexts created
// after a device reset set the attributes again).
cudaError_t set_max_smem(const void* fn, size_t smem);
void forget_smem_attributes();
bool zncc_row_bulk_fits_host(int R, int dtype, const RowArgs& a, int nthreads);
// A pass whose coefficients (and multipliers) can be streamed (at least two slices per line
// group); the shared memory of a block with one or two buffers of them.
bool line_coef_async(const LineArgs& a);
size_t line_pair_smem_bytes(int mode, int dtype, const LineArgs& a, bool co_async);
cudaError_t launch_line_batch(const LineBatch& b, int threads, size_t smem, int mode, int dtype,
                              cudaStream_t st);

cudaError_t launch_zncc_row(int R, const RowBatch& b, int threads, size_t smem, int mode, int dtype,
                            cudaStream_t st);
cudaError_t zncc_row_occupancy(int R, int mode, int dtype, int threads, size_t smem, bool minb2,
                               bool single, int* blocks_per_sm);
size_t line_stage_bytes(int dtype, const LineArgs& a);

// TMA staging of the DT pairs: the chunks whose lanes share one shared-memory wavefront of
// the staged reads (each lane reads 4 entries of elem bytes; a wavefront serves 128 bytes),
// and the bytes of one chunk's slot: its box of kL + G - 1 positions x 4 tq entries, rounded up
// to the 128-byte alignment of a tensor copy's destination.
__host__ __device__ inline int line_tma_chunks_per_wavefront(int tq, int elem) {
    const int g = 32 / (elem * tq);
    return g > 1 ? g : 1;
}
__host__ __device__ inline int line_tma_slot_bytes(int tq, int elem) {
    const int g = line_tma_chunks_per_wavefront(tq, elem);
    return ((16 + g - 1) * 4 * tq * elem + 127) / 128 * 128;
}
// single: the variant for launches of one pair (npairs == 1), which the launchers pick
cudaError_t line_pair_occupancy(int mode, int dtype, int threads, size_t smem, bool single, bool cluster,
                                int* blocks_per_sm);
// clusters of cs CTAs that can be resident at once on the device
cudaError_t line_pair_max_clusters(int mode, int dtype, int threads, size_t smem, bool single, int cs,
                                   int* clusters);
cudaError_t launch_window_stats(const uint8_t* img, int pitch, int W, int H, int r, int x_begin,
                                int nx, int* S, int* Q, float* isig, int2* packed,
                                cudaStream_t st);
struct CoefArgs {
    const uint8_t* guide;
    int pitch, W, H;
    float K, inv_sr255;       // exp(-1/sigma_s), 1/(255 sigma_r)
    float4* coefH;            // [H][W]
    float4* coefV;            // [W][H]
    long long thread0;        // first thread (k_dt_coef_cols: block) of this pair in the launch
};
struct CoefBatch {
    int npairs;
    long long total_threads;
    CoefArgs p[kMaxBatch];
};
cudaError_t launch_dt_coef(const CoefBatch& b, cudaStream_t st);

// One DT pass pair over an A_hat plane (the response of an all-ones plane, Sec. IV-C), a
// line per warp, the weights from the guide: aout = pair(ain, or ones), and the pass's
// multipliers (in_mul ? xscale * ain : 1, yscale / aout) in its line order.
struct AhatArgs {
    const uint8_t* guide;
    int pitch, W, H;
    const float* ain;         // [H][W], or nullptr for an all-ones input
    float* aout;              // [H][W]
    float2* mulmap;           // [nlines][n] or nullptr
    int in_mul;               // mulmap.x = ain (1) or 1 (0)
    int line0;                // first line of this pair in the launch
};
struct AhatBatch {
    int npairs, total_lines, horiz, nmax;
    float K, inv_sr255, s2;
    float xscale, yscale;     // multiplier factors: 1 and s2, or 1/T and s2 T for FastDT codes
    AhatArgs p[kMaxBatch];
};
cudaError_t launch_ahat_pair(const AhatBatch& b, cudaStream_t st);
// Dynamic shared memory of one A_hat pass-pair block for lines of at most nmax positions.
size_t ahat_pass_smem_bytes(int nmax);
long long dt_coef_threads(int W, int H);
// The column coefficients only, coalesced: one block per 32 columns x 4 chunks; thread0 and
// total_threads of the batch count blocks.
cudaError_t launch_dt_coef_cols(const CoefBatch& b, cudaStream_t st);
long long dt_coef_col_blocks(int W, int H);
cudaError_t launch_wta_volume(const void* cost, int dtype, int W, int H, int D, uint16_t* disp,
                              cudaStream_t st);

// The end of a fused WTA: each pixel's key becomes its disparity, and the key is zeroed.
struct WtaFinishArgs {
    unsigned long long* keys;
    uint16_t* disp;
    long long npix, thread0;
};
struct WtaFinishBatch {
    int npairs;
    long long total_threads;
    WtaFinishArgs p[kMaxBatch];
};
cudaError_t launch_wta_finish(const WtaFinishBatch& b, cudaStream_t st);
// The multiplier map of a pass along rows (horiz) or columns of a W x H image: for each
// (line, position), (ain ? ain[pix] : 1, aout ? s2 / aout[pix] : s2), ain/aout [H][W].
// The progressive-scan ZNCC (ablation baseline): packL [H][W] and packR [H][W + D - 1]
// hold (S, inv_sigma bits) of the window centred at x (left) and at x - d (right, centre c
// at index c + D - 1), from k_window_stats.
struct ScanArgs {
    const uint8_t* left;
    const uint8_t* right;
    int pitch, W, H, D;
    const int2* packL;
    const int2* packR;
    void* vol;                // [H][W][D] float or half
};
cudaError_t launch_zncc_scan(int R, const ScanArgs& a, int dtype, cudaStream_t st);
// The same cost volume with the window cross sums as a banded BF16 matrix product on the
// tensor cores (mma.sync, exact FP32 accumulation): identical values (zncc_mma.cuh).
cudaError_t launch_zncc_mma(int R, const ScanArgs& a, int dtype, cudaStream_t st);

cudaError_t launch_mulmap(const float* ain, float xscale, float s2, int W, int H, bool horiz, float2* out,
                          cudaStream_t st);

// The plane-resident fused path (plane.cu): a cluster of cs CTAs holds one disparity plane,
// CTA q the rows [q hb, (q+1) hb), for the cost, every DT pass pair and the WTA.
constexpr int kPlaneThreads = 384;
constexpr int kPlaneWarps = kPlaneThreads / 32;
// Size classes of the kernel (template instances): the longest row segment per lane and the
// most rows per CTA its registers hold, and the CTAs per SM it is compiled for. The host picks
// the smallest class that fits a pair: shorter unrolled loops and, for the first, twice the
// warps per SM.
constexpr int kPlaneClasses = 3;
constexpr int kPlaneSegMaxOf[kPlaneClasses] = {11, 21, 33};      // W <= 352, 672, 1024
constexpr int kPlaneBandMaxOf[kPlaneClasses] = {16, 24, 32};
constexpr int kPlaneMinBlocksOf[kPlaneClasses] = {2, 1, 1};
constexpr int kPlaneBandMax = 32;         // rows per CTA in the largest class
constexpr int kPlaneTileRows = 4;         // rows of window column sums per cost step
constexpr int kPlaneColsPerThread = 4;    // window-sum columns per thread: W + 2r <= 1536
constexpr int kPlaneMaxW = 1024;

// Byte offsets of a CTA's shared memory for a W x H pair of window radius r in clusters of cs.
struct PlaneLayout {
    int hb;                   // rows per CTA
    int wb;                   // row pitch of the image rows (bytes)
    int vw;                   // window-sum columns: W + 2r
    unsigned lut, plane, vt, st, cf, cb, lb, rb, total;
};
__host__ __device__ inline PlaneLayout plane_layout(int W, int H, int r, int cs) {
    PlaneLayout L;
    L.hb = (H + cs - 1) / cs;
    L.wb = (W + 15) & ~15;
    L.vw = W + 2 * r;
    auto up = [](unsigned o) { return (o + 15u) & ~15u; };
    unsigned o = 0;
    L.lut = o;
    o = up(o + 256u * 4u);
    L.plane = o;                                        // float [hb][W]
    o = up(o + (unsigned)L.hb * W * 4u);
    L.vt = o;                                           // int [kPlaneTileRows][vw]
    o = up(o + (unsigned)kPlaneTileRows * L.vw * 4u);
    L.st = o;                                           // int2 [2][kPlaneTileRows][W]: statistics
    o = up(o + 2u * kPlaneTileRows * W * 8u);
    L.cf = o;                                           // float2 [W]: forward maps (cs > 1)
    o = up(o + (cs > 1 ? (unsigned)W * 8u : 0u));
    L.cb = o;                                           // float2 [W]: backward maps (cs > 1)
    o = up(o + (cs > 1 ? (unsigned)W * 8u : 0u));
    L.lb = o;                                           // uint8 [hb + 2r][wb]: left rows
    o = up(o + (unsigned)(L.hb + 2 * r) * L.wb);
    L.rb = o;                                           // uint8 [hb + 2r][wb]: right rows
    o = up(o + (unsigned)(L.hb + 2 * r) * L.wb);
    L.total = o;
    return L;
}

struct PlaneArgs {
    const uint8_t* left;
    const uint8_t* right;
    int pitch, W, H, D, r;
    const int2* statsL;       // [H][W] (S, inv_sigma bits) of the left windows
    const int2* statsR;       // [H][W + D - 1]: right windows centred at c, at index c + D - 1
    unsigned long long* keys; // [H][W] WTA keys, zero before the launch
    int item0;                // items item0 + d, d in [0, D), are this pair's planes
};
struct PlaneBatch {
    int npairs, total_items, nclusters, cs, iters;
    float K, inv_sr255, s2;   // exp(-1/sigma_s), 1/(255 sigma_r), (1 - K)^2
    PlaneArgs p[kMaxBatch];
};
// The smallest size class holding rows of W pixels and bands of hb rows, or -1.
inline int plane_class(int W, int hb) {
    const int seg = ((W + 31) / 32) | 1;
    for (int k = 0; k < kPlaneClasses; ++k)
        if (seg <= kPlaneSegMaxOf[k] && hb <= kPlaneBandMaxOf[k]) return k;
    return -1;
}
cudaError_t plane_max_clusters(int cls, int cs, size_t smem, int* clusters);
cudaError_t launch_plane(const PlaneBatch& b, int cls, size_t smem, cudaStream_t st);
cudaError_t launch_fastdt_codec(const int16_t* values, int n, uint8_t* codes, int16_t* decoded, cudaStream_t st);

// Device allocation of the library (cudaMalloc, or an injected out-of-memory failure when the
// environment variable ZNCC_FAIL_DEVICE_ALLOC is 1).
cudaError_t device_alloc(void** p, size_t bytes);

// Scratch of dt_aggregate_noalloc: the DT coefficients of one W x H image (two float4 per
// pixel) in a static device array of this size; its address on the current device.
constexpr size_t kNoallocScratchBytes = 64ull << 20;
constexpr long long kNoallocMaxPixels = (long long)(kNoallocScratchBytes / (2 * sizeof(float4)));
cudaError_t noalloc_scratch_address(void** p);

// per-radius launchers, one translation unit each
#define ZNCC_DECLARE_ROW(R)                                                                     \
    cudaError_t launch_zncc_row_r##R(const RowBatch& b, int threads, size_t smem, int mode, int dtype, \
                                     cudaStream_t st);                                             \
    cudaError_t zncc_row_occupancy_r##R(int mode, int dtype, int threads, size_t smem, bool minb2, bool single, \
                                        int* bps);                                                    \
    cudaError_t launch_zncc_scan_r##R(const ScanArgs& a, int dtype, cudaStream_t st);                \
    cudaError_t launch_zncc_mma_r##R(const ScanArgs& a, int dtype, cudaStream_t st);
ZNCC_DECLARE_ROW(1)
ZNCC_DECLARE_ROW(2)
ZNCC_DECLARE_ROW(3)
ZNCC_DECLARE_ROW(4)
ZNCC_DECLARE_ROW(5)
ZNCC_DECLARE_ROW(6)
ZNCC_DECLARE_ROW(7)
#undef ZNCC_DECLARE_ROW

}  // namespace zncc
