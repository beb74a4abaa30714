/*
 * zncc.h -- C ABI of libzncc.so: ZNCC matching cost, domain-transformation (DT) cost
 * aggregation and winner-take-all (WTA) disparity on one GB300 GPU (sm_103a).
 *
 * Method: arXiv 2212.00476, "Efficient stereo matching on embedded GPUs with zero-means
 * cross correlation".
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Images are uint8 grayscale, H rows of W pixels, row pitch `pitch` bytes (>= W).
 *    `left` is the reference image I_R, `right` the target image I_T (Sec. III-A): pixel
 *    (x, y) of the left image is matched to (x - d, y) of the right image, d in [0, D).
 *  - Pixel reads outside an image are clamped to its nearest edge pixel (also for target
 *    centres x - d < 0).
 *  - Cost volumes are dense [H][W][D] arrays, the disparity axis fastest, of float
 *    (ZNCC_F32) or IEEE half (ZNCC_F16). Element (x, y, d) is at ((y * W) + x) * D + d.
 *  - Disparity maps are uint16 [H][W] (row pitch W).
 *  - Pointers named *_host are host memory; every other buffer pointer is device memory
 *    of the current CUDA device. The caller owns every buffer it passes; the library never
 *    frees or keeps them. Device buffers must stay valid until the work queued on the
 *    context's stream has completed.
 *  - Calls are asynchronous on the context's stream unless stated otherwise. They return a
 *    status and never abort or throw. On ZNCC_ECUDA the CUDA error text is available from
 *    zncc_last_error(). A context is not thread-safe: use one per host thread or stream.
 *  - Window side `win` = 2r+1 must be odd and in [3, 15]. Window sums are exact in int32
 *    (the largest, n*Q - S^2, stays below 2^31 for every allowed window).
 *  - W must be in [1, 3072] and H in [1, 4096] (a DT line is processed inside one thread
 *    block, and a row's image band inside one block's shared memory); D in [1, 1024].
 */
#ifndef ZNCC_H_
#define ZNCC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ZNCC_OK = 0,
    ZNCC_EINVAL = 1,        /* an argument is out of range or a pointer is NULL          */
    ZNCC_ENOMEM = 2,        /* a device or host allocation failed                        */
    ZNCC_ECUDA = 3,         /* a CUDA runtime call failed; see zncc_last_error()          */
    ZNCC_EBUSY = 4,         /* the server is shutting down or full                       */
    ZNCC_ENOTREADY = 5,     /* serve_poll: the request has not finished yet              */
    ZNCC_ETIMEOUT = 6,      /* serve_poll / serve_destroy: a bounded wait ran out         */
    ZNCC_EUNSUPPORTED = 7   /* a size the kernels do not handle                          */
} zncc_status;

/* Storage types. ZNCC_I8 is the FastDT storage of Sec. IV-C, for the intermediate volume of
 * the fused path only (zncc_run, zncc_run_batch, zncc_run_host, serve_submit): after every DT
 * pass pair but the last, the values v(d) of a pixel, divided by A_hat (the same pass pairs
 * applied to an all-ones plane, the per-pixel bound of |v|), are stored as
 * E = rint(16383 * (v(0) - v(d)) / A_hat), clamped to int16 and cut to an 8-bit code (the six
 * bits next to the leading ones of the two's-complement value and a 2-bit flag naming their
 * position; values >= 0, which do no better than d = 0, are code 0); the next pair reads the
 * code back as -E / 16383 * A_hat. One byte per element; the calls that take a caller-owned
 * cost volume reject it with ZNCC_EINVAL. */
typedef enum { ZNCC_F32 = 0, ZNCC_F16 = 1, ZNCC_I8 = 2 } zncc_dtype;

typedef struct zncc_ctx zncc_ctx;

/* Create a context for W x H pairs, disparities [0, max_disp), window side `win`.
 * Allocates the context's device scratch (window statistics, DT edge weights, the WTA
 * key map) on the current device; the cost volume of zncc_run is allocated on first use.
 * Sec. III-A defines the problem (I_R, I_T, D, window l = 2r+1). */
zncc_status zncc_create(int width, int height, int max_disp, int win, zncc_ctx** out);

/* Free the context and its scratch. Synchronizes the context's stream first. */
zncc_status zncc_destroy(zncc_ctx* ctx);

/* Bind a CUDA stream (cudaStream_t passed as void*; NULL = legacy default stream). */
zncc_status zncc_set_stream(zncc_ctx* ctx, void* cuda_stream);

/* Bytes of a [H][W][D] cost volume of the given storage type (0 on bad arguments). */
size_t zncc_volume_bytes(const zncc_ctx* ctx, zncc_dtype dtype);

/* Window statistics of one image (Sec. IV-B-1, Eq. (sum1)): for each centre (x, y),
 * S = sum of the (2r+1)^2 clamped pixels, Q = sum of their squares (exact int32), and
 * inv_sigma = 1/sqrt(n*Q - S^2) as float (0 when the window is flat), n = (2r+1)^2.
 * This is the per-image term of the rewritten cost, Eq. (2). Any output may be NULL.
 * Outputs are device [H][W]. */
zncc_status zncc_window_stats(zncc_ctx* ctx, const uint8_t* img, int pitch, int32_t* S,
                              int32_t* Q, float* inv_sigma);

/* ZNCC cost volume, Eq. (1) computed through Eq. (2): C(x,y,d) in [-1, 1],
 * C = (n*P - S_R*S_T) / sqrt((n*Q_R - S_R^2)(n*Q_T - S_T^2)) with P the window sum of
 * I_R(x+i,y+j) * I_T(x-d+i,y+j); 0 where either window is flat.
 * cost: device [H][W][D] of `dtype`. */
zncc_status zncc_cost_volume(zncc_ctx* ctx, const uint8_t* left, const uint8_t* right,
                             int pitch, void* cost, zncc_dtype dtype);

/* The same cost volume by the paper's "original" progressive scan (the comparison method of
 * Sec. V-B, Fig. ZNCC_compare): per (row, disparity) the window sum of products slides along
 * the row, one column of 2r+1 products in and one out, every column recomputed from the
 * pixels (no reuse across rows). An ablation baseline for zncc_cost_volume: identical
 * values (the integer numerator is exact, the normalization the same expression), slower.
 * Allocates 8 * (2W + D - 1) * H bytes of context scratch for window statistics on first use.
 * cost: device [H][W][D] of `dtype` (ZNCC_F32 or ZNCC_F16). */
zncc_status zncc_cost_volume_scan(zncc_ctx* ctx, const uint8_t* left, const uint8_t* right,
                                  int pitch, void* cost, zncc_dtype dtype);

/* The same cost volume with the window cross sums P on the tensor cores (the banded
 * correlation as a matrix product): per image row, A[x][(j,i)] = I_R(x+i, y+j) and
 * B[c][(j,i)] = I_T(c+i, y+j) in BF16 (pixels are exact), P(x, d) = (A B^T)[x][x-d] accumulated
 * in FP32, exact because every partial sum of a window stays below 2^24; then Eq. (2) as in
 * zncc_cost_volume. An ablation of the packed-column kernel: identical values. Allocates the
 * same statistics scratch as zncc_cost_volume_scan on first use.
 * cost: device [H][W][D] of `dtype` (ZNCC_F32 or ZNCC_F16). */
zncc_status zncc_cost_volume_mma(zncc_ctx* ctx, const uint8_t* left, const uint8_t* right,
                                 int pitch, void* cost, zncc_dtype dtype);

/* DT cost aggregation in place (Sec. III-B, Eqs. (3)-(6) with the weights of Eq. (11)),
 * `iters` times the pass chain left-to-right, right-to-left, up-to-down, down-to-up.
 * Weights: W = K * exp(-|G(p) - G(q)| / sigma_r), K = exp(-1/sigma_s), G = guide / 255
 * (guide = the reference/left image), p and q the two pixels of the step. Each pass
 * computes out = (1-K) * in + W * out(previous pixel in scan order), starting from
 * (1-K) * in at its first pixel: the paper's literal chain times (1-K)^(4*iters), which
 * keeps |cost| <= 1 and leaves the WTA result unchanged. sigma_s > 0, sigma_r > 0,
 * iters >= 0. cost: device [H][W][D] of `dtype` (F16: each pass rounds its output to half). */
zncc_status dt_aggregate(zncc_ctx* ctx, const uint8_t* guide_left, int pitch, void* cost,
                         zncc_dtype dtype, float sigma_s, float sigma_r, int iters);

/* dt_aggregate without allocating anything. The paper has no counterpart: this entry point
 * serves callers that must not allocate while they run, such as
 *  - a server that has committed its device memory in full to its own pools, for which a
 *    cudaMalloc would fail or evict,
 *  - a loop with a fixed latency budget, which cannot absorb cudaMalloc, nor cudaFree (it
 *    waits for every stream of the device), nor a host heap allocation,
 *  - code that runs where the allocator must not be entered (inside a custom allocator's
 *    own callbacks, or while another thread holds the allocator's lock).
 * It computes what dt_aggregate computes, on a width x height x max_disp volume, without a
 * context: the DT coefficients go to a scratch array compiled into the library's device code
 * (a static __device__ array of 64 MiB). The CUDA driver reserves it on a device when that
 * code is loaded into the device's context: under lazy module loading (CUDA_MODULE_LOADING=
 * LAZY, the default) at the first call of this entry point on the device; under eager loading
 * (CUDA_MODULE_LOADING=EAGER) when the context is created, in every process that loads the
 * library, whether it calls this entry point or not. It stays reserved until the context is
 * destroyed. The call makes no cudaMalloc, cudaFree or host heap allocation, and keeps no
 * device pointer between calls: it looks up the scratch's address (cudaGetSymbolAddress, a
 * host-side lookup) on every call, so a context that is destroyed and created again (after
 * cudaDeviceReset) gets the new address.
 *
 * Limit: width * height <= 2,097,152 pixels (32 bytes of scratch per pixel; 1920 x 1080
 * fits), with width <= 3072, height <= 4096, max_disp <= 1024. A larger image returns
 * ZNCC_EUNSUPPORTED before anything is queued, with the limit in zncc_last_error(NULL).
 *
 * Set-up: the first call on each device reads the device's limits, and its lookup of the
 * scratch's address may load the library's device code; the first call for each new line
 * length, disparity count and storage type chooses its launch shapes (occupancy queries).
 * Make these first calls once, at set-up, before any stream capture begins.
 *
 * Zero state: nothing in the scratch needs to start at zero. Each call writes every
 * coefficient of its image before it reads any, so leftovers of an earlier call are never
 * read.
 *
 * Overlapping calls race: there is one scratch per device, shared by every call in the
 * process. Calls whose GPU work may overlap (on different streams with no ordering between
 * them, or from several host threads) overwrite each other's coefficients and give wrong
 * results. Issue them on one stream, or order them with events. The host-side state is
 * guarded by a mutex, so concurrent calls are safe on the host; only their GPU work races.
 *
 * Arguments: guide_left is device uint8 [H][W] with row pitch `pitch` (>= width); cost is a
 * device [H][W][max_disp] volume of `dtype`, aggregated in place, owned by the caller and
 * valid until the queued work completes. sigma_s > 0, sigma_r > 0, iters in [0, 64]
 * (0 returns at once). cuda_stream is a cudaStream_t passed as void* (NULL = the legacy
 * default stream); the work is queued on it asynchronously. Errors: ZNCC_EINVAL (a NULL
 * pointer or an argument out of range), ZNCC_EUNSUPPORTED (the size limits above),
 * ZNCC_ECUDA (a CUDA call failed); the text is in zncc_last_error(NULL) (per host thread). */
zncc_status dt_aggregate_noalloc(const uint8_t* guide_left, int pitch, int width, int height,
                                 int max_disp, void* cost, zncc_dtype dtype, float sigma_s,
                                 float sigma_r, int iters, void* cuda_stream);

/* WTA disparity (Sec. III-C, Eq. (WTA1)): for each pixel the smallest d with the largest
 * cost (argmin of 1 - C). cost: device [H][W][D]; disp: device uint16 [H][W]. */
zncc_status wta_disparity(zncc_ctx* ctx, const void* cost, zncc_dtype dtype, uint16_t* disp);

/* The FastDT code (Sec. IV-C) on the device, as the fused path's ZNCC_I8 storage applies it:
 * for i < n, codes[i] = the 8-bit code of the 16-bit value values[i] and decoded[i] = the
 * 16-bit value that code stands for (the six kept bits in place, every bit above them one,
 * every bit below zero; code 0 is 0). values, codes, decoded: device arrays of n elements
 * (codes or decoded may be NULL). Runs on `cuda_stream` (NULL: the legacy default stream);
 * ZNCC_EINVAL for n < 0, or values NULL with n > 0 (n == 0 launches nothing); the text of an error is in zncc_last_error(NULL). */
zncc_status fastdt_codec(const int16_t* values, int n, uint8_t* codes, int16_t* decoded, void* cuda_stream);

/* The fused path: window statistics, ZNCC fused with the first horizontal DT pass pair,
 * the remaining DT passes, and WTA fused into the last vertical pass pair, so that the
 * volume is written once per horizontal/vertical hand-over and never read back for WTA.
 * iters == 0 computes ZNCC and WTA in one kernel without storing any volume.
 * `storage` is the type of the context-owned intermediate volume (F16 halves its traffic,
 * I8 quarters it at some loss of accuracy: the FastDT storage above).
 * left/right: device images; disp: device uint16 [H][W]. Sec. V-C fuses ZNCC with L2R and
 * WTA with D2U in the same way. */
zncc_status zncc_run(zncc_ctx* ctx, const uint8_t* left, const uint8_t* right, int pitch,
                     float sigma_s, float sigma_r, int iters, zncc_dtype storage,
                     uint16_t* disp);

/* The fused path over a batch of n <= 32 pairs of uneven sizes (each with its own context,
 * created for its W, H, D and window): every step (the DT coefficients, the cost kernel,
 * each DT pass pair) is one persistent launch over the pairs that share a block shape (the
 * cost kernel: a window size), so that small pairs share the GPU instead of leaving it idle;
 * a pair that fills the GPU by itself (W*H*D >= 2^25) runs its own chain of launches.
 * All launches go to the stream of ctxs[0], on which errors and timings are recorded; the
 * contexts must be distinct and on one device. lefts[i]/rights[i]: device images of pair i
 * (row pitch pitches[i]); disps[i]: its device uint16 disparity map. The DT parameters,
 * iteration count and storage type are common to the batch. Results are identical to n
 * zncc_run calls. Capturable in a CUDA graph. */
zncc_status zncc_run_batch(zncc_ctx* const* ctxs, const uint8_t* const* lefts,
                           const uint8_t* const* rights, const int* pitches,
                           uint16_t* const* disps, int n, float sigma_s, float sigma_r,
                           int iters, zncc_dtype storage);

/* zncc_run from host memory: copies the two images (row pitch `pitch`) to context-owned
 * device buffers, runs the fused path, copies the disparity map back to disp_host
 * (uint16 [H][W]) and synchronizes the stream before returning. Host buffers may be
 * pageable or pinned (pinned copies run asynchronously with respect to other streams). When
 * disp_host is page-locked host memory that the device can address (cudaHostAlloc,
 * cudaHostRegister, pinned torch tensors), the last kernel writes the map there directly
 * and there is no download copy. A call that repeats the previous one with page-locked images
 * and map (the same pointers, pitch, parameters and storage, no tuning or stream change in
 * between) on a stream other than the legacy default stream is captured once as a CUDA graph
 * and replayed from then on, so that the device runs the uploads, kernels and map stores without
 * waiting for the host to issue them; the replay reads the buffers' contents at the time of the
 * call. Where the capture fails the call is issued directly. */
zncc_status zncc_run_host(zncc_ctx* ctx, const uint8_t* left_host, const uint8_t* right_host,
                          int pitch, float sigma_s, float sigma_r, int iters,
                          zncc_dtype storage, uint16_t* disp_host);

/* ---- Serving: continuous batching of independent pairs ---------------------------------
 * A server owns a pool of contexts on the current device, a queue of requests and a scheduler
 * thread. Requests come from host memory and may differ in size, disparity range, window,
 * DT parameters and storage type. Whenever requests wait and slots are free, the scheduler
 * admits them in submission order and launches the small ones (W*H*D < 2^25) that share the
 * DT parameters, the iteration count and the storage type as one batched fused run
 * (zncc_run_batch, up to 32 pairs) and a larger one, which fills the GPU by itself, alone, so
 * that a new launch starts while earlier ones still run: larger pairs in arrival order on a
 * high-priority stream, the batches on a low-priority one, which fill the SMs the larger pairs
 * leave free.
 * Results are identical to running each pair alone: the batched kernels compute every pair
 * exactly as a single zncc_run does. Contexts are reused per request shape; the device memory
 * they hold (cost volume, DT coefficients, A_hat maps, images and disparity map) is charged
 * to `volume_budget_bytes`, and idle ones are freed, least recently used first, when a new
 * shape needs room. The paper has no serving layer; the batched path serves its workload of
 * many independent pairs. All server calls are thread-safe, except that no call may run
 * concurrently with or after serve_destroy. */
typedef struct zncc_server zncc_server;

/* Create a server: volume_budget_bytes (> 0) bounds the device memory of its contexts;
 * max_slots (>= 1) bounds the requests on the GPU at once (1 = one pair per launch, no
 * batching). The scheduler thread binds the device current at this call. */
zncc_status serve_create(size_t volume_budget_bytes, int max_slots, zncc_server** out);

/* Queue one pair: left_host/right_host are uint8 [height][width] (row pitch = width), copied
 * before the call returns (the caller may reuse them at once). The window, DT parameters,
 * iteration count and storage have the meaning and limits of zncc_run. Returns at once with
 * *ticket (> 0). Errors: ZNCC_EINVAL (bad arguments, or a request whose device memory alone
 * exceeds the budget: it could never run), ZNCC_EUNSUPPORTED (sizes beyond the kernels'
 * limits), ZNCC_EBUSY (the server is shutting down, or 65536 requests are outstanding),
 * ZNCC_ENOMEM (host memory). A request that merely has to wait for room is queued. */
zncc_status serve_submit(zncc_server* server, const uint8_t* left_host, const uint8_t* right_host,
                         int width, int height, int max_disp, int win, float sigma_s,
                         float sigma_r, int iters, zncc_dtype storage, uint64_t* ticket);

/* Result of a request: waits up to timeout_us (>= 0) microseconds for it to finish. On
 * completion copies its disparity map to disp_host (uint16 [height][width]), forgets the
 * ticket and returns the request's status: ZNCC_OK, or the error that stopped it
 * (ZNCC_ENOMEM / ZNCC_ECUDA from its context or launch, ZNCC_EBUSY if the server was
 * destroyed before it started). Not finished: ZNCC_ENOTREADY when timeout_us == 0,
 * ZNCC_ETIMEOUT otherwise (the ticket stays valid). Unknown ticket: ZNCC_EINVAL. */
zncc_status serve_poll(zncc_server* server, uint64_t ticket, uint16_t* disp_host, int timeout_us);

/* Where a served request's latency went, measured by the server (milliseconds). Host
 * timestamps: submit (serve_submit), issue (the scheduler starts queuing the request's batch
 * on a stream) and completion (the host function behind the batch's result copies runs);
 * CUDA events around the batch's image uploads, its fused run and its result copies.
 *   queue_ms        submit -> issue: waiting for a slot, budget room or the scheduler
 *   device_wait_ms  issue -> completion, less the batch's event-timed work: waiting on the
 *                   stream behind earlier batches, plus the completion callback's delay
 *   h2d_ms, run_ms, d2h_ms  the batch's uploads, fused run (every pair of the batch) and
 *                   result copies
 *   total_ms        submit -> completion = the sum of the five above
 *   batch_pairs     pairs in the request's batch
 * valid is 0 when the request failed before its batch ran (the times are then 0). */
typedef struct {
    double queue_ms, device_wait_ms, h2d_ms, run_ms, d2h_ms, total_ms;
    int batch_pairs, valid;
} zncc_serve_timing;

/* serve_poll, and on completion the request's latency breakdown in *timing (may be NULL). */
zncc_status serve_poll_timed(zncc_server* server, uint64_t ticket, uint16_t* disp_host, int timeout_us,
                             zncc_serve_timing* timing);

/* Stop the server: requests not yet started end with ZNCC_EBUSY, running batches are waited
 * for (at most 30 s), then every context, buffer and stream is freed. If the running work
 * does not finish in time, returns ZNCC_ETIMEOUT and leaves the server's memory allocated
 * (freeing buffers the GPU may still use would be unsafe). */
zncc_status serve_destroy(zncc_server* server);

/* Text of the last error the server recorded ("" if none); valid until the server's next
 * error. */
const char* serve_last_error(const zncc_server* server);

/* Text of the last error recorded on this context ("" if none). Valid until the next call
 * on the context. ctx == NULL returns the last error of a failed call without a context
 * (zncc_create, dt_aggregate_noalloc) on the calling host thread. */
const char* zncc_last_error(const zncc_ctx* ctx);

/* Faults the context's kernels recorded on the device since the last call (0: none), then
 * cleared. A kernel that waits for asynchronous copies gives up after a bounded number of polls
 * instead of waiting without end, records the fault here and stops: bit 0 = a bulk copy of the
 * cost kernel's image rows did not complete in time (the results of that launch are not
 * valid), bit 1 = the copies had still not landed after a second bounded wait, bit 2 = a TMA
 * copy of a DT pass's next slice did not complete in time (the pass then waits once more and
 * goes on; the map of that run is not valid), bit 3 = a TMA destination in shared memory was
 * not 128-byte aligned (the copy was skipped; the map is not valid). Synchronizes the
 * context's stream. ZNCC_EINVAL for a NULL argument; ZNCC_ECUDA if the read fails. */
zncc_status zncc_device_faults(zncc_ctx* ctx, uint32_t* faults);

/* Static text for a status code. */
const char* zncc_status_string(zncc_status status);

/* Launch-shape knobs of a context (0 = automatic for every key), for autotuning:
 *   ZNCC_TUNE_ROW_MINB2  cost kernel: 1 = register-limited variant with two blocks per SM
 *                        where the block has at most 320 threads, 0 = one block per SM
 *                        without spills, beside which the column coefficients and the A_hat
 *                        chain run on a second stream (default)
 *   ZNCC_TUNE_ROW_SPB    cost kernel: disparity slices per block
 *   ZNCC_TUNE_H_TQ       horizontal DT pairs: lanes per 16-pixel chunk (2, 4 or 8)
 *   ZNCC_TUNE_V_TQ       vertical DT pairs: lanes per 16-pixel chunk (2, 4 or 8)
 *   ZNCC_TUNE_AHAT_SMS   (F16, I8 storage) SMs the cost kernel leaves free for the A_hat chain,
 *                        which runs beside it on a second stream (default 8)
 *   ZNCC_TUNE_PLANE      (F32 storage, iters >= 1) 1 = the plane-resident path for pairs with
 *                        W <= 1024 whose rows split into bands of at most 32 rows over a
 *                        cluster of 1, 2, 4 or 8 CTAs that fit in shared memory (H <= 256):
 *                        each disparity plane stays in shared memory for the cost, every DT
 *                        pass pair and the WTA, and the cost volume is never stored; 0 = the
 *                        streaming path (cost volume in device memory; the default: on GB300
 *                        as fast at 320x96, D = 32 and faster at every larger measured shape)
 *   ZNCC_TUNE_PLANE_CS   the plane-resident path's cluster size (1, 2, 4 or 8; 0 = automatic);
 *                        a size whose band does not fit sends the pair to the streaming path
 *   ZNCC_TUNE_ROW_LOADS  cost kernel fused with the first horizontal pair: 1 = stage the image
 *                        rows with plain loads; 0 (automatic) = bulk asynchronous copies (the
 *                        TMA unit) where both images and the pitch are 16-byte aligned and W is
 *                        a multiple of 16, plain loads elsewhere
 *   ZNCC_TUNE_V_LPC      vertical DT pairs that store the volume: at most this many adjacent
 *                        columns per block (1, 2 or 4; 0 = automatic, which prefers two
 *                        resident blocks per SM). Adjacent columns of a row share DRAM pages,
 *                        so wider groups make longer runs per page at the cost of residency;
 *                        the last vertical pair with WTA keeps the automatic shape
 *   ZNCC_TUNE_LINE_LOADS DT pairs: 1 = stream the next slices into shared memory with 16-byte
 *                        cp.async per thread and position; 0 (automatic) = in the horizontal
 *                        pairs one TMA tensor copy per 16-position chunk and slice, completing
 *                        on per-warp mbarriers, where the volume and its pixel stride are
 *                        16-byte aligned, F32 or F16 reads span at most four chunks per
 *                        shared-memory wavefront, a line fits one CTA and shared memory allows;
 *                        cp.async elsewhere and in the vertical pairs; 2 = TMA in the vertical
 *                        pairs too (a column box fetches one pixel row at a time: faster for
 *                        some shapes, far slower for others)
 *   ZNCC_TUNE_WAIT_DRILL (tests) 1 = every DT pair launch has one thread per block wait, with a
 *                        64-poll limit, for an mbarrier phase that nothing completes; the wait
 *                        runs out and records fault bit 2 (see zncc_device_faults) while the
 *                        results stay those of a normal run. A check of the bounded-wait path
 *                        that faults, traps and hangs nothing
 *   ZNCC_TUNE_AHAT_JOIN  (F16 storage) how the line pairs wait for the A_hat chain on the
 *                        second stream: 1 = the first vertical pair waits for the whole chain;
 *                        2 = line pair p waits for A_hat pass p only, so that the later passes
 *                        run beside the first line pairs; 0 (automatic) = 2 where an A_hat pass
 *                        block (4 warps, 48 bytes per position of the longest line) needs at
 *                        most 64 KB of shared memory and so fits beside the line pairs' blocks
 *                        (1280x384x128: step 0.532 -> 0.519 ms), else 1 (1920x1080x256 with 2:
 *                        5.73 -> 6.10 ms, the passes waiting for free SMs). The maps do not
 *                        depend on it
 * A value a launch cannot use (too many threads or too much shared memory) makes the next
 * call fail with ZNCC_EUNSUPPORTED. Unknown keys give ZNCC_EINVAL. */
typedef enum {
    ZNCC_TUNE_ROW_MINB2 = 1,
    ZNCC_TUNE_ROW_SPB = 2,
    ZNCC_TUNE_H_TQ = 3,
    ZNCC_TUNE_V_TQ = 4,
    ZNCC_TUNE_AHAT_SMS = 5,
    ZNCC_TUNE_PLANE = 6,
    ZNCC_TUNE_PLANE_CS = 7,
    ZNCC_TUNE_ROW_LOADS = 8,
    ZNCC_TUNE_V_LPC = 9,
    ZNCC_TUNE_LINE_LOADS = 10,
    ZNCC_TUNE_WAIT_DRILL = 11,
    ZNCC_TUNE_AHAT_JOIN = 12
} zncc_tune_key;
zncc_status zncc_set_tuning(zncc_ctx* ctx, int key, int value);

/* Number of kernels this library has launched in this process (all contexts). */
uint64_t zncc_kernel_launch_count(void);

/* Per-kernel timing, for measurement. While enabled, every kernel the context launches is
 * bracketed by two CUDA events recorded on the context's stream (events are created on
 * demand and reused). */
zncc_status zncc_profile_enable(zncc_ctx* ctx, int enable);

/* Synchronizes the context's stream, then writes for each kernel kind k < nkinds the summed
 * device time in milliseconds (total_ms[k]) and the number of launches (launches[k]) since
 * the previous read, and forgets them. Kinds are named by zncc_profile_kind_name. */
zncc_status zncc_profile_read(zncc_ctx* ctx, double* total_ms, uint64_t* launches, int nkinds);

/* Number of kernel kinds, and the static name of kind k (NULL when out of range). */
int zncc_profile_nkinds(void);
const char* zncc_profile_kind_name(int kind);

#ifdef __cplusplus
}
#endif

#endif /* ZNCC_H_ */
