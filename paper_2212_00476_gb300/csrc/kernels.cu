// kernels.cu -- window statistics, DT coefficients, DT line pairs and WTA kernels.
#include <algorithm>
#include <mutex>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "zncc_row.cuh"

namespace zncc {

namespace {
struct SmemAttr {
    int dev;
    const void* fn;
    size_t smem;
};
std::mutex g_smem_attr_mu;
std::vector<SmemAttr> g_smem_attr;
}  // namespace

cudaError_t set_max_smem(const void* fn, size_t smem) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_smem_attr_mu);
    SmemAttr* rec = nullptr;
    for (SmemAttr& a : g_smem_attr)
        if (a.dev == dev && a.fn == fn) rec = &a;
    if (rec && rec->smem >= smem) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (rec) rec->smem = smem;
    else g_smem_attr.push_back(SmemAttr{dev, fn, smem});
    return cudaSuccess;
}

void forget_smem_attributes() {
    std::lock_guard<std::mutex> lk(g_smem_attr_mu);
    g_smem_attr.clear();
}

void launch_config(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, dim3 grid, dim3 block, size_t smem,
                   cudaStream_t st, int cluster) {
    cfg = cudaLaunchConfig_t{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.numAttrs = 1;
    if (cluster > 1) {
        attr[1].id = cudaLaunchAttributeClusterDimension;
        attr[1].val.clusterDim.x = cluster;
        attr[1].val.clusterDim.y = 1;
        attr[1].val.clusterDim.z = 1;
        cfg.numAttrs = 2;
    }
    cfg.attrs = attr;
}

// ---------------------------------------------------------------------------------------
// Window statistics (Sec. IV-B-1, Eq. (sum1), Method 1 made separable): block per row y;
// column sums of the 2r+1 clamped rows for every column the row's windows touch, then the
// horizontal window sum of those. S, Q exact int32; inv_sigma = rsqrtf(n Q - S^2) (within 2
// ulp of 1/sqrt) or 0; the cost kernel computes its statistics the same way, bit for bit.
// n Q - S^2 < 2^31 for every window side <= 15 (its maximum is n^2 * 127.5^2), so it is
// computed modulo 2^32 in unsigned arithmetic even where n Q alone would not fit.
// `packed` receives (S, inv_sigma bits) per centre for the cost kernel.
__global__ void k_window_stats(const uint8_t* __restrict__ img, int pitch, int W, int H, int r,
                               int x_begin, int nx, int* __restrict__ S, int* __restrict__ Q,
                               float* __restrict__ isig, int2* __restrict__ packed) {
    extern __shared__ int sm_stats[];
    const int y = blockIdx.x;
    const int ncol = nx + 2 * r;
    int* cs = sm_stats;
    int* cq = sm_stats + ncol;
    for (int t = threadIdx.x; t < ncol; t += blockDim.x) {
        const int xc = min(max(x_begin - r + t, 0), W - 1);
        int s = 0, q = 0;
        for (int j = -r; j <= r; ++j) {
            const int p = img[(size_t)min(max(y + j, 0), H - 1) * pitch + xc];
            s += p;
            q += p * p;
        }
        cs[t] = s;
        cq[t] = q;
    }
    __syncthreads();
    const unsigned n = (unsigned)((2 * r + 1) * (2 * r + 1));
    for (int t = threadIdx.x; t < nx; t += blockDim.x) {
        int s = 0, q = 0;
        for (int i = 0; i <= 2 * r; ++i) {
            s += cs[t + i];
            q += cq[t + i];
        }
        const size_t o = (size_t)y * nx + t;
        const int var = (int)(n * (unsigned)q - (unsigned)s * (unsigned)s);
        const float is = var > 0 ? rsqrtf((float)var) : 0.0f;
        if (S) S[o] = s;
        if (Q) Q[o] = q;
        if (isig) isig[o] = is;
        if (packed) packed[o] = make_int2(s, __float_as_int(is));
    }
}

cudaError_t launch_window_stats(const uint8_t* img, int pitch, int W, int H, int r, int x_begin,
                                int nx, int* S, int* Q, float* isig, int2* packed, cudaStream_t st) {
    const size_t smem = 2 * sizeof(int) * (size_t)(nx + 2 * r);
    k_window_stats<<<H, 256, smem, st>>>(img, pitch, W, H, r, x_begin, nx, S, Q, isig, packed);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// DT coefficients (Sec. III-B, Eq. (11)). The weight of the step between two neighbouring
// pixels p, q is K * exp(-|G(p) - G(q)| / sigma_r), G = guide / 255. For each line (rows for
// the horizontal passes, columns for the vertical ones) and position p, with w(p) the weight
// of the step p-1 -> p (0 at p = 0 and past the line end):
//   (w(p), prod_{j=c..p} w(j), w(p+1), prod_{j=p..c+15} w(j+1)),  c = chunk start (16 | c).
// coefH is [H][W]; coefV is [W][H] (a column is contiguous). One thread per position; the
// 16 positions of a chunk are 16 consecutive lanes, whose products are shuffle scans.
__global__ void k_dt_coef(const __grid_constant__ CoefBatch b) {
    griddep_wait();
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int pi = 0;
    while (pi + 1 < b.npairs && gid >= b.p[pi + 1].thread0) ++pi;
    const CoefArgs& a = b.p[pi];
    const int W = a.W, H = a.H;
    const int nchH = (W + kL - 1) / kL, nchV = (H + kL - 1) / kL;
    const long long local = gid - a.thread0;
    int chunk = (int)(local / kL);
    const int i = (int)(local & (kL - 1));
    const bool horiz = chunk < H * nchH;
    if (!horiz) chunk -= H * nchH;
    const bool live = gid < b.total_threads && (horiz || chunk < W * nchV);
    const int n = horiz ? W : H;
    const int nchl = horiz ? nchH : nchV;
    const int line = live ? chunk / nchl : 0;
    const int p = (live ? chunk - line * nchl : 0) * kL + i;
    auto pix = [&](int q) -> int {
        return horiz ? a.guide[(size_t)line * a.pitch + q] : a.guide[(size_t)q * a.pitch + line];
    };
    auto weight = [&](int q) -> float {    // the step q-1 -> q
        return (live && q >= 1 && q < n) ? a.K * expf(-fabsf((float)(pix(q) - pix(q - 1))) * a.inv_sr255) : 0.0f;
    };
    const float w = weight(p);
    float wn = __shfl_down_sync(kFull, w, 1, kL);
    if (i == kL - 1) wn = weight(p + 1);
    float A = w, B = wn;
#pragma unroll
    for (int off = 1; off < kL; off <<= 1) {
        const float a2 = __shfl_up_sync(kFull, A, off, kL);
        const float b2 = __shfl_down_sync(kFull, B, off, kL);
        if (i >= off) A *= a2;
        if (i + off < kL) B *= b2;
    }
    if (live && p < n) {
        float4* out = horiz ? a.coefH + (size_t)line * W : a.coefV + (size_t)line * H;
        out[p] = make_float4(w, A, wn, B);
    }
}

// ---------------------------------------------------------------------------------------
// A_hat pass pair: the scaled pair of Eqs. (3)-(6) on one plane, one warp per line. The warp
// first stages the line's weights and inputs in shared memory, 16 positions a lane per
// round with every load of the round in flight at once; then lane l takes positions
// [l*seg, (l+1)*seg) (seg odd, so that the lanes' sweeps fall on distinct banks): a sweep
// with zero carry gives the lane's affine map x -> P x + u (P the product of its weights), a
// warp scan composes the maps, and a second sweep from the true carry computes the values;
// the backward pass likewise from the right.
constexpr int kAhatWarps = 4;
constexpr int kAhatArrays = 3;      // per line: weights, inputs, values

__global__ void __launch_bounds__(32 * kAhatWarps) k_ahat_pair(const __grid_constant__ AhatBatch b) {
    extern __shared__ float ahat_smem[];
    griddep_wait();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int gline = blockIdx.x * kAhatWarps + wib;
    if (gline >= b.total_lines) return;
    int pi = 0;
    while (pi + 1 < b.npairs && gline >= b.p[pi + 1].line0) ++pi;
    const AhatArgs& a = b.p[pi];
    const int line = gline - a.line0;
    const bool horiz = b.horiz != 0;
    const int W = a.W, n = horiz ? a.W : a.H;
    const uint8_t* g = a.guide + (horiz ? (size_t)line * a.pitch : (size_t)line);
    const size_t gstep = horiz ? 1 : (size_t)a.pitch;             // guide step along the line
    const float* ain = a.ain ? a.ain + (horiz ? (size_t)line * W : (size_t)line) : nullptr;
    const size_t astep = horiz ? 1 : (size_t)W;                   // plane step along the line
    float* ws = ahat_smem + (size_t)wib * kAhatArrays * b.nmax;   // w(q): the step q-1 -> q
    float* xs = ws + b.nmax;                                      // input
    float* fs = xs + b.nmax;                                      // forward values, then A_hat
    constexpr int kR = 16;
    for (int base = 0; base < n; base += 32 * kR) {
        int gc[kR], gp[kR];
        float in[kR];
#pragma unroll
        for (int k = 0; k < kR; ++k) {
            const int q = base + k * 32 + lane;
            const bool ok = q < n;
            gc[k] = ok ? g[(size_t)q * gstep] : 0;
            gp[k] = ok && q >= 1 ? g[(size_t)(q - 1) * gstep] : 0;
            in[k] = ok && ain ? ain[(size_t)q * astep] : 1.0f;
        }
#pragma unroll
        for (int k = 0; k < kR; ++k) {
            const int q = base + k * 32 + lane;
            if (q < n) {    // the expression of k_dt_coef
                ws[q] = q >= 1 ? b.K * expf(-fabsf((float)(gc[k] - gp[k])) * b.inv_sr255) : 0.0f;
                xs[q] = in[k];
            }
        }
    }
    __syncwarp();
    const int seg = ((n + 31) / 32) | 1;
    const int p0 = min(n, lane * seg), p1 = min(n, p0 + seg);

    // forward: f(p) = c(p) + w(p) f(p-1)
    float P = 1.0f, u = 0.0f;
#pragma unroll 4
    for (int q = p0; q < p1; ++q) {
        const float w = ws[q];
        u = fmaf(w, u, xs[q]);
        P *= w;
    }
    for (int off = 1; off < 32; off <<= 1) {
        const float P2 = __shfl_up_sync(kFull, P, off), u2 = __shfl_up_sync(kFull, u, off);
        if (lane >= off) {
            u = fmaf(P, u2, u);
            P *= P2;
        }
    }
    float x = __shfl_up_sync(kFull, u, 1);
    if (lane == 0) x = 0.0f;
#pragma unroll 4
    for (int q = p0; q < p1; ++q) {
        x = fmaf(ws[q], x, xs[q]);
        fs[q] = x;
    }
    // backward: h(p) = f(p) + w(p+1) h(p+1); w(n) = 0 (the weights are never written again)
    P = 1.0f;
    u = 0.0f;
#pragma unroll 4
    for (int q = p1 - 1; q >= p0; --q) {
        const float w = q + 1 < n ? ws[q + 1] : 0.0f;
        u = fmaf(w, u, fs[q]);
        P *= w;
    }
    for (int off = 1; off < 32; off <<= 1) {
        const float P2 = __shfl_down_sync(kFull, P, off), u2 = __shfl_down_sync(kFull, u, off);
        if (lane + off < 32) {
            u = fmaf(P, u2, u);
            P *= P2;
        }
    }
    x = __shfl_down_sync(kFull, u, 1);
    if (lane == 31) x = 0.0f;
#pragma unroll 4
    for (int q = p1 - 1; q >= p0; --q) {
        x = fmaf(q + 1 < n ? ws[q + 1] : 0.0f, x, fs[q]);
        fs[q] = b.s2 * x;
    }
    __syncwarp();
    float* aout = a.aout + (horiz ? (size_t)line * W : (size_t)line);
    float2* mm = a.mulmap ? a.mulmap + (size_t)line * n : nullptr;
#pragma unroll 8
    for (int q = lane; q < n; q += 32) {
        const float A = fs[q];
        aout[(size_t)q * astep] = A;
        if (mm) mm[q] = make_float2(a.in_mul ? b.xscale * xs[q] : 1.0f, b.yscale / A);
    }
    griddep_launch_dependents();
}

size_t ahat_pass_smem_bytes(int nmax) { return (size_t)kAhatWarps * kAhatArrays * nmax * sizeof(float); }

cudaError_t launch_ahat_pair(const AhatBatch& b, cudaStream_t st) {
    const size_t smem = ahat_pass_smem_bytes(b.nmax);
    cudaError_t e = set_max_smem((const void*)k_ahat_pair, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[2];
    launch_config(cfg, attr, dim3((b.total_lines + kAhatWarps - 1) / kAhatWarps), dim3(32 * kAhatWarps), smem, st, 1);
    return cudaLaunchKernelEx(&cfg, k_ahat_pair, b);
}

// The column coefficients alone (coefV), coalesced: thread (column x, chunk c) computes the
// chunk's 16 positions in order (guide reads of one row are consecutive across the warp's
// columns), and the warp writes its 32 columns x 16 positions through shared memory so that
// each column's 256 contiguous bytes go out together. Values as in k_dt_coef.
constexpr int kColWarps = 4;

__global__ void __launch_bounds__(32 * kColWarps) k_dt_coef_cols(const __grid_constant__ CoefBatch b) {
    __shared__ float4 tile[kColWarps][32][kL + 1];
    griddep_wait();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int pi = 0;
    while (pi + 1 < b.npairs && (long long)blockIdx.x >= b.p[pi + 1].thread0) ++pi;
    const CoefArgs& a = b.p[pi];
    const int W = a.W, H = a.H;
    const int nchV = (H + kL - 1) / kL, ncg = (nchV + kColWarps - 1) / kColWarps;
    const int local = (int)(blockIdx.x - a.thread0);
    const int x0 = (local / ncg) * 32, c = (local % ncg) * kColWarps + wib;
    if (c >= nchV) return;                  // whole warps
    const int x = x0 + lane, p0 = c * kL;
    const bool live = x < W;
    const uint8_t* g = a.guide + (live ? x : 0);
    int gv[kL + 2];                         // guide at p0 - 1 .. p0 + 16
#pragma unroll
    for (int i = 0; i < kL + 2; ++i) {
        const int p = p0 - 1 + i;
        gv[i] = live && p >= 0 && p < H ? g[(size_t)p * a.pitch] : 0;
    }
    float w[kL + 1];                        // w(p0 + i): the step p0 + i - 1 -> p0 + i
#pragma unroll
    for (int i = 0; i <= kL; ++i) {
        const int q = p0 + i;
        w[i] = (q >= 1 && q < H) ? a.K * expf(-fabsf((float)(gv[i + 1] - gv[i])) * a.inv_sr255) : 0.0f;
    }
    float A = 1.0f, B[kL];
    B[kL - 1] = w[kL];
#pragma unroll
    for (int i = kL - 2; i >= 0; --i) B[i] = B[i + 1] * w[i + 1];
#pragma unroll
    for (int i = 0; i < kL; ++i) {
        A = i == 0 ? w[0] : A * w[i];
        tile[wib][lane][i] = make_float4(w[i], A, w[i + 1], B[i]);
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 16; ++k) {          // columns 2k, 2k+1: 16 lanes each
        const int col = 2 * k + (lane >> 4), i = lane & (kL - 1);
        if (x0 + col < W && p0 + i < H) a.coefV[(size_t)(x0 + col) * H + p0 + i] = tile[wib][col][i];
    }
}

long long dt_coef_col_blocks(int W, int H) {
    const int nchV = (H + kL - 1) / kL;
    return (long long)((W + 31) / 32) * ((nchV + kColWarps - 1) / kColWarps);
}

cudaError_t launch_dt_coef_cols(const CoefBatch& b, cudaStream_t st) {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[2];
    launch_config(cfg, attr, dim3((unsigned)b.total_threads), dim3(32 * kColWarps), 0, st, 1);
    return cudaLaunchKernelEx(&cfg, k_dt_coef_cols, b);
}

long long dt_coef_threads(int W, int H) {
    return (long long)kL * ((long long)H * ((W + kL - 1) / kL) + (long long)W * ((H + kL - 1) / kL));
}

cudaError_t launch_dt_coef(const CoefBatch& b, cudaStream_t st) {
    const long long blocks = (b.total_threads + 255) / 256;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[2];
    launch_config(cfg, attr, dim3((unsigned)blocks), dim3(256), 0, st, 1);
    return cudaLaunchKernelEx(&cfg, k_dt_coef, b);
}

// ---------------------------------------------------------------------------------------
// DT line pair (Sec. III-B, Eqs. (3)-(6)): the forward and the backward recursive pass
// along rows (L2R then R2L) or columns (U2D then D2U) of a cost volume, or, for the last
// pair of the chain, folded into a per-pixel running best without writing the volume back
// (Sec. V-C fuses WTA with D2U in the same way).
//
// Work: lines in groups of lpc, each group with nslices disparity slices of 4*tq
// disparities; an item is (group, slice), numbered group-major (FastDT stores: a whole group,
// whose slices are coded against d = 0 of the first). The grid is sized to the
// resident blocks (persistent); block b processes the items [b*per_block, (b+1)*per_block)
// in order, restaging the coefficients when the group changes. A line longer than one block
// can hold at the chosen lanes per chunk spans the CTAs of a thread-block cluster (one line
// per cluster), which exchange their warps' chunk maps through distributed shared memory. With aligned 4-disparity
// groups (async) each thread streams its elements of the next item into shared memory with
// cp.async while the current one is computed, across group boundaries: two staging buffers,
// each refilled (two items ahead) as soon as the forward sweep has consumed it. In Wta mode a
// block keeps a running best over the slices it sees of a line group and merges it into the
// per-pixel keys (atomicMax) when the group or its range ends.
static size_t elem_bytes(int dtype) { return dtype == 0 ? 4 : (dtype == 1 ? 2 : 1); }

size_t line_stage_bytes(int dtype, const LineArgs& a) {
    if (a.async && a.tma) return 2ull * a.lpc * a.nch * line_tma_slot_bytes(a.tq, (int)elem_bytes(dtype));
    return a.async ? 2ull * a.lpc * a.nch * a.tq * kL * (4 * elem_bytes(dtype)) : 0;
}


// Every pair of a launch has the same block shape (tq, nch, lpc, async): the launcher groups
// pairs that way, so the shape and this thread's place in it are read from pair 0 at
// constant offsets of the parameter block; only extents, strides and pointers differ between
// pairs. SINGLE: the launch holds one pair, whose arguments are then all read at constant
// offsets instead of through a dynamic index. CLUSTER: lines span the CTAs of a cluster.
template <typename T, int MODE, bool SINGLE, bool CLUSTER>
__global__ void __launch_bounds__(512) k_line_pair(const __grid_constant__ LineBatch b) {
    extern __shared__ __align__(128) float4 smem4[];
    // (tma) per staging buffer and warp, an mbarrier that the first lanes of the warp's chunks
    // arrive on once per fill (a line is whole warps, so a chunk never straddles two warps)
    __shared__ unsigned long long tbar[2][16];
    // TMA staging: the pairs' flag (the launcher groups pairs by it) and 128-byte aligned buffers
    const bool tma = !CLUSTER && b.p[0].tma != 0 && b.p[0].async != 0 && (smem_addr(smem4) & 127u) == 0;
    if (tma && threadIdx.x < 2 * (blockDim.x >> 5))
        mbar_init(&tbar[threadIdx.x & 1][threadIdx.x >> 1], (unsigned)(32 / b.p[0].tq));
    // (tests) the wait drill: thread 0 waits, bounded, for a phase of an mbarrier that nothing
    // arrives on, records the timeout like a copy that did not land, and goes on; no copy is in
    // flight on that barrier, and the pass computes as without the drill
    __shared__ unsigned long long drill_bar;
    if (b.drill && threadIdx.x == 0) mbar_init(&drill_bar, 1);
    if (tma || b.drill) __syncthreads();
    if (b.drill && threadIdx.x == 0 && !mbar_wait(&drill_bar, 0, kDrillWaitPolls) && b.fault)
        atomicOr(b.fault, kFaultTmaWait);
    griddep_wait();
    auto P = [&](int pi) -> const LineArgs& { return b.p[SINGLE ? 0 : pi]; };
    const int lane = threadIdx.x & 31;
    // A line spans the cs CTAs of a cluster (consecutive blocks), CTA `rank` holding chunks
    // [rank * nch, rank * nch + nch); the cluster's CTAs take the same items in lock step.
    const int cs = CLUSTER ? b.p[0].cs : 1;
    const int rank = CLUSTER ? cluster_rank() : 0;
    const int cid = blockIdx.x / cs, ncl = b.grid / cs;
    const int i0 = (int)((long long)cid * b.total_items / ncl);
    const int i1 = (int)((long long)(cid + 1) * b.total_items / ncl);
    // the block's steps: from the first step of item i0 to the first step of item i1
    auto step_of_item = [&](int item) -> int {
        if (item >= b.total_items) return b.total_steps;
        int q = 0;
        if (!SINGLE)
            while (item >= b.p[q].item0 + b.p[q].nitems) ++q;
        const LineArgs& a = P(q);
        const int spi = a.nsteps / a.nitems;
        return a.step0 + (item - a.item0) * spi;
    };
    const int s0 = step_of_item(i0), s1 = step_of_item(i1);

    // block shape (shared by the launch's pairs) and this thread's place in it
    const int tq = b.p[0].tq, nch = b.p[0].nch, lpc = b.p[0].lpc;
    const bool async = b.p[0].async != 0;
    const int per_line = nch * tq, nwl = per_line >> 5, ds = kG * tq;
    const int nwl_all = cs * nwl;                   // warps of a whole line
    const bool active = (int)threadIdx.x < lpc * per_line;
    const int li = active ? threadIdx.x / per_line : 0;
    const int tl = active ? threadIdx.x - li * per_line : 0;
    const int k = tl / tq, dq = tl - k * tq, wl = tl >> 5;
    const int kg = rank * nch + k;                  // chunk within the whole line
    const int pos0 = rank * nch * kL;               // first line position of this CTA

    // A cursor over steps: the pair, the line group and the slice of a step, advanced one
    // step at a time.
    struct Cursor {
        int s, pi, g, sl, nslices, ngroups;
        int gseq;                                   // line groups entered since the block's first step
    };
    auto set_pair = [&](Cursor& c) {
        const LineArgs& a = P(c.pi);
        c.nslices = (a.dcount + ds - 1) / ds;
        c.ngroups = a.nsteps / c.nslices;
    };
    auto seek = [&](int s) -> Cursor {          // once per block
        Cursor c;
        c.s = s;
        c.pi = 0;
        if (!SINGLE)
            while (c.pi + 1 < b.npairs && s >= b.p[c.pi].step0 + b.p[c.pi].nsteps) ++c.pi;
        set_pair(c);
        const int ls = s - P(c.pi).step0;
        c.g = ls / c.nslices;
        c.sl = ls - c.g * c.nslices;
        c.gseq = 0;
        return c;
    };
    auto advance = [&](Cursor& c) {
        ++c.s;
        if (++c.sl == c.nslices) {
            c.sl = 0;
            ++c.gseq;
            if (++c.g == c.ngroups && !SINGLE && c.pi + 1 < b.npairs) {
                c.g = 0;
                ++c.pi;
                set_pair(c);
            }
        }
    };
    auto line_of = [&](const Cursor& c) { return c.g * lpc + li; };
    auto elem0 = [&](const LineArgs& a, const Cursor& c) -> size_t {   // the chunk's first group
        return (size_t)line_of(c) * a.line_stride + (size_t)(kg * kL) * a.elem_stride + c.sl * ds + dq * kG;
    };
    // staging buffers: [2][kL][threads] groups of 4 entries: position i of this thread's
    // chunk at stage_at(buf) + i * sstride (consecutive threads, consecutive groups). With TMA
    // a buffer is [lines][chunks] slots of line_tma_slot_bytes, one box of kL + G - 1 positions
    // x ds entries per (line, chunk), G = the chunks whose lanes share a shared-memory wavefront
    // of the reads below: chunk k's box starts k mod G positions early, so that the G chunks
    // read distinct banks; the thread's position i is at stage_at(buf) + (i + k mod G) * ds.
    const int nthr = lpc * per_line;
    const int sstride = tma ? ds : nthr * 4;
    const int tma_g = line_tma_chunks_per_wavefront(tq, (int)sizeof(T));
    const int tma_slot = line_tma_slot_bytes(tq, (int)sizeof(T)) / (int)sizeof(T);     // entries
    T* const stage0 = reinterpret_cast<T*>(smem4) +
                      (tma ? (size_t)(li * nch + k) * tma_slot + (k % tma_g) * ds + dq * kG
                           : (size_t)threadIdx.x * 4);
    const size_t buf_entries = tma ? (size_t)lpc * nch * tma_slot : (size_t)kL * nthr * 4;
    auto stage_at = [&](int buf) -> T* { return stage0 + (size_t)buf * buf_entries; };
    // shared memory: [stage][coefficients: 1 or 2 buffers][multipliers: as many][scan
    // buffers], the per-position arrays [lpc][nch][kCS], chunk-major. Without A_hat scaling
    // (has_mul false) there are no multipliers; with co_async the arrays of a line group are
    // streamed into the other buffer by cp.async along with the volume of its first step.
    const bool has_mul = b.p[0].mulmap != nullptr;
    const bool co_async = b.co_async != 0;
    const int arr = lpc * nch * kCS;
    const int nbuf = co_async ? 2 : 1;
    constexpr bool kFast = std::is_same<T, uint8_t>::value;          // FastDT codes
    float4* co_all = reinterpret_cast<float4*>(reinterpret_cast<char*>(smem4) + b.stage_bytes);
    float2* mul_all = reinterpret_cast<float2*>(co_all + nbuf * arr);
    // (FastDT store) the reference value v(d_arb = 0) of each position of the group's lines
    float* ref_all = reinterpret_cast<float*>(mul_all + (has_mul ? nbuf * arr : 0));
    float4* sb_all = reinterpret_cast<float4*>(ref_all + (kFast && MODE == kLineStore ? arr : 0));
    float* sa_all = reinterpret_cast<float*>(sb_all + lpc * 2 * nwl_all * tq);
    const int cthr = (li * nch + k) * kCS;                         // this thread's chunk
    float4* sb = sb_all + li * 2 * nwl_all * tq;
    float* sa = sa_all + li * 2 * nwl_all * tq;

    // the coefficients (and multipliers) of the line group at cursor pc into buffer cbuf
    auto prefetch_coef = [&](const Cursor& pc, int cbuf) {
        const LineArgs& a = P(pc.pi);
        float4* dst = co_all + cbuf * arr;
        float2* mdst = mul_all + cbuf * arr;
        for (int l2 = 0; l2 < lpc; ++l2) {
            const int ln = pc.g * lpc + l2;
            for (int t = threadIdx.x; t < nch * kL; t += blockDim.x) {
                const int gp = pos0 + t;
                const bool in = ln < a.nlines && gp < a.n;
                cp_async<16>(dst + l2 * nch * kCS + cpos(t),
                             in ? a.coef + (size_t)ln * a.coef_line_stride + gp : a.coef, in);
                if (has_mul)
                    cp_async<8>(mdst + l2 * nch * kCS + cpos(t),
                                in ? a.mulmap + (size_t)ln * a.n + gp : a.mulmap, in);
            }
        }
    };
    // prefetch of the step at cursor pc into stage buffer buf. With vec the entries per pixel
    // are a multiple of 4, so a group with any valid disparity lies whole inside the volume;
    // its entries past dcount are never stored or compared. The first step of a line group
    // also brings the group's coefficients (co_async).
    auto prefetch = [&](const Cursor& pc, int buf) {
        if (co_async && pc.s < s1 && (pc.sl == 0 || pc.s == s0)) prefetch_coef(pc, pc.gseq & 1);
        if (!tma && async && pc.s < s1 && active) {
            const LineArgs& a = P(pc.pi);
            const T* src = a.src ? reinterpret_cast<const T*>(a.src) : reinterpret_cast<const T*>(a.vol);
            const bool ok = line_of(pc) < a.nlines && pc.sl * ds + dq * kG < a.dcount;
            const T* q = src + (ok ? elem0(a, pc) : 0);
            const long long es = a.elem_stride;
            const int npos = a.n - kg * kL;
            T* st = stage_at(buf);
            if (ok && npos >= kL) {                 // a whole chunk: no per-position test
#pragma unroll
                for (int i = 0; i < kL; ++i) cp_async<4 * sizeof(T)>(st + i * sstride, q + (size_t)i * es, true);
            } else {
#pragma unroll
                for (int i = 0; i < kL; ++i) {
                    const bool valid = ok && i < npos;
                    cp_async<4 * sizeof(T)>(st + i * sstride, valid ? q + (size_t)i * es : src, valid);
                }
            }
        }
        cp_async_commit();
    };
    // (tma) the step at cursor pc into buffer buf: the first lane of each chunk copies the
    // chunk's box into the start of its slot (lines past the pass and positions or entries past
    // the line read as zero). A slot start that is not 128-byte aligned (which the layout above
    // rules out) is recorded as a fault and not copied to.
    auto prefetch_tma = [&](const Cursor& pc, int buf) {
        if (!tma || !active || dq != 0 || pc.s >= s1) return;
        const LineArgs& a = P(pc.pi);
        const CUtensorMap* m = &b.tmap[SINGLE ? 0 : pc.pi];
        const int d0 = pc.sl * ds, p0 = kg * kL - k % tma_g, line = line_of(pc);
        T* const slot = reinterpret_cast<T*>(smem4) + (size_t)buf * buf_entries + (size_t)(li * nch + k) * tma_slot;
        unsigned long long* bar = &tbar[buf][threadIdx.x >> 5];
        if (smem_addr(slot) & 127u) {
            if (b.fault) atomicOr(b.fault, kFaultTmaAlign);
            mbar_arrive(bar);
            return;
        }
        fence_proxy_async_smem();                   // this warp's reads of the slot, then the copy
        mbar_expect_tx(bar, (unsigned)((kL + tma_g - 1) * ds * sizeof(T)));
        if (a.horiz) tma_load_3d(slot, m, d0, p0, line, bar);
        else tma_load_3d(slot, m, d0, line, p0, bar);
    };
    Cursor o = seek(s0);
    Cursor pf = o;                              // two steps ahead of o
    prefetch(pf, 0);
    prefetch_tma(pf, 0);
    advance(pf);
    prefetch(pf, 1);
    prefetch_tma(pf, 1);
    advance(pf);

    if (cs > 1) cluster_sync_all();                 // every CTA of the cluster has started

    WtaRegs wr;
    int cur_pi = -1, cur_g = -1;
    for (int n_s = 0; o.s < s1; advance(o), ++n_s) {
        const int pi = o.pi;
        const LineArgs& a = P(pi);
        const int line = line_of(o);
        const bool line_ok = active && line < a.nlines;
        if (o.s + 1 == s1) griddep_launch_dependents();             // this block's last step

        cp_async_wait<1>();                                            // this step's copies landed
        if (pi != cur_pi || o.g != cur_g) {     // a new line group: its coefficients (and multipliers)
            __syncthreads();
            if (!co_async) {
                for (int l2 = 0; l2 < lpc; ++l2) {
                    const int ln = o.g * lpc + l2;
                    const bool ok = ln < a.nlines;
                    for (int t = threadIdx.x; t < nch * kL; t += blockDim.x) {
                        const int gp = pos0 + t;
                        const bool in = ok && gp < a.n;
                        co_all[l2 * nch * kCS + cpos(t)] =
                            in ? __ldg(a.coef + (size_t)ln * a.coef_line_stride + gp) : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
            }
            if (has_mul && !co_async) {
                for (int l2 = 0; l2 < lpc; ++l2) {
                    const int ln = o.g * lpc + l2;
                    const bool ok = ln < a.nlines;
                    for (int t = threadIdx.x; t < nch * kL; t += blockDim.x) {
                        const int gp = pos0 + t;
                        mul_all[l2 * nch * kCS + cpos(t)] =
                            ok && gp < a.n ? __ldg(a.mulmap + (size_t)ln * a.n + gp) : make_float2(0.f, 0.f);
                    }
                }
            }
            if constexpr (MODE == kLineWta) wr.reset();
            __syncthreads();
            cur_pi = pi;
            cur_g = o.g;
        }
        const int cb = co_async ? (o.gseq & 1) * arr : 0;
        const float4* co = co_all + cb + cthr;                       // this thread's chunk
        const float2* mul = has_mul ? mul_all + cb + cthr : nullptr;
        const int dl = o.sl * ds + dq * kG;                        // entry of d_first
        const int nvalid = max(0, min(4, a.dcount - dl));
        const bool any = line_ok && nvalid > 0;
        const int npos = a.n - kg * kL;
        T* vol = reinterpret_cast<T*>(a.vol);
        float v[kL][4];
        if (a.src_ones) {
#pragma unroll
            for (int i = 0; i < kL; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) v[i][j] = (any && i < npos && j < nvalid) ? 1.0f : 0.0f;
        } else if (async) {
            if (tma && active) {
                // this warp's boxes of the step (bounded wait; a timeout is recorded, then waited
                // for once more)
                unsigned long long* bar = &tbar[n_s & 1][threadIdx.x >> 5];
                const unsigned par = (unsigned)(n_s >> 1) & 1u;
                if (!mbar_wait(bar, par, kBulkWaitPolls)) {
                    if (b.fault) atomicOr(b.fault, kFaultTmaWait);
                    mbar_wait(bar, par, kBulkWaitPolls);
                }
            }
            const T* st = stage_at(n_s & 1);
#pragma unroll
            for (int i = 0; i < kL; ++i) lds4(st + i * sstride, v[i]);
            if (tma) {
                __syncwarp();                       // the chunk's lanes have read its slot
                prefetch_tma(pf, n_s & 1);          // two steps ahead, into the same buffer
            }
        } else {
            const T* src = a.src ? reinterpret_cast<const T*>(a.src) : vol;
            const T* q = src + (line_ok ? elem0(a, o) : 0);
#pragma unroll
            for (int i = 0; i < kL; ++i) {
                if (any && i < npos) ld4(q, nvalid, a.vec != 0, v[i]);
                else v[i][0] = v[i][1] = v[i][2] = v[i][3] = 0.0f;
                q += a.elem_stride;
            }
        }
        if (has_mul && active) {         // (FastDT codes always have multipliers)
#pragma unroll
            for (int i = 0; i < kL; ++i) mul4<true>(mul[i].x, v[i]);
        }
        // the staging buffer is free once the forward sweep has read it: refill it two ahead
        dt_pair<MODE != kLineWta, true>(v, co, tq, dq, lane, rank * nwl + wl, nwl_all, sa, sb, a.s2, mul,
                [&]() {
                    prefetch(pf, n_s & 1);
                    advance(pf);
                }, active, cs);
        if constexpr (MODE == kLineWta) {
            if (active) wr.fold(v, nvalid, a.d_base + dl);
            // at the group's last slice, or the block's last step, merge this block's best
            if ((o.sl == o.nslices - 1 || o.s + 1 == s1) && active) {
                wr.merge(tq, lane, [&](int i, float best, int bd) {
                    const int pos = kg * kL + i;
                    if (line_ok && pos < a.n) {
                        const size_t pix = (size_t)line * a.pix_line + (size_t)pos * a.pix_pos;
                        atomicMax(a.keys + pix, wta_key(best, bd));
                    }
                });
            }
        } else if constexpr (kFast) {
            // near-zero-mean codes against d_arb = 0, held by lane dq 0 in the group's first
            // slice (a block processes whole line groups, slices in order)
            if (o.sl == 0) {
                if (dq == 0 && active)
#pragma unroll
                    for (int i = 0; i < kL; ++i) ref_all[cthr + i] = v[i][0];
                __syncthreads();
            }
            T* q = vol + (line_ok ? elem0(a, o) : 0);
            const long long es = a.elem_stride;
#pragma unroll
            for (int i = 0; i < kL; ++i)
                if (any && i < npos)
                    *reinterpret_cast<unsigned*>(q + (size_t)i * es) = fastdt_pack(v[i], ref_all[cthr + i], nvalid);
        } else {
            T* q = vol + (line_ok ? elem0(a, o) : 0);
            const long long es = a.elem_stride;
            if (any && npos >= kL && nvalid == 4 && a.vec) {     // a whole chunk of whole groups
#pragma unroll
                for (int i = 0; i < kL; ++i) st4(q + (size_t)i * es, 4, true, v[i]);
            } else {
#pragma unroll
                for (int i = 0; i < kL; ++i)
                    if (any && i < npos) st4(q + (size_t)i * es, nvalid, a.vec != 0, v[i]);
            }
        }
    }
    cp_async_wait<0>();
    if (cs > 1) cluster_sync_all();                 // no CTA leaves while others may store to it
}

bool line_coef_async(const LineArgs& a) {
    const int nslices = (a.dcount + kG * a.tq - 1) / (kG * a.tq);
    return nslices >= 2;
}

size_t line_pair_smem_bytes(int mode, int dtype, const LineArgs& a, bool co_async) {
    const int nwl_all = a.cs * a.nch * a.tq / 32;
    const size_t per_pos = (16ull + (a.mulmap ? 8ull : 0ull)) * (co_async ? 2 : 1) +
                           (dtype == 2 && mode == kLineStore ? 4ull : 0ull);
    return line_stage_bytes(dtype, a) + (size_t)a.lpc * (per_pos * a.nch * kCS + dt_scan_bytes(nwl_all, a.tq));
}

// The multipliers of the last pass pair (its result is not stored): (xscale * ain, or 1; s2).
__global__ void k_mulmap(const float* __restrict__ ain, float xscale, float s2, int W, int H, int horiz,
                         float2* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)W * H) return;
    const int n = horiz ? W : H;
    const int line = (int)(i / n), pos = (int)(i - (long long)line * n);
    const size_t pix = horiz ? (size_t)line * W + pos : (size_t)pos * W + line;
    out[i] = make_float2(ain ? xscale * ain[pix] : 1.0f, s2);
}

cudaError_t launch_mulmap(const float* ain, float xscale, float s2, int W, int H, bool horiz, float2* out,
                          cudaStream_t st) {
    const long long n = (long long)W * H;
    k_mulmap<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ain, xscale, s2, W, H, horiz ? 1 : 0, out);
    return cudaGetLastError();
}

// The FastDT code of each 16-bit value and the value it decodes to (Sec. IV-C), four values a
// thread through the packing and unpacking of the DT kernels.
__global__ void k_fastdt_codec(const int16_t* __restrict__ values, int n, uint8_t* __restrict__ codes,
                               int16_t* __restrict__ decoded) {
    const long long i0 = 4ll * ((long long)blockIdx.x * blockDim.x + threadIdx.x);
    if (i0 >= n) return;
    const int nvalid = (int)min(4ll, n - i0);
    int E[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) E[j] = j < nvalid ? (int)values[i0 + j] : 0;
    const unsigned word = fastdt_pack_codes(E, nvalid);
    float o[4];
    fastdt_unpack(word, o);
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (j < nvalid) {
            if (codes) codes[i0 + j] = (uint8_t)(word >> (8 * j));
            if (decoded) decoded[i0 + j] = (int16_t)(-(int)o[j]);
        }
}

cudaError_t launch_fastdt_codec(const int16_t* values, int n, uint8_t* codes, int16_t* decoded, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int threads = (n + 3) / 4;
    k_fastdt_codec<<<(threads + 255) / 256, 256, 0, st>>>(values, n, codes, decoded);
    return cudaGetLastError();
}

template <bool SINGLE, bool CLUSTER>
static void (*line_pair_fn_t(int mode, int dtype))(LineBatch) {
    if (mode == kLineStore)
        return dtype == 0 ? k_line_pair<float, kLineStore, SINGLE, CLUSTER>
                          : dtype == 1 ? k_line_pair<__half, kLineStore, SINGLE, CLUSTER>
                                       : k_line_pair<uint8_t, kLineStore, SINGLE, CLUSTER>;
    return dtype == 0 ? k_line_pair<float, kLineWta, SINGLE, CLUSTER>
                      : dtype == 1 ? k_line_pair<__half, kLineWta, SINGLE, CLUSTER>
                                   : k_line_pair<uint8_t, kLineWta, SINGLE, CLUSTER>;
}

static void (*line_pair_fn(int mode, int dtype, bool single, bool cluster))(LineBatch) {
    if (cluster) return single ? line_pair_fn_t<true, true>(mode, dtype) : line_pair_fn_t<false, true>(mode, dtype);
    return single ? line_pair_fn_t<true, false>(mode, dtype) : line_pair_fn_t<false, false>(mode, dtype);
}

cudaError_t line_pair_occupancy(int mode, int dtype, int threads, size_t smem, bool single, bool cluster,
                                int* blocks_per_sm) {
    void (*fn)(LineBatch) = line_pair_fn(mode, dtype, single, cluster);
    cudaError_t e = set_max_smem((const void*)fn, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, threads, smem);
}

cudaError_t line_pair_max_clusters(int mode, int dtype, int threads, size_t smem, bool single, int cs,
                                   int* clusters) {
    void (*fn)(LineBatch) = line_pair_fn(mode, dtype, single, true);
    cudaError_t e = set_max_smem((const void*)fn, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(clusters, fn, &cfg);
}

cudaError_t launch_line_batch(const LineBatch& b, int threads, size_t smem, int mode, int dtype,
                              cudaStream_t st) {
    const int cs = b.p[0].cs;
    void (*fn)(LineBatch) = line_pair_fn(mode, dtype, b.npairs == 1, cs > 1);
    cudaError_t e = set_max_smem((const void*)fn, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[2];
    launch_config(cfg, attr, dim3(b.grid), dim3(threads), smem, st, cs);
    return cudaLaunchKernelEx(&cfg, fn, b);
}

// ---------------------------------------------------------------------------------------
// End of the fused WTA: key -> disparity, key -> 0 (ready for the next run).
__global__ void k_wta_finish(const __grid_constant__ WtaFinishBatch b) {
    griddep_wait();
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int pi = 0;
    while (pi + 1 < b.npairs && gid >= b.p[pi + 1].thread0) ++pi;
    const WtaFinishArgs& a = b.p[pi];
    const long long i = gid - a.thread0;
    if (i < a.npix) {
        a.disp[i] = wta_key_disparity(a.keys[i]);
        a.keys[i] = 0ull;
    }
}

cudaError_t launch_wta_finish(const WtaFinishBatch& b, cudaStream_t st) {
    const long long blocks = (b.total_threads + 255) / 256;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[2];
    launch_config(cfg, attr, dim3((unsigned)blocks), dim3(256), 0, st, 1);
    return cudaLaunchKernelEx(&cfg, k_wta_finish, b);
}

// ---------------------------------------------------------------------------------------
// WTA over a stored volume (Sec. III-C, Eq. (WTA1)): one warp per pixel, the smallest d
// among the largest costs.
template <typename T>
__global__ void k_wta_volume(const T* __restrict__ cost, int npix, int D, uint16_t* __restrict__ disp) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= npix) return;
    const T* c = cost + (size_t)warp * D;
    float best = -INFINITY;
    int bd = 0x7FFFFFFF;
    for (int d = lane; d < D; d += 32) {
        const float v = (float)c[d];
        if (v > best) { best = v; bd = d; }
    }
    for (int off = 16; off > 0; off >>= 1) {
        const float ob = __shfl_xor_sync(kFull, best, off);
        const int od = __shfl_xor_sync(kFull, bd, off);
        if (ob > best || (ob == best && od < bd)) { best = ob; bd = od; }
    }
    if (lane == 0) disp[warp] = (uint16_t)(bd == 0x7FFFFFFF ? 0 : bd);
}

cudaError_t launch_wta_volume(const void* cost, int dtype, int W, int H, int D, uint16_t* disp,
                              cudaStream_t st) {
    const int npix = W * H;
    const int blocks = (npix + 7) / 8;
    if (dtype == 0) k_wta_volume<float><<<blocks, 256, 0, st>>>((const float*)cost, npix, D, disp);
    else k_wta_volume<__half><<<blocks, 256, 0, st>>>((const __half*)cost, npix, D, disp);
    return cudaGetLastError();
}

bool zncc_row_bulk_fits_host(int R, int dtype, const RowArgs& a, int nthreads) {
    return zncc_row_bulk_fits(R, dtype, a, nthreads);
}

size_t zncc_row_smem_bytes(int R, int mode, int dtype, const RowArgs& a, int nthreads) {
    return zncc_row_smem(R, mode, dtype, a, nthreads);
}

cudaError_t launch_zncc_row(int R, const RowBatch& b, int threads, size_t smem, int mode, int dtype,
                            cudaStream_t st) {
    switch (R) {
        case 1: return launch_zncc_row_r1(b, threads, smem, mode, dtype, st);
        case 2: return launch_zncc_row_r2(b, threads, smem, mode, dtype, st);
        case 3: return launch_zncc_row_r3(b, threads, smem, mode, dtype, st);
        case 4: return launch_zncc_row_r4(b, threads, smem, mode, dtype, st);
        case 5: return launch_zncc_row_r5(b, threads, smem, mode, dtype, st);
        case 6: return launch_zncc_row_r6(b, threads, smem, mode, dtype, st);
        case 7: return launch_zncc_row_r7(b, threads, smem, mode, dtype, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_zncc_scan(int R, const ScanArgs& a, int dtype, cudaStream_t st) {
    switch (R) {
        case 1: return launch_zncc_scan_r1(a, dtype, st);
        case 2: return launch_zncc_scan_r2(a, dtype, st);
        case 3: return launch_zncc_scan_r3(a, dtype, st);
        case 4: return launch_zncc_scan_r4(a, dtype, st);
        case 5: return launch_zncc_scan_r5(a, dtype, st);
        case 6: return launch_zncc_scan_r6(a, dtype, st);
        case 7: return launch_zncc_scan_r7(a, dtype, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_zncc_mma(int R, const ScanArgs& a, int dtype, cudaStream_t st) {
    switch (R) {
        case 1: return launch_zncc_mma_r1(a, dtype, st);
        case 2: return launch_zncc_mma_r2(a, dtype, st);
        case 3: return launch_zncc_mma_r3(a, dtype, st);
        case 4: return launch_zncc_mma_r4(a, dtype, st);
        case 5: return launch_zncc_mma_r5(a, dtype, st);
        case 6: return launch_zncc_mma_r6(a, dtype, st);
        case 7: return launch_zncc_mma_r7(a, dtype, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t zncc_row_occupancy(int R, int mode, int dtype, int threads, size_t smem, bool minb2,
                               bool single, int* blocks_per_sm) {
    switch (R) {
        case 1: return zncc_row_occupancy_r1(mode, dtype, threads, smem, minb2, single, blocks_per_sm);
        case 2: return zncc_row_occupancy_r2(mode, dtype, threads, smem, minb2, single, blocks_per_sm);
        case 3: return zncc_row_occupancy_r3(mode, dtype, threads, smem, minb2, single, blocks_per_sm);
        case 4: return zncc_row_occupancy_r4(mode, dtype, threads, smem, minb2, single, blocks_per_sm);
        case 5: return zncc_row_occupancy_r5(mode, dtype, threads, smem, minb2, single, blocks_per_sm);
        case 6: return zncc_row_occupancy_r6(mode, dtype, threads, smem, minb2, single, blocks_per_sm);
        case 7: return zncc_row_occupancy_r7(mode, dtype, threads, smem, minb2, single, blocks_per_sm);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace zncc
