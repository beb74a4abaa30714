// kernels.cu -- window statistics, DT edge weights, DT line pairs and WTA kernels.
#include "common.cuh"
#include "kernels.h"
#include "zncc_row.cuh"

namespace zncc {

// ---------------------------------------------------------------------------------------
// Window statistics (Sec. IV-B-1, Eq. (sum1), Method 1 made separable): block per row y;
// column sums of the 2r+1 clamped rows for every column the row's windows touch, then the
// horizontal window sum of those. S, Q exact int32; inv_sigma = 1/sqrt(n Q - S^2) or 0.
// n Q - S^2 < 2^31 for every window side <= 15 (its maximum is n^2 * 127.5^2), so it is
// computed modulo 2^32 in unsigned arithmetic even where n Q alone would not fit.
__global__ void k_window_stats(const uint8_t* __restrict__ img, int pitch, int W, int H, int r,
                               int x_begin, int nx, int* __restrict__ S, int* __restrict__ Q,
                               float* __restrict__ isig) {
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
        if (S) S[o] = s;
        if (Q) Q[o] = q;
        if (isig) {
            const int var = (int)(n * (unsigned)q - (unsigned)s * (unsigned)s);
            isig[o] = var > 0 ? 1.0f / sqrtf((float)var) : 0.0f;
        }
    }
}

cudaError_t launch_window_stats(const uint8_t* img, int pitch, int W, int H, int r, int x_begin,
                                int nx, int* S, int* Q, float* isig, cudaStream_t st) {
    const size_t smem = 2 * sizeof(int) * (size_t)(nx + 2 * r);
    k_window_stats<<<H, 256, smem, st>>>(img, pitch, W, H, r, x_begin, nx, S, Q, isig);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// DT edge weights (Sec. III-B, Eq. (11)): the weight of the step between two neighbouring
// pixels p, q is K * exp(-|G(p) - G(q)| / sigma_r), G = guide / 255. eh[y][x] is the step
// (x-1, y) -> (x, y); evt[x][y] (stored transposed, so a column is contiguous) the step
// (x, y-1) -> (x, y); both 0 where the step leaves the image.
__global__ void k_dt_weights(const uint8_t* __restrict__ g, int pitch, int W, int H, float K,
                             float inv_sr255, float* __restrict__ eh, float* __restrict__ evt) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W) return;
    const int c = g[(size_t)y * pitch + x];
    float wh = 0.0f, wv = 0.0f;
    if (x > 0) wh = K * expf(-fabsf((float)(c - (int)g[(size_t)y * pitch + x - 1])) * inv_sr255);
    if (y > 0) wv = K * expf(-fabsf((float)(c - (int)g[(size_t)(y - 1) * pitch + x])) * inv_sr255);
    eh[(size_t)y * W + x] = wh;
    evt[(size_t)x * H + y] = wv;
}

cudaError_t launch_dt_weights(const uint8_t* guide, int pitch, int W, int H, float K,
                              float inv_sr255, float* eh, float* evt, cudaStream_t st) {
    dim3 grid((W + 127) / 128, H);
    k_dt_weights<<<grid, 128, 0, st>>>(guide, pitch, W, H, K, inv_sr255, eh, evt);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// DT line pair (Sec. III-B, Eqs. (3)-(6)): the forward and the backward recursive pass
// along rows (L2R then R2L) or columns (U2D then D2U) of a cost volume, in place, or, for
// the last pair of the chain, folded into the WTA keys without writing the volume back
// (Sec. V-C fuses WTA with D2U in the same way). Block = lpc lines x one disparity slice.
template <typename T, int MODE>
__global__ void __launch_bounds__(512) k_line_pair(LineArgs a) {
    extern __shared__ float smem_f[];
    const int ds = a.ds, tq = ds / kG, nch = a.nch;
    const int per_line = nch * tq;
    const int li = threadIdx.x / per_line;
    const int rem = threadIdx.x - li * per_line;
    const int k = rem / tq, dq = rem - (rem / tq) * tq;
    const int line0 = blockIdx.x * a.lpc;
    const int line = line0 + li;
    const int dl = blockIdx.y * ds + dq * kG;             // local disparity index
    const int nvalid = max(0, min(4, a.dcount - dl));
    const bool line_ok = line < a.nlines;
    const bool vec = a.vec != 0;

    DtShared sm = dt_carve(smem_f, a.lpc, nch, ds);
    dt_stage_weights(sm, a.ew, a.ew_line_stride, line0, a.nlines, a.lpc, nch, a.n);

    T* vol = reinterpret_cast<T*>(a.vol);
    T* base = vol + (size_t)(line_ok ? line : 0) * a.line_stride + dl;
    float v[kL][4];
#pragma unroll
    for (int i = 0; i < kL; ++i) {
        const int pos = k * kL + i;
        if (line_ok && pos < a.n && nvalid > 0) ld4(base + (size_t)pos * a.elem_stride, nvalid, vec, v[i]);
        else v[i][0] = v[i][1] = v[i][2] = v[i][3] = 0.0f;
    }
    __syncthreads();
    dt_chunk_products(sm, li, k, dq);
    __syncthreads();
    dt_line_pair(v, sm, li, k, dq, nch, ds, a.s);

    if constexpr (MODE == kLineWta) {
#pragma unroll
        for (int i = 0; i < kL; ++i) {
            const int pos = k * kL + i;
            const bool ok = line_ok && pos < a.n;
            const size_t pix = ok ? (size_t)line * a.pix_line + (size_t)pos * a.pix_pos : 0;
            wta_fold(v[i], nvalid, a.d_base + dl, tq, dq, ok, a.keys + pix);
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < kL; ++i) {
        const int pos = k * kL + i;
        if (line_ok && pos < a.n && nvalid > 0) st4(base + (size_t)pos * a.elem_stride, nvalid, vec, v[i]);
    }
}

size_t line_pair_smem_bytes(int lpc, int nch, int ds) { return dt_shared_bytes(lpc, nch, ds); }

cudaError_t launch_line_pair(const LineArgs& a, int mode, int dtype, cudaStream_t st) {
    dim3 grid((a.nlines + a.lpc - 1) / a.lpc, (a.dcount + a.ds - 1) / a.ds);
    dim3 block(a.lpc * a.nch * (a.ds / kG));
    const size_t smem = line_pair_smem_bytes(a.lpc, a.nch, a.ds);
    void (*fn)(LineArgs) = nullptr;
    if (mode == kLineStore) fn = dtype == 0 ? k_line_pair<float, kLineStore> : k_line_pair<__half, kLineStore>;
    else fn = dtype == 0 ? k_line_pair<float, kLineWta> : k_line_pair<__half, kLineWta>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, block, smem, st>>>(a);
    return cudaGetLastError();
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
        const float ob = __shfl_xor_sync(0xFFFFFFFFu, best, off);
        const int od = __shfl_xor_sync(0xFFFFFFFFu, bd, off);
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

__global__ void k_wta_finalize(const unsigned long long* __restrict__ keys, int npix,
                               uint16_t* __restrict__ disp) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < npix) disp[p] = (uint16_t)wta_key_disp(keys[p]);
}

cudaError_t launch_wta_finalize(const unsigned long long* keys, int npix, uint16_t* disp,
                                cudaStream_t st) {
    k_wta_finalize<<<(npix + 255) / 256, 256, 0, st>>>(keys, npix, disp);
    return cudaGetLastError();
}

size_t zncc_row_smem_bytes(int R, int mode, int nch, int ds) { return zncc_row_smem(R, mode, nch, ds); }

cudaError_t launch_zncc_row(int R, const RowArgs& a, int mode, int dtype, cudaStream_t st) {
    switch (R) {
        case 1: return launch_zncc_row_r1(a, mode, dtype, st);
        case 2: return launch_zncc_row_r2(a, mode, dtype, st);
        case 3: return launch_zncc_row_r3(a, mode, dtype, st);
        case 4: return launch_zncc_row_r4(a, mode, dtype, st);
        case 5: return launch_zncc_row_r5(a, mode, dtype, st);
        case 6: return launch_zncc_row_r6(a, mode, dtype, st);
        case 7: return launch_zncc_row_r7(a, mode, dtype, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace zncc
