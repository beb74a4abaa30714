// zncc_row.cuh -- ZNCC cost of one image row for a slice of disparities, optionally fused
// with the first horizontal DT pass pair (Sec. V-C fuses the cost with L2R the same way) or
// with WTA (no aggregation). Instantiated once per window radius R in zncc_rN.cu.
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace zncc {

// Block (row y, disparity slice [d0, d0+ds)): thread (chunk k, dq) computes the costs of
// pixels x in [16k, 16k+16) for the four disparities d0 + 4dq .. d0 + 4dq + 3. The chunk
// count is padded to whole warps; pixels x >= W are computed from clamped reads and dropped.
//
// Cost (Eq. (1) through Eq. (2)): with P = sum over the window of I_R(x+i, y+j) *
// I_T(x-d+i, y+j), n = (2R+1)^2 and the window sums S of each image,
//   C = (n P - S_R(x) S_T(x-d)) * inv_sigma_R(x) * inv_sigma_T(x-d),
// inv_sigma = 1/sqrt(n Q - S^2) (0 for a flat window, which makes C = 0). The integer
// numerator is exact: its true value is bounded by sqrt((nQ_R - S_R^2)(nQ_T - S_T^2)) <
// 2^31, so it is computed modulo 2^32 in unsigned arithmetic.
//
// P is built from column sums over the window's rows: the block packs, for every column
// of the band of rows y-R..y+R, up to 16 pixels into four 32-bit words, so that a column
// dot product is at most four __dp4a. A thread walks x' from 16k-R to 16k+15+R keeping
// the target columns of its four disparities in a sliding register window (one new
// shared-memory load per step serves all four, since column x'-d at step x' is column
// (x'-1)-(d-1) of the previous step), and turns the running prefix of column sums into the
// window sums P(x) = prefix(x+R) - prefix(x-R-1).
template <int R, typename T, int MODE>
__global__ void __launch_bounds__(512) k_zncc_row(RowArgs a) {
    constexpr int l = 2 * R + 1;
    constexpr int NW = (l + 3) / 4;     // packed words per column
    extern __shared__ uint4 smem_u4[];

    const int y = blockIdx.x;
    const int ds = a.ds, tq = ds / kG, nch = a.nch;
    const int d0 = a.d_begin + blockIdx.y * ds;
    const int tid = threadIdx.x;
    const int dq = tid % tq, k = tid / tq;
    const int span = nch * kL;
    const int W = a.W, H = a.H;

    // ---- shared memory carve (all arrays in the four-plane layout) ----
    const int NLP = span + 2 * R;              // left columns x' in [-R, span+R)
    const int NRP = span + 2 * R + ds - 1;     // right columns x'' in [xr0, xr0+NRP)
    const int xr0 = -R - (d0 + ds - 1);
    const int NSR = span + ds - 1;             // target centres c in [c0, c0+NSR)
    const int c0 = -(d0 + ds - 1);
    const int pLP = plane_of(NLP), pRP = plane_of(NRP), pSL = plane_of(span), pSR = plane_of(NSR);
    uint4* LP = smem_u4;
    uint4* RP = LP + 4 * pLP;
    int* SL = reinterpret_cast<int*>(RP + 4 * pRP);
    float* ISL = reinterpret_cast<float*>(SL + 4 * pSL);
    int* SR = reinterpret_cast<int*>(ISL + 4 * pSL);
    float* ISR = reinterpret_cast<float*>(SR + 4 * pSR);

    // ---- stage the packed bands and the window statistics ----
    for (int t = tid; t < NLP + NRP; t += blockDim.x) {
        const bool is_left = t < NLP;
        const int ix = is_left ? t : t - NLP;
        const int xc = min(max(is_left ? ix - R : xr0 + ix, 0), W - 1);
        const uint8_t* img = is_left ? a.left : a.right;
        unsigned w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int j = 0; j < l; ++j) {
            const int yc = min(max(y - R + j, 0), H - 1);
            w[j >> 2] |= (unsigned)img[(size_t)yc * a.pitch + xc] << (8 * (j & 3));
        }
        uint4 pk = make_uint4(w[0], w[1], w[2], w[3]);
        if (is_left) LP[p4(ix, pLP)] = pk;
        else RP[p4(ix, pRP)] = pk;
    }
    for (int t = tid; t < span; t += blockDim.x) {
        const bool in = t < W;
        SL[p4(t, pSL)] = in ? a.SL[(size_t)y * W + t] : 0;
        ISL[p4(t, pSL)] = in ? a.ISL[(size_t)y * W + t] : 0.0f;
    }
    const int WE = W + a.D - 1;   // extended target statistics: centre c at column c + D - 1
    for (int t = tid; t < NSR; t += blockDim.x) {
        const int gi = c0 + t + a.D - 1;
        const bool in = gi >= 0 && c0 + t < W;
        SR[p4(t, pSR)] = in ? a.SR[(size_t)y * WE + gi] : 0;
        ISR[p4(t, pSR)] = in ? a.ISR[(size_t)y * WE + gi] : 0.0f;
    }
    __syncthreads();

    // ---- window sums of products P for 16 pixels x 4 disparities ----
    const int x0 = k * kL;
    const int d_first = d0 + dq * kG;
    int P[kL][4];
#pragma unroll
    for (int i = 0; i < kL; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) P[i][j] = 0;

    // RP index of column x' - d_first - j at step t (x' = x0 - R + t): base + t - j
    const int rbase = x0 - R - d_first - xr0;          // >= 3 since 4dq + 3 <= ds - 1
    uint4 rp[4];
    rp[1] = RP[p4(rbase - 1, pRP)];
    rp[2] = RP[p4(rbase - 2, pRP)];
    rp[3] = RP[p4(rbase - 3, pRP)];
    unsigned pre[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int t = 0; t < kL + 2 * R; ++t) {
        const uint4 lp = LP[p4(x0 + t, pLP)];
        rp[0] = RP[p4(rbase + t, pRP)];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            unsigned cs = __dp4a(lp.x, rp[j].x, 0u);
            if (NW > 1) cs = __dp4a(lp.y, rp[j].y, cs);
            if (NW > 2) cs = __dp4a(lp.z, rp[j].z, cs);
            if (NW > 3) cs = __dp4a(lp.w, rp[j].w, cs);
            pre[j] += cs;
            if (t - 2 * R >= 0 && t - 2 * R < kL) P[t - 2 * R][j] += (int)pre[j];
            if (t + 1 < kL) P[t + 1][j] -= (int)pre[j];
        }
        rp[3] = rp[2];
        rp[2] = rp[1];
        rp[1] = rp[0];
    }

    // ---- normalization, Eq. (2) ----
    const unsigned n = (unsigned)(l * l);
    const int nvalid = max(0, min(4, a.d_end - d_first));
    float v[kL][4];
#pragma unroll
    for (int i = 0; i < kL; ++i) {
        const int x = x0 + i;
        const unsigned sl = (unsigned)at4(SL, x0, i, pSL);
        const float isl = at4(ISL, x0, i, pSL);
        // target centre x - d_first - j sits at SR index x - d_first - j - c0
        const int sbase = x - d_first - c0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const unsigned sr = (unsigned)SR[p4(sbase - j, pSR)];
            const float isr = ISR[p4(sbase - j, pSR)];
            const unsigned num = n * (unsigned)P[i][j] - sl * sr;
            const bool ok = x < W && j < nvalid;
            v[i][j] = ok ? (float)(int)num * isl * isr : 0.0f;
        }
    }

    if constexpr (MODE == kModeWta) {
#pragma unroll
        for (int i = 0; i < kL; ++i) {
            const int x = x0 + i;
            wta_fold(v[i], nvalid, d_first, tq, dq, x < W, a.keys + (size_t)y * W + min(x, W - 1));
        }
        return;
    }
    if constexpr (MODE == kModeHPair) {
        // the DT scratch reuses the band and statistics area, which is dead from here on
        __syncthreads();
        DtShared dsm = dt_carve(reinterpret_cast<float*>(smem_u4), 1, nch, ds);
        dt_stage_weights(dsm, a.eh, W, y, H, 1, nch, W);
        __syncthreads();
        dt_chunk_products(dsm, 0, k, dq);
        __syncthreads();
        dt_line_pair(v, dsm, 0, k, dq, nch, ds, a.s);
    }

    // ---- store [H][W][dstride] ----
    T* out = reinterpret_cast<T*>(a.vol);
    const int dl = d_first - a.d_out0;
    const bool vec = a.vec != 0;
#pragma unroll
    for (int i = 0; i < kL; ++i) {
        const int x = x0 + i;
        if (x < W && nvalid > 0)
            st4(out + ((size_t)y * W + x) * a.dstride + dl, nvalid, vec, v[i]);
    }
}

// Host-visible shared-memory size of one block of k_zncc_row.
inline size_t zncc_row_smem(int R, int mode, int nch, int ds) {
    const int span = nch * kL;
    size_t b = 16ull * 4 * (plane_of(span + 2 * R) + plane_of(span + 2 * R + ds - 1));
    b += 8ull * 4 * (plane_of(span) + plane_of(span + ds - 1));
    if (mode == kModeHPair && dt_shared_bytes(1, nch, ds) > b) b = dt_shared_bytes(1, nch, ds);
    return b;
}

template <int R>
cudaError_t launch_zncc_row_impl(const RowArgs& a, int mode, int dtype, cudaStream_t st) {
    dim3 grid(a.H, (a.d_end - a.d_begin + a.ds - 1) / a.ds);
    dim3 block(a.nch * (a.ds / kG));
    size_t smem = zncc_row_smem(R, mode, a.nch, a.ds);
    void (*fn)(RowArgs) = nullptr;
    if (mode == kModeRaw) fn = dtype == 0 ? k_zncc_row<R, float, kModeRaw> : k_zncc_row<R, __half, kModeRaw>;
    else if (mode == kModeHPair) fn = dtype == 0 ? k_zncc_row<R, float, kModeHPair> : k_zncc_row<R, __half, kModeHPair>;
    else fn = k_zncc_row<R, float, kModeWta>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, block, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace zncc
