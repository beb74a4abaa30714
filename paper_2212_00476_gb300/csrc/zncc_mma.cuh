// zncc_mma.cuh -- the window cross sums of Eq. (2) as a banded matrix product on the tensor
// cores, an ablation of the packed-column cost kernel (the tensor-core variant of the
// correlation): for an image row y, a tile of 64 pixels x and 128 disparities,
//   P(x, d) = sum_j sum_i L(x + i, y + j) R(x - d + i, y + j) = (A B^T)[x][c],  c = x - d,
// with A[x][(j, i)] = L(x + i, y + j) and B[c][(j, i)] = R(c + i, y + j). Pixels 0..255 are exact
// in BF16 and every partial sum of a window (at most 225 * 255^2 < 2^24) is an exact FP32
// integer, so the MMA (mma.sync m16n8k16, BF16 in, FP32 accumulate) gives the integer P exactly
// and the normalization is the expression of the other cost kernels: the values agree bit for
// bit with zncc_cost_volume.
//
// A block walks a strip of kMmaRows rows. K is laid out as a ring of 2r+1 slots of 16 entries,
// slot s holding the 2r+1 column offsets (then zeros) of the image row congruent to s modulo
// 2r+1; the next output row replaces one slot (the row that left the window), so A and B are
// built once per strip plus one slot per row. Warps w and w + 4 multiply the rows
// [16w, 16w+16) of A by the 18 column tiles of B that band of centres c = x - d needs (10 and 8
// of them). The products pass through shared memory to be normalized, with the row's window
// statistics staged there too, and stored with consecutive disparities on consecutive lanes.
// Instantiated once per window radius R in zncc_row.cu.
#pragma once

#include <cuda_bf16.h>

#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace zncc {

constexpr int kMmaTM = 64;                    // pixels per block (4 warps x 16 rows of A)
constexpr int kMmaTD = 128;                   // disparities per block
constexpr int kMmaN = kMmaTM + kMmaTD;        // centres per block (TM + TD - 1, padded)
constexpr int kMmaThreads = 256;             // 8 warps: two per 16-row tile of A
constexpr int kMmaRows = 8;                   // image rows per block
constexpr int kMmaNT = (kMmaTD + 15 + 7) / 8; // column tiles of a 16-row tile's band (18)
constexpr int kMmaNTW = 10;                   // of which a warp takes 10 (first) or 8 (second)

template <int R>
struct MmaShape {
    static constexpr int l = 2 * R + 1;
    static constexpr int K = 16 * l;          // l slots of 16
    static constexpr int KS = K + 8;          // row stride (entries): conflict-free ldmatrix rows
    static constexpr int LW = kMmaTM + 2 * R; // staged left columns of one row
    static constexpr int RW = kMmaN + 2 * R;  // staged right columns of one row
    static constexpr size_t a_bytes = (size_t)kMmaTM * KS * 2;
    static constexpr size_t b_bytes = (size_t)kMmaN * KS * 2;
    static constexpr size_t out_bytes = (size_t)kMmaTM * kMmaTD * 4;
    static constexpr size_t stats_bytes = (size_t)(kMmaTM + kMmaN) * 8;
    static constexpr size_t stage_bytes = ((size_t)(LW + RW) + 15) / 16 * 16;
    static constexpr size_t smem = a_bytes + b_bytes + out_bytes + stats_bytes + stage_bytes;
};

__device__ __forceinline__ void ldsm_x4(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3, const void* p) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(s));
}

__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                               unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Two pixel values as a packed BF16 pair (exact: integers below 256).
__device__ __forceinline__ unsigned bf16_pair(int lo, int hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn((float)lo, (float)hi);
    return *reinterpret_cast<const unsigned*>(&v);
}

template <int R, typename T>
__global__ void __launch_bounds__(kMmaThreads) k_zncc_mma(const __grid_constant__ ScanArgs a) {
    using S = MmaShape<R>;
    constexpr int l = S::l, KS = S::KS, LW = S::LW, RW = S::RW;
    extern __shared__ __align__(16) unsigned char msm[];
    __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(msm);                      // [TM][KS]
    __nv_bfloat16* Bs = reinterpret_cast<__nv_bfloat16*>(msm + S::a_bytes);         // [N][KS]
    float* outs = reinterpret_cast<float*>(msm + S::a_bytes + S::b_bytes);           // [TM][TD]
    int2* sst = reinterpret_cast<int2*>(msm + S::a_bytes + S::b_bytes + S::out_bytes); // [TM] left, [N] right
    uint8_t* Ls = msm + S::a_bytes + S::b_bytes + S::out_bytes + S::stats_bytes;     // [LW]
    uint8_t* Rs = Ls + LW;                                                           // [RW]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int W = a.W, H = a.H, D = a.D;
    const int x0 = blockIdx.x * kMmaTM, d_lo = blockIdx.y * kMmaTD;
    const int y_begin = blockIdx.z * kMmaRows, y_end = min(H, y_begin + kMmaRows);
    const int Dc = min(kMmaTD, D - d_lo);
    const int c0 = x0 - d_lo - kMmaTD + 1;                // centre of B row 0
    constexpr unsigned nwin = (unsigned)(l * l);

    // slot of image row rho (any integer, clamped when read): rho mod l
    auto fill_slot = [&](int rho) {
        const int slot = ((rho % l) + l) % l;
        const size_t row = (size_t)min(max(rho, 0), H - 1) * a.pitch;
        for (int u = tid; u < LW; u += kMmaThreads) Ls[u] = a.left[row + min(max(x0 - R + u, 0), W - 1)];
        for (int u = tid; u < RW; u += kMmaThreads) Rs[u] = a.right[row + min(max(c0 - R + u, 0), W - 1)];
        __syncthreads();
        // A[m][16 slot + i] = L(x0 + m + i - R), B[n][16 slot + i] = R(c0 + n + i - R), zero for i >= l
        for (int e = tid; e < (kMmaTM + kMmaN) * 8; e += kMmaThreads) {
            const int row_ab = e >> 3, i = (e & 7) * 2;
            const bool isA = row_ab < kMmaTM;
            const int m = isA ? row_ab : row_ab - kMmaTM;
            const uint8_t* src = isA ? Ls : Rs;
            const int v0 = i < l ? src[m + i] : 0, v1 = i + 1 < l ? src[m + i + 1] : 0;
            __nv_bfloat16* dst = (isA ? As : Bs) + m * KS + 16 * slot + i;
            *reinterpret_cast<unsigned*>(dst) = bf16_pair(v0, v1);
        }
        __syncthreads();
    };

    for (int rho = y_begin - R; rho < y_begin + R; ++rho) fill_slot(rho);
    const int m0 = 16 * (warp & 3), nt0 = m0 / 8 + (warp >> 2) * kMmaNTW;     // this warp's first column tile
    const int ntw = (warp >> 2) ? kMmaNT - kMmaNTW : kMmaNTW;
    const int nmin = m0 + kMmaTD - Dc;                    // smallest centre column with a valid d
    const int2* pl = a.packL;
    for (int y = y_begin; y < y_end; ++y) {
        fill_slot(y + R);                                 // the window's rows y - R .. y + R are in the ring
        float acc[kMmaNTW][4];
#pragma unroll
        for (int t = 0; t < kMmaNTW; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.0f;
#pragma unroll
        for (int ks = 0; ks < l; ++ks) {
            unsigned a0, a1, a2, a3;
            ldsm_x4(a0, a1, a2, a3, As + (m0 + (lane & 15)) * KS + ks * 16 + (lane >> 4) * 8);
#pragma unroll
            for (int t = 0; t < kMmaNTW; t += 2) {
                const int nb = 8 * (nt0 + t);
                if (t >= ntw || nb + 15 < nmin) continue; // not this warp's, or no valid disparity
                unsigned b0, b1, b2, b3;
                ldsm_x4(b0, b1, b2, b3, Bs + (nb + (lane & 7) + ((lane >> 4) << 3)) * KS + ks * 16 + ((lane >> 3) & 1) * 8);
                mma_bf16_16816(acc[t], a0, a1, a2, a3, b0, b1);
                mma_bf16_16816(acc[t + 1], a0, a1, a2, a3, b2, b3);
            }
        }
        // C[m][n] = P(x0 + m, d_lo + dl) with dl = m + TD - 1 - n
#pragma unroll
        for (int t = 0; t < kMmaNTW; ++t)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int m = m0 + (lane >> 2) + (e >= 2 ? 8 : 0);
                const int n = 8 * (nt0 + t) + 2 * (lane & 3) + (e & 1);
                const int dl = m + kMmaTD - 1 - n;
                if (t < ntw && dl >= 0 && dl < Dc) outs[m * kMmaTD + dl] = acc[t][e];
            }
        {   // the row's statistics: left centres x0 + m, right centres c0 + n (one entry per thread)
            const int k = tid;
            if (k < kMmaTM) {
                const int x = x0 + k;
                if (x < W) sst[k] = pl[(size_t)y * W + x];
            } else if (k < kMmaTM + kMmaN) {
                const int idx = c0 + (k - kMmaTM) + D - 1;          // centre c at index c + D - 1
                if (idx >= 0 && idx < W + D - 1) sst[k] = a.packR[(size_t)y * (W + D - 1) + idx];
            }
        }
        __syncthreads();
        for (int m = warp; m < kMmaTM; m += kMmaThreads / 32) {
            const int x = x0 + m;
            if (x >= W) break;
            const int2 st = sst[m];
            T* out = reinterpret_cast<T*>(a.vol) + ((size_t)y * W + x) * D + d_lo;
            for (int dl = lane; dl < Dc; dl += 32) {
                const int2 sr = sst[kMmaTM + m + kMmaTD - 1 - dl];   // centre x - d = c0 + n
                const unsigned P = (unsigned)outs[m * kMmaTD + dl];
                const unsigned num = nwin * P - (unsigned)st.x * (unsigned)sr.x;
                const float c = (float)(int)num * __int_as_float(st.y) * __int_as_float(sr.y);
                if constexpr (std::is_same<T, float>::value) out[dl] = c;
                else out[dl] = __float2half_rn(c);
            }
        }
        // (the next fill_slot's first barrier orders these reads of outs before the next writes)
    }
}

template <int R>
cudaError_t launch_zncc_mma_impl(const ScanArgs& a, int dtype, cudaStream_t st) {
    const size_t smem = MmaShape<R>::smem;
    const dim3 grid((a.W + kMmaTM - 1) / kMmaTM, (a.D + kMmaTD - 1) / kMmaTD, (a.H + kMmaRows - 1) / kMmaRows);
    if (dtype == 0) {
        cudaError_t e = set_max_smem((const void*)k_zncc_mma<R, float>, smem);
        if (e != cudaSuccess) return e;
        k_zncc_mma<R, float><<<grid, kMmaThreads, smem, st>>>(a);
    } else {
        cudaError_t e = set_max_smem((const void*)k_zncc_mma<R, __half>, smem);
        if (e != cudaSuccess) return e;
        k_zncc_mma<R, __half><<<grid, kMmaThreads, smem, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace zncc
