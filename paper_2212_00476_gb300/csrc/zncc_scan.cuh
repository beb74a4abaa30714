// zncc_scan.cuh -- the paper's "original" progressive-scan ZNCC (the comparison method of
// Sec. V-B): every window sum of products is slid along the row, one new column in and one
// old column out, and every column's products are recomputed from the pixels of the 2r+1
// rows (no reuse across rows, no packed arithmetic). It is kept as an ablation baseline for
// the packed-column cost kernel (k_zncc_row) and gives the same values bit for bit: the
// integer numerator is exact and the normalization is the same expression.
// Instantiated once per window radius R in zncc_row.cu.
#pragma once

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace zncc {

constexpr int kScanSeg = 64;        // x positions per thread
constexpr int kScanThreads = 128;   // disparities per block

// Thread (disparity d, row y, segment of kScanSeg positions): the window sum P(x, d) at the
// segment start from 2r+1 columns, then one new column per step; the columns of the current
// window stay in a ring of registers (the loop is unrolled by 2r+1 so the ring index is static).
template <int R, typename T>
__global__ void __launch_bounds__(kScanThreads) k_zncc_scan(const __grid_constant__ ScanArgs a) {
    constexpr int l = 2 * R + 1;
    constexpr unsigned n = (unsigned)(l * l);
    const int d = blockIdx.x * kScanThreads + threadIdx.x;
    const int y = blockIdx.z;
    const int x0 = blockIdx.y * kScanSeg, x1 = min(a.W, x0 + kScanSeg);
    if (d >= a.D) return;
    const int W = a.W, H = a.H;
    const uint8_t* rl[l];
    const uint8_t* rr[l];
#pragma unroll
    for (int j = 0; j < l; ++j) {
        const size_t row = (size_t)min(max(y - R + j, 0), H - 1) * a.pitch;
        rl[j] = a.left + row;
        rr[j] = a.right + row;
    }
    auto column = [&](int xp) -> unsigned {      // sum over the rows of I_R(xp) * I_T(xp - d)
        const int xl = min(max(xp, 0), W - 1), xr = min(max(xp - d, 0), W - 1);
        unsigned s = 0u;
#pragma unroll
        for (int j = 0; j < l; ++j) s += (unsigned)rl[j][xl] * (unsigned)rr[j][xr];
        return s;
    };
    unsigned ring[l];
    unsigned P = 0u;
#pragma unroll
    for (int i = 0; i < l; ++i) {
        ring[i] = column(x0 - R + i);
        P += ring[i];
    }
    const int2* sl = a.packL + (size_t)y * W;
    const int2* sr = a.packR + (size_t)y * (W + a.D - 1) + (a.D - 1) - d;     // centre x - d
    T* out = reinterpret_cast<T*>(a.vol) + d;
    for (int x = x0; x < x1; x += l) {
#pragma unroll
        for (int k = 0; k < l; ++k) {
            const int xx = x + k;
            if (xx < x1) {
                const int2 L = sl[xx], Rs = sr[xx];
                const unsigned num = n * P - (unsigned)L.x * (unsigned)Rs.x;
                const float c = (float)(int)num * __int_as_float(L.y) * __int_as_float(Rs.y);
                if constexpr (std::is_same<T, float>::value) out[((size_t)y * W + xx) * a.D] = c;
                else out[((size_t)y * W + xx) * a.D] = __float2half_rn(c);
                const unsigned cn = column(xx + 1 + R);
                P += cn - ring[k];
                ring[k] = cn;
            }
        }
    }
}

template <int R>
cudaError_t launch_zncc_scan_impl(const ScanArgs& a, int dtype, cudaStream_t st) {
    const dim3 grid((a.D + kScanThreads - 1) / kScanThreads, (a.W + kScanSeg - 1) / kScanSeg, a.H);
    if (dtype == 0) k_zncc_scan<R, float><<<grid, kScanThreads, 0, st>>>(a);
    else k_zncc_scan<R, __half><<<grid, kScanThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace zncc
