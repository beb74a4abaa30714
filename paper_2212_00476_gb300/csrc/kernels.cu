// kernels.cu -- window statistics, DT coefficients, DT line pairs and WTA kernels.
#include <algorithm>

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
        const float is = var > 0 ? 1.0f / sqrtf((float)var) : 0.0f;
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
__global__ void k_dt_coef(const uint8_t* __restrict__ g, int pitch, int W, int H, float K,
                          float inv_sr255, float4* __restrict__ coefH, float4* __restrict__ coefV) {
    const int nchH = (W + kL - 1) / kL, nchV = (H + kL - 1) / kL;
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    int chunk = gid / kL;
    const int i = gid & (kL - 1);
    const bool horiz = chunk < H * nchH;
    if (!horiz) chunk -= H * nchH;
    const bool live = horiz || chunk < W * nchV;
    const int n = horiz ? W : H;
    const int nchl = horiz ? nchH : nchV;
    const int line = live ? chunk / nchl : 0;
    const int p = (live ? chunk - line * nchl : 0) * kL + i;
    auto pix = [&](int q) -> int {
        return horiz ? g[(size_t)line * pitch + q] : g[(size_t)q * pitch + line];
    };
    auto weight = [&](int q) -> float {    // the step q-1 -> q
        return (live && q >= 1 && q < n) ? K * expf(-fabsf((float)(pix(q) - pix(q - 1))) * inv_sr255) : 0.0f;
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
        float4* out = horiz ? coefH + (size_t)line * W : coefV + (size_t)line * H;
        out[p] = make_float4(w, A, wn, B);
    }
}

cudaError_t launch_dt_coef(const uint8_t* guide, int pitch, int W, int H, float K, float inv_sr255,
                           float4* coefH, float4* coefV, cudaStream_t st) {
    const long long total = (long long)kL * (H * ((W + kL - 1) / kL) + W * ((H + kL - 1) / kL));
    k_dt_coef<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(guide, pitch, W, H, K, inv_sr255, coefH, coefV);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// DT line pair (Sec. III-B, Eqs. (3)-(6)): the forward and the backward recursive pass
// along rows (L2R then R2L) or columns (U2D then D2U) of a cost volume, or, for the last
// pair of the chain, folded into a per-pixel running best without writing the volume back
// (Sec. V-C fuses WTA with D2U in the same way).
//
// Work: lines in groups of lpc, each group with nslices disparity slices of 4*tq
// disparities; an item is (group, slice), numbered group-major. The grid is sized to the
// resident blocks (persistent); block b processes the items [b*per_block, (b+1)*per_block)
// in order, restaging the coefficients when the group changes. With aligned 4-disparity
// groups (async) each thread streams its elements of the next item into shared memory with
// cp.async while the current one is computed, across group boundaries: two staging buffers,
// each refilled (two items ahead) as soon as the forward sweep has consumed it. In Wta mode
// per_block is a multiple of nslices: a block sees every disparity of its lines.
template <typename T>
__host__ __device__ inline size_t line_stage_bytes(const LineArgs& a) {
    return a.async ? 2ull * a.lpc * kL * a.nch * a.tq * (4 * sizeof(T)) : 0;
}

int line_pair_items(const LineArgs& a) {
    const int nslices = (a.dcount + kG * a.tq - 1) / (kG * a.tq);
    return ((a.nlines + a.lpc - 1) / a.lpc) * nslices;
}

template <typename T, int MODE>
__global__ void __launch_bounds__(512) k_line_pair(LineArgs a) {
    extern __shared__ float4 smem4[];
    const int tq = a.tq, nch = a.nch, ds = kG * tq;
    const int per_line = nch * tq, nwl = per_line >> 5, span = nch * kL;
    const int li = threadIdx.x / per_line;
    const int tl = threadIdx.x - li * per_line;
    const int k = tl / tq, dq = tl - k * tq;
    const int lane = threadIdx.x & 31, wl = tl >> 5;
    const int pX = plane_of(span);

    T* stage = reinterpret_cast<T*>(smem4);                           // [2][lpc][kL][per_line] x 4
    float4* co_all = reinterpret_cast<float4*>(reinterpret_cast<char*>(smem4) + line_stage_bytes<T>(a));
    float2* mul_all = reinterpret_cast<float2*>(co_all + a.lpc * 4 * pX);   // [lpc][4 pX]
    float4* sb_all = reinterpret_cast<float4*>(mul_all + a.lpc * 4 * pX);   // [lpc][2 nwl tq]
    float* sa_all = reinterpret_cast<float*>(sb_all + a.lpc * 2 * nwl * tq);
    const float4* co = co_all + li * 4 * pX;
    const float2* mul = mul_all + li * 4 * pX;
    float4* sb = sb_all + li * 2 * nwl * tq;
    float* sa = sa_all + li * 2 * nwl * tq;

    const int nslices = (a.dcount + ds - 1) / ds;
    const int total = ((a.nlines + a.lpc - 1) / a.lpc) * nslices;
    const int it0 = blockIdx.x * a.per_block;
    const int it1 = min(total, it0 + a.per_block);
    T* vol = reinterpret_cast<T*>(a.vol);
    const T* src = a.src ? reinterpret_cast<const T*>(a.src) : vol;
    const bool vec = a.vec != 0, async = a.async != 0, ones = a.src_ones != 0;
    const bool scaled_in = a.ahat_in != nullptr;
    const int npos = a.n - k * kL;                                     // positions of this chunk
    auto elem0 = [&](int line, int sl) -> size_t {                   // the chunk's first group
        return (size_t)line * a.line_stride + (size_t)(k * kL) * a.elem_stride + sl * ds + dq * kG;
    };
    auto stage_at = [&](int buf, int i) -> T* {
        return stage + ((size_t)((buf * a.lpc + li) * kL + i) * per_line + tl) * 4;
    };
    // prefetch of item `it` into the stage buffer. With vec the entries per pixel are a
    // multiple of 4, so a group with any valid disparity lies whole inside the volume; its
    // entries past dcount are never stored or compared.
    auto prefetch = [&](int it, int buf) {
        if (it < it1) {
            const int g = it / nslices, sl = it - g * nslices;
            const int line = g * a.lpc + li;
            const bool ok = line < a.nlines && sl * ds + dq * kG < a.dcount;
            const T* p = src + (ok ? elem0(line, sl) : 0);
#pragma unroll
            for (int i = 0; i < kL; ++i) {
                const bool valid = ok && i < npos;
                cp_async<4 * sizeof(T)>(stage_at(buf, i), valid ? p + (size_t)i * a.elem_stride : src, valid);
            }
        }
        cp_async_commit();
    };
    if (async) {
        prefetch(it0, 0);
        prefetch(it0 + 1, 1);
    }

    WtaRegs wr;
    int cur_group = -1;
    for (int it = it0, n_it = 0; it < it1; ++it, ++n_it) {
        const int g = it / nslices, sl = it - g * nslices;
        const int line = g * a.lpc + li;
        const bool line_ok = line < a.nlines;
        if (g != cur_group) {          // stage the coefficients and multipliers of group g
            __syncthreads();
            for (int l2 = 0; l2 < a.lpc; ++l2) {
                const int ln = g * a.lpc + l2;
                const bool ok = ln < a.nlines;
                for (int t = threadIdx.x; t < span; t += blockDim.x) {
                    const bool in = ok && t < a.n;
                    co_all[l2 * 4 * pX + cidx(t, pX)] =
                        in ? __ldg(a.coef + (size_t)ln * a.coef_line_stride + t) : make_float4(0.f, 0.f, 0.f, 0.f);
                    const size_t pix = (size_t)ln * a.pix_line + (size_t)t * a.pix_pos;
                    const float mi = in && a.ahat_in ? __ldg(a.ahat_in + pix) : 1.0f;
                    const float mo = in && a.ahat_out ? a.s2 / __ldg(a.ahat_out + pix) : a.s2;
                    mul_all[l2 * 4 * pX + cidx(t, pX)] = make_float2(mi, mo);
                }
            }
            if constexpr (MODE == kLineWta) wr.reset();
            __syncthreads();
            cur_group = g;
        }
        const int dl = sl * ds + dq * kG;                              // entry of d_first
        const int nvalid = max(0, min(4, a.dcount - dl));
        const bool any = line_ok && nvalid > 0;
        float v[kL][4];
        if (ones) {
#pragma unroll
            for (int i = 0; i < kL; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) v[i][j] = (any && i < npos && j < nvalid) ? 1.0f : 0.0f;
        } else if (async) {
            cp_async_wait<1>();                                        // this item's copies landed
#pragma unroll
            for (int i = 0; i < kL; ++i) lds4(stage_at(n_it & 1, i), v[i]);
        } else {
            const T* q = src + (line_ok ? elem0(line, sl) : 0);
#pragma unroll
            for (int i = 0; i < kL; ++i) {
                if (any && i < npos) ld4(q, nvalid, vec, v[i]);
                else v[i][0] = v[i][1] = v[i][2] = v[i][3] = 0.0f;
                q += a.elem_stride;
            }
        }
        if (scaled_in) {
#pragma unroll
            for (int i = 0; i < kL; ++i) {
                const float m = mul[cidx(k * kL + i, pX)].x;
#pragma unroll
                for (int j = 0; j < 4; ++j) v[i][j] *= m;
            }
        }
        // the staging buffer is free once the forward sweep has read it: refill it two ahead
        dt_pair(v, co, pX, k, tq, dq, lane, wl, nwl, sa, sb, a.s2, mul, [&]() {
            if (async) prefetch(it + 2, n_it & 1);
        });
        if constexpr (MODE == kLineWta) {
            wr.fold(v, nvalid, a.d_base + dl);
            if (sl == nslices - 1) {                                   // the group's last slice
#pragma unroll
                for (int i = 0; i < kL; ++i) {
                    float best;
                    int bd;
                    wta_reduce_lanes(wr.entry(i), tq, best, bd);
                    const int pos = k * kL + i;
                    if (dq == 0 && line_ok && pos < a.n) {
                        const size_t pix = (size_t)line * a.pix_line + (size_t)pos * a.pix_pos;
                        if (!a.wta.first) {                            // earlier launches: smaller d
                            const float pb = a.wta.bestv[pix];
                            if (!(best > pb)) { best = pb; bd = a.wta.bestd[pix]; }
                        }
                        if (a.wta.last) a.wta.disp[pix] = (uint16_t)bd;
                        else {
                            a.wta.bestv[pix] = best;
                            a.wta.bestd[pix] = bd;
                        }
                    }
                }
            }
        } else {
            T* q = vol + (line_ok ? elem0(line, sl) : 0);
#pragma unroll
            for (int i = 0; i < kL; ++i) {
                if (any && i < npos) st4(q, nvalid, vec, v[i]);
                q += a.elem_stride;
            }
        }
    }
    if (async) cp_async_wait<0>();
}

size_t line_pair_smem_bytes(int mode, int dtype, const LineArgs& a) {
    const int pX = plane_of(a.nch * kL);
    const int nwl = a.nch * a.tq / 32;
    size_t b = dtype == 0 ? line_stage_bytes<float>(a) : line_stage_bytes<__half>(a);
    b += (size_t)a.lpc * ((16ull + 8ull) * 4 * pX + dt_scan_bytes(nwl, a.tq));
    return b;
}

static void (*line_pair_fn(int mode, int dtype))(LineArgs) {
    if (mode == kLineStore) return dtype == 0 ? k_line_pair<float, kLineStore> : k_line_pair<__half, kLineStore>;
    return dtype == 0 ? k_line_pair<float, kLineWta> : k_line_pair<__half, kLineWta>;
}

cudaError_t line_pair_occupancy(const LineArgs& a, int mode, int dtype, int* blocks_per_sm) {
    void (*fn)(LineArgs) = line_pair_fn(mode, dtype);
    const size_t smem = line_pair_smem_bytes(mode, dtype, a);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, a.lpc * a.nch * a.tq, smem);
}

cudaError_t launch_line_pair(const LineArgs& a, int mode, int dtype, cudaStream_t st) {
    const int total = line_pair_items(a);
    dim3 grid((total + a.per_block - 1) / a.per_block);
    dim3 block(a.lpc * a.nch * a.tq);
    const size_t smem = line_pair_smem_bytes(mode, dtype, a);
    void (*fn)(LineArgs) = line_pair_fn(mode, dtype);
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

size_t zncc_row_smem_bytes(int R, int mode, const RowArgs& a, int nthreads) {
    return zncc_row_smem(R, mode, a, nthreads);
}

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
