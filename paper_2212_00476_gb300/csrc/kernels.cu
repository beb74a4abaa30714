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
// along rows (L2R then R2L) or columns (U2D then D2U) of a cost volume, in place, or, for
// the last pair of the chain, folded into a per-pixel running best without writing the
// volume back (Sec. V-C fuses WTA with D2U in the same way). Block = lpc lines x a run of
// spb disparity slices (4*tq disparities each); the lines' coefficients are staged once.
// With aligned 4-disparity groups (vec) each thread streams its elements of the next two
// slices into shared memory with cp.async while the current slice is being computed.
template <typename T>
__host__ __device__ inline size_t line_stage_bytes(const LineArgs& a) {
    return a.async ? 2ull * a.lpc * kL * a.nch * a.tq * (4 * sizeof(T)) : 0;
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
    const int line0 = blockIdx.x * a.lpc;
    const int line = line0 + li;
    const bool line_ok = line < a.nlines;
    const int pX = plane_of(span);

    T* stage = reinterpret_cast<T*>(smem4);                           // [2][lpc][kL][per_line] x 4
    float4* co_all = reinterpret_cast<float4*>(reinterpret_cast<char*>(smem4) + line_stage_bytes<T>(a));
    float4* sb_all = co_all + a.lpc * 4 * pX;                          // [lpc][2 nwl tq]
    float* sa_all = reinterpret_cast<float*>(sb_all + a.lpc * 2 * nwl * tq);
    float* rbv_all = sa_all + a.lpc * 2 * nwl * tq;                    // [lpc][4 pX] (Wta)
    int* rbd_all = reinterpret_cast<int*>(rbv_all + a.lpc * 4 * pX);
    const float4* co = co_all + li * 4 * pX;
    float4* sb = sb_all + li * 2 * nwl * tq;
    float* sa = sa_all + li * 2 * nwl * tq;
    float* rbv = rbv_all + li * 4 * pX;
    int* rbd = rbd_all + li * 4 * pX;

    const int nslices = (a.dcount + ds - 1) / ds;
    const int s_begin = blockIdx.y * a.spb;
    const int s_end = min(nslices, s_begin + a.spb);
    T* vol = reinterpret_cast<T*>(a.vol);
    const bool vec = a.vec != 0;
    const bool async = a.async != 0;
    const int npos = a.n - k * kL;                                     // positions of this chunk
    // the chunk's first element group of slice sl
    auto chunk_base = [&](int sl) -> T* {
        return vol + (size_t)(line_ok ? line : 0) * a.line_stride + (size_t)(k * kL) * a.elem_stride + sl * ds + dq * kG;
    };
    auto stage_at = [&](int buf, int i) -> T* {
        return stage + ((size_t)((buf * a.lpc + li) * kL + i) * per_line + tl) * 4;
    };
    // prefetch of slice sl into stage buffer buf. With vec the entries per pixel are a
    // multiple of 4, so a group with any valid disparity lies whole inside the volume; its
    // entries past dcount are never stored or compared.
    auto prefetch = [&](int sl, int buf) {
        if (sl < s_end) {
            const bool ok = line_ok && sl * ds + dq * kG < a.dcount;
            const T* src = chunk_base(sl);
#pragma unroll
            for (int i = 0; i < kL; ++i) {
                const bool valid = ok && i < npos;
                cp_async<4 * sizeof(T)>(stage_at(buf, i), valid ? src + (size_t)i * a.elem_stride : vol, valid);
            }
        }
        cp_async_commit();
    };
    if (async) {
        prefetch(s_begin, 0);
        prefetch(s_begin + 1, 1);
    }

    for (int l2 = 0; l2 < a.lpc; ++l2) {
        const int ln = line0 + l2;
        const bool ok = ln < a.nlines;
        for (int t = threadIdx.x; t < span; t += blockDim.x) {
            co_all[l2 * 4 * pX + cidx(t, pX)] =
                ok && t < a.n ? __ldg(a.coef + (size_t)ln * a.coef_line_stride + t) : make_float4(0.f, 0.f, 0.f, 0.f);
            if constexpr (MODE == kLineWta) {
                const bool in = ok && t < a.n && !a.wta.first;
                const size_t pix = (size_t)ln * a.pix_line + (size_t)t * a.pix_pos;
                rbv_all[l2 * 4 * pX + p4(t, pX)] = in ? a.wta.bestv[pix] : -INFINITY;
                rbd_all[l2 * 4 * pX + p4(t, pX)] = in ? a.wta.bestd[pix] : 0;
            }
        }
    }
    __syncthreads();

    for (int sl = s_begin, it = 0; sl < s_end; ++sl, ++it) {
        const int dl = sl * ds + dq * kG;                              // entry of d_first
        const int nvalid = max(0, min(4, a.dcount - dl));
        const bool any = line_ok && nvalid > 0;
        float v[kL][4];
        if (async) {
            cp_async_wait<1>();                                        // this slice's copies landed
#pragma unroll
            for (int i = 0; i < kL; ++i) lds4(stage_at(it & 1, i), v[i]);
        } else {
            const T* q = chunk_base(sl);
#pragma unroll
            for (int i = 0; i < kL; ++i) {
                if (any && i < npos) ld4(q, nvalid, vec, v[i]);
                else v[i][0] = v[i][1] = v[i][2] = v[i][3] = 0.0f;
                q += a.elem_stride;
            }
        }
        dt_pair(v, co, pX, k, tq, dq, lane, wl, nwl, sa, sb, a.s2);
        // the stage buffer was consumed by the sweeps above: refill it with slice sl + 2
        if (async) prefetch(sl + 2, it & 1);
        if constexpr (MODE == kLineWta) {
#pragma unroll
            for (int i = 0; i < kL; ++i) {
                float best;
                int bd;
                wta_group(v[i], nvalid, a.d_base + dl, tq, best, bd);
                const int pos = k * kL + i;
                if (dq == 0 && pos < a.n && best > rbv[p4(pos, pX)]) {
                    rbv[p4(pos, pX)] = best;
                    rbd[p4(pos, pX)] = bd;
                }
            }
        } else {
            T* q = chunk_base(sl);
#pragma unroll
            for (int i = 0; i < kL; ++i) {
                if (any && i < npos) st4(q, nvalid, vec, v[i]);
                q += a.elem_stride;
            }
        }
    }
    if (async) cp_async_wait<0>();
    if constexpr (MODE == kLineWta) {
        if (dq == 0 && line_ok) {
#pragma unroll
            for (int i = 0; i < kL; ++i) {
                const int pos = k * kL + i;
                if (pos >= a.n) break;
                const size_t pix = (size_t)line * a.pix_line + (size_t)pos * a.pix_pos;
                if (a.wta.last) a.wta.disp[pix] = (uint16_t)rbd[p4(pos, pX)];
                else {
                    a.wta.bestv[pix] = rbv[p4(pos, pX)];
                    a.wta.bestd[pix] = rbd[p4(pos, pX)];
                }
            }
        }
    }
}

size_t line_pair_smem_bytes(int mode, int dtype, const LineArgs& a) {
    const int pX = plane_of(a.nch * kL);
    const int nwl = a.nch * a.tq / 32;
    size_t b = dtype == 0 ? line_stage_bytes<float>(a) : line_stage_bytes<__half>(a);
    b += (size_t)a.lpc * (16ull * 4 * pX + dt_scan_bytes(nwl, a.tq));
    if (mode == kLineWta) b += (size_t)a.lpc * 8 * 4 * pX;
    return b;
}

cudaError_t launch_line_pair(const LineArgs& a, int mode, int dtype, cudaStream_t st) {
    const int ds = kG * a.tq;
    const int nslices = (a.dcount + ds - 1) / ds;
    dim3 grid((a.nlines + a.lpc - 1) / a.lpc, (nslices + a.spb - 1) / a.spb);
    dim3 block(a.lpc * a.nch * a.tq);
    const size_t smem = line_pair_smem_bytes(mode, dtype, a);
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
