// common.cuh -- device helpers shared by the ZNCC / DT / WTA kernels (sm_103a).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace zncc {

// Positions of one line handled by one thread (a "chunk") and disparities per thread.
constexpr int kL = 16;
constexpr int kG = 4;

// Shared-memory arrays indexed by a pixel coordinate are stored as four interleaved
// planes, entry idx at (idx & 3) * plane + (idx >> 2). In every access pattern below the
// lanes of a warp share idx & 3 and spread over consecutive idx >> 2, so the 32 lanes hit
// distinct banks (plain layouts put lanes 16 or 64 entries apart on the same bank).
__host__ __device__ __forceinline__ int plane_of(int len) { return ((len + 3) / 4 + 31) & ~31; }
__device__ __forceinline__ int p4(int idx, int plane) { return (idx & 3) * plane + (idx >> 2); }
// Entry start + i of a four-plane array, for start a multiple of 4 (i known at compile time).
template <typename T>
__device__ __forceinline__ T& at4(T* base, int start, int i, int plane) {
    return base[(i & 3) * plane + (start >> 2) + (i >> 2)];
}

// ---- cost-volume element access: 4 consecutive disparities per thread ----------------

__device__ __forceinline__ void ld4(const float* p, int nvalid, bool vec, float (&o)[4]) {
    if (vec && nvalid == 4) {
        float4 t = *reinterpret_cast<const float4*>(p);
        o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] = j < nvalid ? p[j] : 0.0f;
    }
}

// Half values travel as raw 16-bit patterns inside 32-bit words (low half = lower address);
// __ushort_as_half / __half_as_ushort convert without type-punned pointer accesses.
__device__ __forceinline__ float half_lo(unsigned w) { return __half2float(__ushort_as_half((unsigned short)(w & 0xFFFFu))); }
__device__ __forceinline__ float half_hi(unsigned w) { return __half2float(__ushort_as_half((unsigned short)(w >> 16))); }
__device__ __forceinline__ unsigned half_pack(float lo, float hi) {
    return (unsigned)__half_as_ushort(__float2half_rn(lo)) | ((unsigned)__half_as_ushort(__float2half_rn(hi)) << 16);
}

__device__ __forceinline__ void ld4(const __half* p, int nvalid, bool vec, float (&o)[4]) {
    if (vec && nvalid == 4) {
        const uint2 t = *reinterpret_cast<const uint2*>(p);
        o[0] = half_lo(t.x); o[1] = half_hi(t.x); o[2] = half_lo(t.y); o[3] = half_hi(t.y);
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] = j < nvalid ? __half2float(p[j]) : 0.0f;
    }
}

__device__ __forceinline__ void st4(float* p, int nvalid, bool vec, const float (&o)[4]) {
    if (vec && nvalid == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (j < nvalid) p[j] = o[j];
    }
}

__device__ __forceinline__ void st4(__half* p, int nvalid, bool vec, const float (&o)[4]) {
    if (vec && nvalid == 4) {
        *reinterpret_cast<uint2*>(p) = make_uint2(half_pack(o[0], o[1]), half_pack(o[2], o[3]));
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (j < nvalid) p[j] = __float2half_rn(o[j]);
    }
}

// ---- WTA key: the largest key is the largest cost, ties broken toward the smallest d ----

__device__ __forceinline__ unsigned long long wta_key(float v, int d) {
    unsigned u = (v == 0.0f) ? 0u : __float_as_uint(v);   // -0 and +0 compare equal
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);        // order-preserving map to uint
    return ((unsigned long long)u << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)d);
}

__device__ __forceinline__ int wta_key_disp(unsigned long long k) {
    return (int)(0xFFFFFFFFu - (unsigned)(k & 0xFFFFFFFFull));
}

// Per-pixel WTA over this thread's 4 disparities and the tq lanes that share the pixel
// (consecutive lanes of one warp); the first of them folds the result into the key map.
// All lanes of the warp must call this together.
__device__ __forceinline__ void wta_fold(const float (&c)[4], int nvalid, int d_first,
                                         int tq, int dq, bool pix_valid,
                                         unsigned long long* key_at) {
    float best = -INFINITY;
    int bd = 0x7FFFFFFF;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (j < nvalid && c[j] > best) { best = c[j]; bd = d_first + j; }
    for (int off = 1; off < tq; off <<= 1) {
        float ob = __shfl_xor_sync(0xFFFFFFFFu, best, off);
        int od = __shfl_xor_sync(0xFFFFFFFFu, bd, off);
        if (ob > best || (ob == best && od < bd)) { best = ob; bd = od; }
    }
    if (dq == 0 && pix_valid && bd != 0x7FFFFFFF) atomicMax(key_at, wta_key(best, bd));
}

// ---- DT line pair: forward then backward recursive pass along a line ------------------
//
// A line of n positions (a row for the horizontal pair, a column for the vertical pair)
// is split into chunks of kL positions; thread (line, chunk k, dq) holds the costs of its
// chunk for disparities 4*dq .. 4*dq+3 of the block's disparity slice in registers.
// e[pos] is the weight of the step (pos-1) -> pos (0 at pos = 0 and for pos >= n), so the
// forward pass uses e[pos] and the backward pass e[pos+1] (the weight W_L(x) of Eq. (3)
// equals W_R(x-1) of Eq. (4): both come from the same two guide pixels, Eq. (11)).
// Each pass is out = s*in + w*out_prev with s = 1-K. A chunk is first scanned with a zero
// carry-in; the carries between chunks are the composition of the chunks' affine maps
// x -> A x + B, computed with a Kogge-Stone scan over the chunks in shared memory; each
// element is then corrected by (product of weights from the chunk edge) * carry.

struct DtShared {
    float* e;      // [lpc][4*plane]    edge weights per line, four-plane layout
    float* acum;   // [lpc][4*plane]    prod_{j=start..pos} e[j]
    float* bcum;   // [lpc][4*plane]    prod_{j=pos..last} e[j+1]
    float* sa;     // [2][lpc][nch]     scan: A part (disparity independent)
    float* sb;     // [2][lpc][nch][ds] scan: B part
    int plane;     // plane length of e/acum/bcum (entries per plane)
};

__host__ __device__ inline size_t dt_shared_bytes(int lpc, int nch, int ds) {
    int plane = plane_of(nch * kL + 1);
    return sizeof(float) * ((size_t)lpc * 4 * plane * 3 + 2ull * lpc * nch +
                            2ull * lpc * nch * ds);
}

__device__ __forceinline__ DtShared dt_carve(float* base, int lpc, int nch, int ds) {
    DtShared s;
    s.plane = plane_of(nch * kL + 1);
    size_t line = 4 * (size_t)s.plane;
    s.e = base;
    s.acum = s.e + lpc * line;
    s.bcum = s.acum + lpc * line;
    s.sa = s.bcum + lpc * line;
    s.sb = s.sa + 2 * lpc * nch;
    return s;
}

// Cooperative load of the edge weights of the block's lines: line li of the block is
// global line (line0 + li); weights at ew[line * ew_line_stride + pos], pos in [1, n).
__device__ __forceinline__ void dt_stage_weights(const DtShared& sm, const float* __restrict__ ew,
                                                 long long ew_line_stride, int line0, int nlines,
                                                 int lpc, int nch, int n) {
    int span = nch * kL + 1;
    for (int t = threadIdx.x; t < lpc * span; t += blockDim.x) {
        int li = t / span, pos = t - li * span;
        int line = line0 + li;
        float w = 0.0f;
        if (line < nlines && pos >= 1 && pos < n) w = __ldg(ew + line * ew_line_stride + pos);
        sm.e[li * 4 * sm.plane + p4(pos, sm.plane)] = w;
    }
}

// Thread dq == 0 of each chunk writes the chunk's cumulative weight products.
__device__ __forceinline__ void dt_chunk_products(const DtShared& sm, int li, int k, int dq) {
    if (dq != 0) return;
    const float* e = sm.e + li * 4 * sm.plane;
    float* ac = sm.acum + li * 4 * sm.plane;
    float* bc = sm.bcum + li * 4 * sm.plane;
    int start = k * kL;
    float a = 1.0f;
#pragma unroll
    for (int i = 0; i < kL; ++i) {
        a *= at4(e, start, i, sm.plane);
        at4(ac, start, i, sm.plane) = a;
    }
    float b = 1.0f;
#pragma unroll
    for (int i = kL - 1; i >= 0; --i) {
        b *= at4(e, start, i + 1, sm.plane);
        at4(bc, start, i, sm.plane) = b;
    }
}

// Inclusive Kogge-Stone scan of affine maps over the chunks of each line, per disparity.
// dir = +1 composes chunk k with chunks < k (forward pass); dir = -1 with chunks > k.
// On return sa/sb[buf] hold the inclusive composites; the function returns buf.
__device__ __forceinline__ int dt_scan(const DtShared& sm, int li, int k, int dq, int nch,
                                       int ds, float A, float (&B)[4], int dir) {
    int buf = 0;
    float* sa = sm.sa;
    float* sb = sm.sb;
    const int lpc_nch = (int)(blockDim.x / ((unsigned)ds / kG));   // lpc * nch
    auto ia = [&](int b, int kk) { return b * lpc_nch + li * nch + kk; };
    auto ib = [&](int b, int kk, int j) { return (ia(b, kk)) * ds + dq * kG + j; };
    if (dq == 0) sa[ia(0, k)] = A;
#pragma unroll
    for (int j = 0; j < 4; ++j) sb[ib(0, k, j)] = B[j];
    __syncthreads();
    for (int off = 1; off < nch; off <<= 1) {
        int nb = k - dir * off;
        if (nb >= 0 && nb < nch) {
            float A2 = sa[ia(buf, nb)];
#pragma unroll
            for (int j = 0; j < 4; ++j) B[j] = fmaf(A, sb[ib(buf, nb, j)], B[j]);
            A *= A2;
        }
        if (dq == 0) sa[ia(buf ^ 1, k)] = A;
#pragma unroll
        for (int j = 0; j < 4; ++j) sb[ib(buf ^ 1, k, j)] = B[j];
        buf ^= 1;
        __syncthreads();
    }
    return buf;
}

// The pair of passes over the costs v of this thread's chunk (in place). All threads of
// the block must call it (it synchronizes the block). li: line within the block.
__device__ __forceinline__ void dt_line_pair(float (&v)[kL][4], const DtShared& sm, int li,
                                             int k, int dq, int nch, int ds, float s) {
    const float* e = sm.e + li * 4 * sm.plane;
    const float* ac = sm.acum + li * 4 * sm.plane;
    const float* bc = sm.bcum + li * 4 * sm.plane;
    const int start = k * kL;
    const int ds_idx = dq * kG;
    const int lpc_nch = (int)(blockDim.x / ((unsigned)ds / kG));

    // forward pass of the chunk with zero carry-in
    float f[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < kL; ++i) {
        float w = at4(e, start, i, sm.plane);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            f[j] = fmaf(w, f[j], s * v[i][j]);
            v[i][j] = f[j];
        }
    }
    float A = at4(ac, start, kL - 1, sm.plane);
    int buf = dt_scan(sm, li, k, dq, nch, ds, A, f, +1);
    float F[4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
        F[j] = k > 0 ? sm.sb[(buf * lpc_nch + li * nch + (k - 1)) * ds + ds_idx + j] : 0.0f;
    __syncthreads();   // the backward scan reuses the buffers

    // forward carry correction, then the backward pass with zero carry-in
    float g[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = kL - 1; i >= 0; --i) {
        float a = at4(ac, start, i, sm.plane);
        float w = at4(e, start, i + 1, sm.plane);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float ft = fmaf(a, F[j], v[i][j]);
            g[j] = fmaf(w, g[j], s * ft);
            v[i][j] = g[j];
        }
    }
    float Bb = at4(bc, start, 0, sm.plane);
    buf = dt_scan(sm, li, k, dq, nch, ds, Bb, g, -1);
    float G[4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
        G[j] = k + 1 < nch ? sm.sb[(buf * lpc_nch + li * nch + (k + 1)) * ds + ds_idx + j] : 0.0f;
#pragma unroll
    for (int i = 0; i < kL; ++i) {
        float b = at4(bc, start, i, sm.plane);
#pragma unroll
        for (int j = 0; j < 4; ++j) v[i][j] = fmaf(b, G[j], v[i][j]);
    }
}

}  // namespace zncc
