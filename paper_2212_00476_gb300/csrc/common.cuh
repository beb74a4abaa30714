// common.cuh -- device helpers shared by the ZNCC / DT / WTA kernels (sm_103a).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

namespace zncc {

// Positions of one line handled by one thread (a "chunk") and disparities per thread.
constexpr int kL = 16;
constexpr int kG = 4;
constexpr unsigned kFull = 0xFFFFFFFFu;

// Shared-memory arrays indexed by a pixel coordinate are stored as four interleaved
// planes, entry idx at (idx & 3) * plane + (idx >> 2): in the access patterns below the
// lanes of a warp share idx & 3 and spread over distinct idx >> 2, which keeps 16-byte
// accesses free of bank conflicts (plain layouts put lanes 16 or 64 entries apart).
__host__ __device__ __forceinline__ int plane_of(int len) { return ((len + 3) / 4 + 31) & ~31; }
__device__ __forceinline__ int p4(int idx, int plane) { return (idx & 3) * plane + (idx >> 2); }
// Entry start + i of a four-plane array, for start a multiple of 4 (i known at compile time).
template <typename T>
__device__ __forceinline__ T& at4(T* base, int start, int i, int plane) {
    return base[(i & 3) * plane + (start >> 2) + (i >> 2)];
}
// Per-position arrays of a DT line (coefficients, multipliers) are chunk-major: the kL entries of a chunk are contiguous and chunks are kCS = kL + 1 entries
// apart. A thread then reaches every entry of its chunk at a constant offset from one
// pointer, and the lanes of a warp, which read the same position of consecutive chunks, fall
// on distinct banks (the padding entry shifts each chunk by one 16-byte group).
constexpr int kCS = kL + 1;
__host__ __device__ __forceinline__ int cpos(int pos) { return (pos >> 4) * kCS + (pos & (kL - 1)); }

// ---- cost-volume element access: 4 consecutive disparities per thread ----------------

__device__ __forceinline__ void fastdt_unpack(unsigned word, float (&o)[4]);

__device__ __forceinline__ void ld4(const float* p, int nvalid, bool vec, float (&o)[4]) {
    if (vec && nvalid == 4) {
        float4 t = *reinterpret_cast<const float4*>(p);
        o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] = j < nvalid ? p[j] : 0.0f;
    }
}

// Half values travel as pairs inside 32-bit words (low half = lower address), converted a
// pair at a time by the half2 intrinsics (one paired conversion each way; converting the
// halves one by one took the slower conversion unit, about 2M instructions more per F16 line
// pass at 1280x384x128). memcpy moves the bits between the word and the half2 without a
// type-punned pointer access. Both directions round exactly as the scalar conversions do.
__device__ __forceinline__ float2 half2_unpack(unsigned w) {
    __half2 h;
    memcpy(&h, &w, sizeof(w));
    return __half22float2(h);
}
__device__ __forceinline__ unsigned half_pack(float lo, float hi) {
    const __half2 h = __floats2half2_rn(lo, hi);
    unsigned w;
    memcpy(&w, &h, sizeof(w));
    return w;
}

__device__ __forceinline__ void ld4(const __half* p, int nvalid, bool vec, float (&o)[4]) {
    if (vec && nvalid == 4) {
        const uint2 t = *reinterpret_cast<const uint2*>(p);
        const float2 a = half2_unpack(t.x), b = half2_unpack(t.y);
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] = j < nvalid ? __half2float(p[j]) : 0.0f;
    }
}

// FastDT codes: four per 32-bit word (4-byte aligned groups of a padded pixel stride), read
// as -E (the caller scales by A_hat / kFastT)
__device__ __forceinline__ void ld4(const uint8_t* p, int nvalid, bool vec, float (&o)[4]) {
    (void)nvalid;
    (void)vec;
    fastdt_unpack(*reinterpret_cast<const unsigned*>(p), o);
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

// ---- FastDT storage (Sec. IV-C): 8-bit codes of near-zero-mean 16-bit costs -------------
// A stored value is E = rint(kFastT * (v(d_arb) - v(d)) / A_hat) as a 16-bit integer
// (values that do no better than d_arb, E >= 0, are 0); its code keeps the six bits next to
// the leading ones of the two's-complement value (bits 14..9, 10..5 or 6..1) and a 2-bit flag
// for the position (01, 10, 11). Four codes (four consecutive disparities) share a 32-bit
// word, the lowest disparity in the lowest byte. The code, branch-free: E < -2048 keeps bits
// 14..9, E < -128 bits 10..5, else bits 6..1.
constexpr float kFastT = 16383.0f;

__device__ __forceinline__ unsigned fastdt_encode(int value) {
    const int t = (value < -2048) + (value < -128);          // 2, 1, 0
    const int low = 1 + 4 * t;                                // lowest kept bit: 9, 5, 1
    const unsigned code = (((unsigned)(value >> low) & 0x3Fu) << 2) | (unsigned)(3 - t);
    return value < 0 ? code : 0u;
}

// E from the values, normalised and scaled by kFastT (at least -32768): ref - v rounded to the
// nearest integer, ties to even, by adding 1.5 * 2^23 (exact for |E| < 2^22; larger E is
// positive and codes to 0 either way).
__device__ __forceinline__ int fastdt_quantize(float ref, float v) {
    const float y = fmaxf(ref - v, -32768.0f);
    return __float_as_int(y + 12582912.0f) - 0x4B400000;
}

// four values of E -> a word of four codes (entries j >= nvalid code 0)
__device__ __forceinline__ unsigned fastdt_pack_codes(const int (&E)[4], int nvalid) {
    unsigned c[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) c[j] = j < nvalid ? fastdt_encode(E[j]) : 0u;
    return __byte_perm(__byte_perm(c[0], c[1], 0x0040), __byte_perm(c[2], c[3], 0x0040), 0x5410);
}

// four values and the reference (normalised, scaled by kFastT) -> a word of four codes
__device__ __forceinline__ unsigned fastdt_pack(const float (&v)[4], float ref, int nvalid) {
    int E[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) E[j] = fastdt_quantize(ref, v[j]);
    return fastdt_pack_codes(E, nvalid);
}

// A word of four codes -> -E of each as an exact float (code 0 -> 0; larger is better). A code
// with six bits s and flag f stands for E = (s - 64) * 2^low, low = 9, 5, 1 for f = 1, 2, 3:
// the six bits in place, ones above them, zeros below. Per byte, 64 - s becomes a float by
// placing it in the mantissa of 2^23, and 2^low comes from a four-entry table of exponent
// bytes indexed by f (2^9, 2^5, 2^1, and 0 for f = 0).
__device__ __forceinline__ void fastdt_unpack(unsigned word, float (&o)[4]) {
    const unsigned F = word & 0x03030303u;
    const unsigned M = 0x40404040u - ((word >> 2) & 0x3F3F3F3Fu);
    const unsigned sel[4] = {((F << 12) & 0x3000u) | 0x444u, ((F << 4) & 0x3000u) | 0x444u,
                             ((F >> 4) & 0x3000u) | 0x444u, ((F >> 12) & 0x3000u) | 0x444u};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float m = __int_as_float(__byte_perm(M, 0x4B000000u, 0x7440u | j)) - 8388608.0f;
        o[j] = m * __int_as_float(__byte_perm(0x40424400u, 0u, sel[j]));
    }
}

__device__ __forceinline__ void lds4(const uint8_t* p, float (&o)[4]) {
    fastdt_unpack(*reinterpret_cast<const unsigned*>(p), o);
}

// ---- asynchronous global -> shared copies (cp.async) ------------------------------------
// A copy of `bytes` from global to shared memory that bypasses registers; with valid ==
// false nothing is read and the destination is zero-filled. Each thread waits for its own
// copies (cp.async.wait_group), so a thread that reads back only what it copied needs no
// block barrier.
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int src_bytes = valid ? BYTES : 0;
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes)
                     : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(s), "l"(gmem), "n"(BYTES),
                     "r"(src_bytes)
                     : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// ---- bulk asynchronous copies (the TMA unit) completing on a shared-memory mbarrier ----
// One thread arms the barrier with the byte count it expects and issues the copies; every
// thread then waits for the barrier's phase to complete. Destination and source addresses and
// the size of each copy must be multiples of 16 bytes.
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar)) : "memory");
}
// A 3-D box of a tensor map (TMA) into shared memory (128-byte aligned), completing its bytes
// on the mbarrier. Coordinates are element indices, innermost first; parts of the box outside
// the tensor read as zero.
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int c0, int c1, int c2,
                                            unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_addr(dst)), "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
        : "memory");
}
// Orders this thread's earlier generic-proxy accesses of shared memory before later bulk copies
// into it (the copies run in the async proxy).
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
// Waits for the phase of the given parity to complete, at most `limit` polls; false if it did
// not complete in time.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, unsigned limit) {
    const unsigned a = smem_addr(bar);
    for (unsigned it = 0; it < limit; ++it) {
        unsigned done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

// The four consecutive disparities of one element group, read back from shared memory.
__device__ __forceinline__ void lds4(const float* p, float (&o)[4]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}
__device__ __forceinline__ void lds4(const __half* p, float (&o)[4]) {
    const uint2 t = *reinterpret_cast<const uint2*>(p);
    const float2 a = half2_unpack(t.x), b = half2_unpack(t.y);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}

// ---- programmatic dependent launch -------------------------------------------------------
// A kernel launched with programmatic stream serialization may start while the kernel before
// it on the stream is finishing; griddep_wait() returns once that kernel has completed and its
// memory is visible, so every kernel calls it before touching global memory. A kernel calls
// griddep_launch_dependents() when its remaining work no longer needs the whole device, so
// that the next kernel's launch overlaps its tail. Both are no-ops without the attribute.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;"); }

// ---- thread-block clusters: a DT line split across the CTAs of a cluster ---------------
// The CTA's rank in its cluster (0 for a launch without clusters).
__device__ __forceinline__ int cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return (int)r;
}
// Barrier over every thread of the cluster; shared-memory writes before it (local or to other
// CTAs of the cluster) are visible to every thread of the cluster after it.
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// The barrier between the phases of a line pair: the block's, or the cluster's when the line
// spans cs > 1 CTAs.
__device__ __forceinline__ void line_sync(int cs) {
    if (cs > 1) cluster_sync_all();
    else __syncthreads();
}
// Stores to the same shared-memory offset in the CTA of the given rank (distributed shared
// memory).
__device__ __forceinline__ unsigned cluster_addr(const void* p, int rank) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_rank(float* p, int rank, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(cluster_addr(p, rank)), "f"(v) : "memory");
}
__device__ __forceinline__ void st_rank(float4* p, int rank, float4 v) {
    asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(cluster_addr(p, rank)), "f"(v.x),
                 "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

// ---- WTA (Eq. (WTA1)): the largest cost wins, ties go to the smallest d ----------------

// ---- DT line pair: forward then backward recursive pass along a line ------------------
//
// A line (a row for the horizontal pair, a column for the vertical pair) is split into
// chunks of kL positions; thread (chunk k, dq) holds the costs of its chunk for 4 disparities
// in registers. The pair of Eqs. (3)-(4) (or (5)-(6)) in the scaled form is
//   f(p) = s c(p) + w(p) f(p-1),   g(p) = s f(p) + w(p+1) g(p+1),   s = 1 - K,
// w(p) the weight of the step p-1 -> p (Eq. (11)). It is computed in the literal form
// u = c + w u_prev, h = u + w' h_next, which is the same chain divided by s^2 (both passes
// are linear), and scaled by s^2 at the end. Each chunk is swept with a zero carry-in; the
// carries are compositions of the chunks' affine maps x -> A x + B (A = product of the
// chunk's weights), scanned across the chunks of a warp with shuffles and across the warps
// of a line through shared memory.
//
// Per-position coefficients (float4, disparity independent, computed once per image):
//   x = w(p), y = A(p) = prod_{j = chunk start .. p} w(j),
//   z = w(p+1), w = B(p) = prod_{j = p .. chunk end} w(j+1),
// zero past the line end, so that padded chunks carry nothing.
//
// co: the kL coefficients of this thread's chunk in shared memory (co[i] for position i of
// the chunk); sa/sb: the line's scan buffers, 2 * nwl * tq entries each; wl / nwl: this
// thread's warp within the line and the warps per line. The result is scaled by s2 =
// (1-K)^2, or per position by mul[i].y when mul (the chunk's multipliers) is given; SCALE
// false leaves it unscaled (a positive factor per pixel, which a WTA that follows ignores).
// after_forward() runs once the forward sweep has consumed the input values (the caller may
// then overwrite where they came from). Synchronizes the block twice; threads with active ==
// false (whole warps) only take part in the barriers.
// A line may span the cs CTAs of a thread-block cluster: wl / nwl then number the warps of
// the whole line, each warp's chunk map is stored into the scan buffers of every CTA of the
// cluster, and the two barriers are the cluster's.
struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

// The output scale of a position: the y of a multiplier pair, or the value itself.
__device__ __forceinline__ float out_scale(const float2& m) { return m.y; }
__device__ __forceinline__ float out_scale(float m) { return m; }

// o[j] = fmaf(s, y[j], z[j]) and x[j] = s * x[j] for the four disparities of a position (o may
// be y or z). PACKED: as two packed pairs (__ffma2_rn / __fmul2_rn, sm_100 and later), which
// round each component exactly as fmaf and a single multiply do: the same bits in half the
// floating-point instructions.
template <bool PACKED>
__device__ __forceinline__ void fma4(float s, const float (&y)[4], const float (&z)[4], float (&o)[4]) {
    if constexpr (PACKED) {
        const float2 ss = make_float2(s, s);
        const float2 r0 = __ffma2_rn(ss, make_float2(y[0], y[1]), make_float2(z[0], z[1]));
        const float2 r1 = __ffma2_rn(ss, make_float2(y[2], y[3]), make_float2(z[2], z[3]));
        o[0] = r0.x; o[1] = r0.y; o[2] = r1.x; o[3] = r1.y;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] = fmaf(s, y[j], z[j]);
    }
}
template <bool PACKED>
__device__ __forceinline__ void mul4(float s, float (&x)[4]) {
    if constexpr (PACKED) {
        const float2 ss = make_float2(s, s);
        const float2 r0 = __fmul2_rn(ss, make_float2(x[0], x[1]));
        const float2 r1 = __fmul2_rn(ss, make_float2(x[2], x[3]));
        x[0] = r0.x; x[1] = r0.y; x[2] = r1.x; x[3] = r1.y;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) x[j] = s * x[j];
    }
}

// PACKED: the sweeps, scans and carries use the packed pairs of fma4 / mul4 (the DT line
// passes: 15% fewer instructions; in the cost kernel's fused pair the packed form measured
// slower, 117 -> 124 us at 1280x384x128, so that one keeps the scalar form).
template <bool SCALE = true, bool PACKED = false, typename Hook = NoHook, typename MulT = float2>
__device__ __forceinline__ void dt_pair(float (&v)[kL][4], const float4* __restrict__ co, int tq, int dq,
                                        int lane, int wl, int nwl, float* sa, float4* sb, float s2,
                                        const MulT* __restrict__ mul = nullptr,
                                        Hook after_forward = Hook(), bool active = true, int cs = 1) {
    float A = 0.f, Ae = 1.f;
    float B[4], Be[4], F[4], G[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) B[j] = Be[j] = F[j] = G[j] = 0.f;

    // ---- phase 1: forward sweep of the chunk with zero carry-in, warp scan of its map ----
    if (active) {
        float u[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < kL; ++i) {
            const float w = co[i].x;
            fma4<PACKED>(w, u, v[i], u);
#pragma unroll
            for (int j = 0; j < 4; ++j) v[i][j] = u[j];
        }
    }
    after_forward();
    if (active) {
        A = co[kL - 1].y;
#pragma unroll
        for (int j = 0; j < 4; ++j) B[j] = v[kL - 1][j];
        // rounds at lane offsets tq, 2 tq, .. 16, unrolled with constant offsets
#pragma unroll
        for (int r5 = 0; r5 < 5; ++r5) {
            const int off = 1 << r5;
            if (off < tq) continue;
            const float A2 = __shfl_up_sync(kFull, A, off);
            float B2[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) B2[j] = __shfl_up_sync(kFull, B[j], off);
            if (lane >= off) {
                fma4<PACKED>(A, B2, B, B);
                A *= A2;
            }
        }
        Ae = __shfl_up_sync(kFull, A, tq);
#pragma unroll
        for (int j = 0; j < 4; ++j) Be[j] = __shfl_up_sync(kFull, B[j], tq);
        if (lane < tq) {
            Ae = 1.0f;
            Be[0] = Be[1] = Be[2] = Be[3] = 0.0f;
        }
        if (lane >= 32 - tq) {
            const float4 b4 = make_float4(B[0], B[1], B[2], B[3]);
            if (cs == 1) {
                sa[wl * tq + dq] = A;
                sb[wl * tq + dq] = b4;
            } else {
                for (int r = 0; r < cs; ++r) {
                    st_rank(sa + wl * tq + dq, r, A);
                    st_rank(sb + wl * tq + dq, r, b4);
                }
            }
        }
    }
    line_sync(cs);

    // ---- phase 2: carry from the warps before, corrected forward values, backward sweep ----
    if (active) {
        // the warps before: a short loop, not unrolled (a few iterations; unrolling it cost
        // issue slots and registers)
#pragma unroll 1
        for (int w2 = 0; w2 < wl; ++w2) {
            const float a2 = sa[w2 * tq + dq];
            const float4 b2 = sb[w2 * tq + dq];
            const float b4[4] = {b2.x, b2.y, b2.z, b2.w};
            fma4<PACKED>(a2, F, b4, F);
        }
        fma4<PACKED>(Ae, F, Be, F);
        float h[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int i = kL - 1; i >= 0; --i) {
            const float4 c = co[i];
            if constexpr (PACKED) {
                float ft[4];
                fma4<true>(c.y, F, v[i], ft);
                fma4<true>(c.z, h, ft, h);
#pragma unroll
                for (int j = 0; j < 4; ++j) v[i][j] = h[j];
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float ft = fmaf(c.y, F[j], v[i][j]);
                    h[j] = fmaf(c.z, h[j], ft);
                    v[i][j] = h[j];
                }
            }
        }
        A = co[0].w;
#pragma unroll
        for (int j = 0; j < 4; ++j) B[j] = h[j];
#pragma unroll
        for (int r5 = 0; r5 < 5; ++r5) {
            const int off = 1 << r5;
            if (off < tq) continue;
            const float A2 = __shfl_down_sync(kFull, A, off);
            float B2[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) B2[j] = __shfl_down_sync(kFull, B[j], off);
            if (lane + off < 32) {
                fma4<PACKED>(A, B2, B, B);
                A *= A2;
            }
        }
        Ae = __shfl_down_sync(kFull, A, tq);
#pragma unroll
        for (int j = 0; j < 4; ++j) Be[j] = __shfl_down_sync(kFull, B[j], tq);
        if (lane >= 32 - tq) {
            Ae = 1.0f;
            Be[0] = Be[1] = Be[2] = Be[3] = 0.0f;
        }
        if (lane < tq) {
            const float4 b4 = make_float4(B[0], B[1], B[2], B[3]);
            if (cs == 1) {
                sa[(nwl + wl) * tq + dq] = A;
                sb[(nwl + wl) * tq + dq] = b4;
            } else {
                for (int r = 0; r < cs; ++r) {
                    st_rank(sa + (nwl + wl) * tq + dq, r, A);
                    st_rank(sb + (nwl + wl) * tq + dq, r, b4);
                }
            }
        }
    }
    line_sync(cs);

    // ---- phase 3: carry from the warps after, backward correction, scale ----
    if (active) {
#pragma unroll 1
        for (int w2 = nwl - 1; w2 > wl; --w2) {
            const float a2 = sa[(nwl + w2) * tq + dq];
            const float4 b2 = sb[(nwl + w2) * tq + dq];
            const float b4[4] = {b2.x, b2.y, b2.z, b2.w};
            fma4<PACKED>(a2, G, b4, G);
        }
        fma4<PACKED>(Ae, G, Be, G);
        if (SCALE && (mul || s2 != 1.0f)) {
#pragma unroll
            for (int i = 0; i < kL; ++i) {
                const float b = co[i].w;
                const float m = mul ? out_scale(mul[i]) : s2;
                fma4<PACKED>(b, G, v[i], v[i]);
                mul4<PACKED>(m, v[i]);
            }
        } else {                            // unscaled (s2 == 1: the caller runs the literal chain)
#pragma unroll
            for (int i = 0; i < kL; ++i) {
                const float b = co[i].w;
                fma4<PACKED>(b, G, v[i], v[i]);
            }
        }
    }
}

// One round of the transposed lane reduction of WtaRegs::merge: of the P (value, d) entries a
// lane holds, it keeps the lower half (upper == false) or the upper half and sends the other
// half to its partner lane (lane ^ off), merging what it receives: larger value, then smaller d.
template <int P>
__device__ __forceinline__ void wta_halve(float (&bv)[kL], int (&bd)[kL], bool upper, int off) {
#pragma unroll
    for (int k = 0; k < P / 2; ++k) {
        const float ov = __shfl_xor_sync(kFull, upper ? bv[k] : bv[k + P / 2], off);
        const int od = __shfl_xor_sync(kFull, upper ? bd[k] : bd[k + P / 2], off);
        float mv = upper ? bv[k + P / 2] : bv[k];
        int md = upper ? bd[k + P / 2] : bd[k];
        if (ov > mv || (ov == mv && od < md)) {
            mv = ov;
            md = od;
        }
        bv[k] = mv;
        bd[k] = md;
    }
}

// ---- per-thread WTA running best over the slices a block visits, in registers -----------
// rv[i]: best value of position i over this thread's disparities so far; rd: the matching
// disparities as 16-bit fields, two per word. Ties keep the smaller d (slices arrive in
// increasing d, and a later equal value does not replace an earlier one).
struct WtaRegs {
    float rv[kL];
    unsigned rd[kL / 2];
    __device__ __forceinline__ void reset() {
#pragma unroll
        for (int i = 0; i < kL; ++i) rv[i] = -INFINITY;
#pragma unroll
        for (int i = 0; i < kL / 2; ++i) rd[i] = 0xFFFFFFFFu;
    }
    __device__ __forceinline__ void fold(const float (&v)[kL][4], int nvalid, int d_first) {
        if (nvalid == 4) {
            fold4(v, d_first);
            return;
        }
#pragma unroll
        for (int i = 0; i < kL; ++i) {
            float m = -INFINITY;
            int jj = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (j < nvalid && v[i][j] > m) { m = v[i][j]; jj = j; }
            if (m > rv[i]) {
                rv[i] = m;
                const unsigned d = (unsigned)(d_first + jj) & 0xFFFFu;
                rd[i >> 1] = (i & 1) ? ((rd[i >> 1] & 0x0000FFFFu) | (d << 16)) : ((rd[i >> 1] & 0xFFFF0000u) | d);
            }
        }
    }
    // A whole group of four disparities: the group's maximum by three fmaxf, its index from
    // the pair compares (the first pair wins a tie between the pairs, the first element a tie
    // within a pair: the smallest d), and the 16-bit disparity inserted by a byte permute.
    __device__ __forceinline__ void fold4(const float (&v)[kL][4], int d_first) {
#pragma unroll
        for (int i = 0; i < kL; ++i) {
            const float m01 = fmaxf(v[i][0], v[i][1]), m23 = fmaxf(v[i][2], v[i][3]);
            const bool lo = m01 >= m23;
            const float m = lo ? m01 : m23;
            const int jj = lo ? (v[i][0] >= v[i][1] ? 0 : 1) : (v[i][2] >= v[i][3] ? 2 : 3);
            const bool better = m > rv[i];
            rv[i] = better ? m : rv[i];
            const unsigned d = (unsigned)(d_first + jj);
            const unsigned ins = (i & 1) ? __byte_perm(rd[i >> 1], d, 0x5410) : __byte_perm(rd[i >> 1], d, 0x3254);
            rd[i >> 1] = better ? ins : rd[i >> 1];
        }
    }
    // Reduces the running bests of the tq lanes of a chunk (consecutive lanes, tq a power of two
    // up to 16) by halving rounds: after them lane dq holds the bests of kL / tq positions of the
    // chunk, which it passes to emit(position in the chunk, value, d); every lane emits a share.
    template <typename Emit>
    __device__ __forceinline__ void merge(int tq, int lane, Emit emit) const {
        float bv[kL];
        int bd[kL];
#pragma unroll
        for (int i = 0; i < kL; ++i) {
            const float2 e = entry(i);
            bv[i] = e.x;
            bd[i] = __float_as_int(e.y);
        }
        int base = 0, held = kL;
        if (tq > 1) { const bool u = (lane & 1) != 0; wta_halve<16>(bv, bd, u, 1); base += u ? 8 : 0; held = 8; }
        if (tq > 2) { const bool u = (lane & 2) != 0; wta_halve<8>(bv, bd, u, 2); base += u ? 4 : 0; held = 4; }
        if (tq > 4) { const bool u = (lane & 4) != 0; wta_halve<4>(bv, bd, u, 4); base += u ? 2 : 0; held = 2; }
        if (tq > 8) { const bool u = (lane & 8) != 0; wta_halve<2>(bv, bd, u, 8); base += u ? 1 : 0; held = 1; }
#pragma unroll
        for (int k = 0; k < kL; ++k)
            if (k < held) emit(base + k, bv[k], bd[k]);
    }
    __device__ __forceinline__ float2 entry(int i) const {
        const unsigned d = (i & 1) ? (rd[i >> 1] >> 16) : (rd[i >> 1] & 0xFFFFu);
        return make_float2(rv[i], __int_as_float(d == 0xFFFFu ? 0x7FFFFFFF : (int)d));
    }
};

// A (value, d) pair as a 64-bit key whose unsigned order is the WTA order: larger values
// first, then smaller d. High word: the float's bits made order-preserving; low word: ~d.
__device__ __forceinline__ unsigned long long wta_key(float v, int d) {
    const unsigned u = __float_as_uint(v);
    const unsigned hi = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((unsigned long long)hi << 32) | (unsigned)(~(unsigned)d);
}
__device__ __forceinline__ uint16_t wta_key_disparity(unsigned long long key) {
    return (uint16_t)(~(unsigned)key);
}

// Shared-memory bytes of one line's scan buffers.
__host__ __device__ inline size_t dt_scan_bytes(int nwl, int tq) {
    return (size_t)2 * nwl * tq * (sizeof(float4) + sizeof(float));
}

}  // namespace zncc
