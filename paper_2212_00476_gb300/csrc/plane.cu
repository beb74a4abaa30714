// plane.cu -- the plane-resident fused path: ZNCC cost (Eq. (2)), every DT pass pair
// (Eqs. (3)-(6), 2 x iters pairs) and the WTA (Eq. (WTA1)) of one disparity plane without the
// cost volume ever leaving shared memory.
//
// A thread-block cluster of cs CTAs owns one plane C(., ., d) at a time: CTA q holds the rows
// [q hb, (q+1) hb) of it (hb = ceil(H / cs) <= BANDMAX, the size class's) as FP32 in shared
// memory, with the left and right image rows of its band and r halo rows above and below
// (clamped to the image, as every window access is). Per disparity d:
//   cost      column sums of L(x', .) R(x' - d, .) over the 2r+1 rows of each window, slid
//             down the band four rows at a time, then the row sum of 2r+1 of them and Eq. (2)
//             with the window statistics of k_window_stats, which stream into shared memory
//             by cp.async while the column sums run (exact int32 numerator, the same FP32
//             expression as the other cost kernels, so the values agree bit for bit);
//   H pairs   a warp per row, a segment of the row per lane in registers: the forward pass
//             as affine maps composed by a warp scan, then the values from the true carry;
//             the backward pass likewise from the right; the result scaled by (1 - K)^2;
//   V pairs   a thread per column, the band's run of it in registers; the maps of the bands
//             are composed across the cluster through distributed shared memory (one cluster
//             barrier per direction);
//   WTA       the last V pair writes nothing back: each value goes into the pixel's 64-bit
//             key (value, d) by atomicMax, which k_wta_finish turns into the disparity.
// The DT weights K exp(-|dG| / sigma_r) depend only on the integer |dG| of the uint8 guide
// (the left image), so a 256-entry table of the same expression as k_dt_coef gives them.
// Clusters take the disparities (over all pairs of the launch) round robin.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace zncc {

namespace {

__device__ __forceinline__ float2 ld_rank(const float2* p, int rank) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];"
                 : "=f"(v.x), "=f"(v.y)
                 : "r"(cluster_addr(p, rank))
                 : "memory");
    return v;
}

__device__ __forceinline__ float weight(const float* lut, int a, int b) { return lut[abs(a - b)]; }


}  // namespace

template <int SEGMAX, int BANDMAX, int MINB>
__global__ void __launch_bounds__(kPlaneThreads, MINB) k_plane(const __grid_constant__ PlaneBatch b) {
    extern __shared__ __align__(16) unsigned char psm[];
    griddep_wait();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cs = b.cs;
    const int q = cs > 1 ? cluster_rank() : 0;
    const int cid = blockIdx.x / cs;
    float* lut = reinterpret_cast<float*>(psm);
    for (int i = tid; i < 256; i += kPlaneThreads) lut[i] = b.K * expf(-(float)i * b.inv_sr255);

    int staged = -1;                          // the pair whose image rows are in shared memory
    for (int item = cid; item < b.total_items; item += b.nclusters) {
        int pi = 0;
        while (pi + 1 < b.npairs && item >= b.p[pi + 1].item0) ++pi;
        const PlaneArgs& a = b.p[pi];
        const int d = item - a.item0;
        const int W = a.W, H = a.H, r = a.r;
        const PlaneLayout Ly = plane_layout(W, H, r, cs);
        const int hb = Ly.hb, wb = Ly.wb, vw = Ly.vw;
        const int y0 = q * hb, hq = max(0, min(hb, H - y0));    // rows of this CTA's band
        float* plane = reinterpret_cast<float*>(psm + Ly.plane);
        int* vt = reinterpret_cast<int*>(psm + Ly.vt);
        float2* cf = reinterpret_cast<float2*>(psm + Ly.cf);
        float2* cb = reinterpret_cast<float2*>(psm + Ly.cb);
        uint8_t* lb = psm + Ly.lb;            // rows y0 - r .. y0 + hb + r - 1 (clamped)
        uint8_t* rb = psm + Ly.rb;
        if (pi != staged) {
            __syncthreads();                  // the previous pair's rows are no longer read
            const int nrows = hb + 2 * r;
            const uintptr_t al = reinterpret_cast<uintptr_t>(a.left) | reinterpret_cast<uintptr_t>(a.right) |
                                 (uintptr_t)a.pitch | (uintptr_t)W;
            if ((al & 15) == 0 || (al & 3) == 0) {   // copies of 16 or 4 bytes, straight to shared memory
                const int sh = (al & 15) == 0 ? 4 : 2, gpr = W >> sh, ng = nrows * gpr;
                for (int e = tid; e < ng; e += kPlaneThreads) {
                    const int k = e / gpr, x = (e - k * gpr) << sh;
                    const size_t src = (size_t)min(max(y0 - r + k, 0), H - 1) * a.pitch + x;
                    if (sh == 4) {
                        cp_async<16>(lb + k * wb + x, a.left + src, true);
                        cp_async<16>(rb + k * wb + x, a.right + src, true);
                    } else {
                        cp_async<4>(lb + k * wb + x, a.left + src, true);
                        cp_async<4>(rb + k * wb + x, a.right + src, true);
                    }
                }
                cp_async_commit();
                cp_async_wait<0>();
            } else {
                for (int e = tid; e < nrows * W; e += kPlaneThreads) {
                    const int k = e / W, x = e - k * W;
                    const size_t src = (size_t)min(max(y0 - r + k, 0), H - 1) * a.pitch + x;
                    lb[k * wb + x] = a.left[src];
                    rb[k * wb + x] = a.right[src];
                }
            }
            staged = pi;
            __syncthreads();
        }

        // ---- cost: C(x, y0 + t) for t in [0, hq) ----
        const unsigned n = (unsigned)((2 * r + 1) * (2 * r + 1));
        int vs[kPlaneColsPerThread];
#pragma unroll
        for (int j = 0; j < kPlaneColsPerThread; ++j) vs[j] = 0;
        int2* stL = reinterpret_cast<int2*>(psm + Ly.st);      // [kPlaneTileRows][W]
        int2* stR = stL + kPlaneTileRows * W;
        for (int t0 = 0; t0 < hq; t0 += kPlaneTileRows) {
            const int tr = min(kPlaneTileRows, hq - t0);
            // the tile's window statistics stream into shared memory while the column sums run
            for (int tt = 0; tt < tr; ++tt) {
                const int y = y0 + t0 + tt;
                const int2* gl = a.statsL + (size_t)y * W;
                const int2* gr = a.statsR + (size_t)y * (W + a.D - 1) + (a.D - 1 - d);
                for (int x = tid; x < W; x += kPlaneThreads) {
                    cp_async<8>(stL + tt * W + x, gl + x, true);
                    cp_async<8>(stR + tt * W + x, gr + x, true);
                }
            }
            cp_async_commit();
#pragma unroll
            for (int j = 0; j < kPlaneColsPerThread; ++j) {
                const int u = tid + j * kPlaneThreads;      // column x' = u - r of the window sums
                if (u < vw) {
                    const int uc = min(max(u - r, 0), W - 1), vc = min(max(u - r - d, 0), W - 1);
                    int s = vs[j];
                    for (int t = t0; t < t0 + tr; ++t) {
                        if (t == 0) {
                            s = 0;
                            for (int k = 0; k <= 2 * r; ++k) s += (int)lb[k * wb + uc] * (int)rb[k * wb + vc];
                        } else {
                            s += (int)lb[(t + 2 * r) * wb + uc] * (int)rb[(t + 2 * r) * wb + vc] -
                                 (int)lb[(t - 1) * wb + uc] * (int)rb[(t - 1) * wb + vc];
                        }
                        vt[(t - t0) * vw + u] = s;
                    }
                    vs[j] = s;
                }
            }
            cp_async_wait<0>();
            __syncthreads();
            for (int tt = 0; tt < tr; ++tt)
                for (int x = tid; x < W; x += kPlaneThreads) {
                    const int* v = vt + tt * vw + x;
                    unsigned P = 0u;
                    for (int i = 0; i <= 2 * r; ++i) P += (unsigned)v[i];
                    const int2 sl = stL[tt * W + x], sr = stR[tt * W + x];
                    const unsigned num = n * P - (unsigned)sl.x * (unsigned)sr.x;
                    plane[(t0 + tt) * W + x] = (float)(int)num * __int_as_float(sl.y) * __int_as_float(sr.y);
                }
            __syncthreads();
        }

        // ---- DT pass pairs: 1, 3, ... along rows, 2, 4, ... along columns ----
        const float s2 = b.s2;
        const int npairs = 2 * b.iters;
        const uint8_t* G = lb + r * wb;       // guide row of band row t: G + t * wb
        for (int p = 1; p <= npairs; ++p) {
            if (p & 1) {
                const int seg = ((W + 31) / 32) | 1;
                const int p0 = min(W, lane * seg), len = min(W, p0 + seg) - p0;
                for (int t = warp; t < hq; t += kPlaneWarps) {
                    float* row = plane + t * W;
                    const uint8_t* g = G + t * wb;
                    float xv[SEGMAX], w[SEGMAX + 1];     // w[k]: the step p0+k-1 -> p0+k
                    int gp = g[max(p0 - 1, 0)];
#pragma unroll
                    for (int k = 0; k <= SEGMAX; ++k) {
                        if (k <= len) {
                            const int pos = p0 + k;
                            const int gc = pos < W ? g[pos] : gp;
                            w[k] = (pos >= 1 && pos < W) ? weight(lut, gc, gp) : 0.0f;
                            gp = gc;
                        }
                        if (k < len) xv[k] = row[p0 + k];
                    }
                    // forward: f(x) = c(x) + w(x) f(x-1)
                    float u = 0.0f, P = 1.0f;
#pragma unroll
                    for (int k = 0; k < SEGMAX; ++k)
                        if (k < len) {
                            u = fmaf(w[k], u, xv[k]);
                            P *= w[k];
                        }
                    for (int off = 1; off < 32; off <<= 1) {
                        const float P2 = __shfl_up_sync(kFull, P, off), u2 = __shfl_up_sync(kFull, u, off);
                        if (lane >= off) {
                            u = fmaf(P, u2, u);
                            P *= P2;
                        }
                    }
                    float c = __shfl_up_sync(kFull, u, 1);
                    if (lane == 0) c = 0.0f;
#pragma unroll
                    for (int k = 0; k < SEGMAX; ++k)
                        if (k < len) {
                            c = fmaf(w[k], c, xv[k]);
                            xv[k] = c;
                        }
                    // backward: h(x) = f(x) + w(x+1) h(x+1)
                    u = 0.0f;
                    P = 1.0f;
#pragma unroll
                    for (int k = SEGMAX - 1; k >= 0; --k)
                        if (k < len) {
                            u = fmaf(w[k + 1], u, xv[k]);
                            P *= w[k + 1];
                        }
                    for (int off = 1; off < 32; off <<= 1) {
                        const float P2 = __shfl_down_sync(kFull, P, off), u2 = __shfl_down_sync(kFull, u, off);
                        if (lane + off < 32) {
                            u = fmaf(P, u2, u);
                            P *= P2;
                        }
                    }
                    c = __shfl_down_sync(kFull, u, 1);
                    if (lane == 31) c = 0.0f;
#pragma unroll
                    for (int k = SEGMAX - 1; k >= 0; --k)
                        if (k < len) {
                            c = fmaf(w[k + 1], c, xv[k]);
                            row[p0 + k] = s2 * c;
                        }
                }
            } else {
                const bool wta = p == npairs;
                for (int x0 = 0; x0 < W; x0 += kPlaneThreads) {    // the same count in every CTA
                    const int x = x0 + tid;
                    const bool col = x < W, live = col && hq > 0;
                    float xv[BANDMAX], w[BANDMAX + 1];   // w[k]: the step y0+k-1 -> y0+k
                    if (live) {
                        int gp = G[-wb + x];
#pragma unroll
                        for (int k = 0; k <= BANDMAX; ++k) {
                            if (k <= hq) {
                                const int y = y0 + k;
                                const int gc = y < H ? G[k * wb + x] : gp;
                                w[k] = (y >= 1 && y < H) ? weight(lut, gc, gp) : 0.0f;
                                gp = gc;
                            }
                            if (k < hq) xv[k] = plane[k * W + x];
                        }
                    }
                    float u = 0.0f, P = 1.0f;
                    if (live) {
#pragma unroll
                        for (int k = 0; k < BANDMAX; ++k)
                            if (k < hq) {
                                u = fmaf(w[k], u, xv[k]);
                                P *= w[k];
                            }
                    }
                    float c = 0.0f;
                    if (cs > 1) {
                        if (col) cf[x] = make_float2(u, P);
                        cluster_sync_all();
                        if (live)
                            for (int qq = 0; qq < q; ++qq) {
                                const float2 m = ld_rank(cf + x, qq);
                                c = fmaf(m.y, c, m.x);
                            }
                    }
                    if (live) {
#pragma unroll
                        for (int k = 0; k < BANDMAX; ++k)
                            if (k < hq) {
                                c = fmaf(w[k], c, xv[k]);
                                xv[k] = c;
                            }
                    }
                    u = 0.0f;
                    P = 1.0f;
                    if (live) {
#pragma unroll
                        for (int k = BANDMAX - 1; k >= 0; --k)
                            if (k < hq) {
                                u = fmaf(w[k + 1], u, xv[k]);
                                P *= w[k + 1];
                            }
                    }
                    c = 0.0f;
                    if (cs > 1) {
                        if (col) cb[x] = make_float2(u, P);
                        cluster_sync_all();
                        if (live)
                            for (int qq = cs - 1; qq > q; --qq) {
                                const float2 m = ld_rank(cb + x, qq);
                                c = fmaf(m.y, c, m.x);
                            }
                    }
                    if (live) {
#pragma unroll
                        for (int k = BANDMAX - 1; k >= 0; --k)
                            if (k < hq) {
                                c = fmaf(w[k + 1], c, xv[k]);
                                const float v = s2 * c;
                                if (wta) atomicMax(a.keys + (size_t)(y0 + k) * W + x, wta_key(v, d));
                                else plane[k * W + x] = v;
                            }
                    }
                }
            }
            __syncthreads();
        }
    }
    if (cs > 1) cluster_sync_all();           // no CTA leaves while another may read its carries
}

namespace {
using PlaneKernel = void (*)(PlaneBatch);
PlaneKernel plane_kernel(int cls) {
    switch (cls) {
        case 0: return k_plane<kPlaneSegMaxOf[0], kPlaneBandMaxOf[0], kPlaneMinBlocksOf[0]>;
        case 1: return k_plane<kPlaneSegMaxOf[1], kPlaneBandMaxOf[1], kPlaneMinBlocksOf[1]>;
        default: return k_plane<kPlaneSegMaxOf[2], kPlaneBandMaxOf[2], kPlaneMinBlocksOf[2]>;
    }
}
}  // namespace

cudaError_t plane_max_clusters(int cls, int cs, size_t smem, int* clusters) {
    if (cls < 0 || cls >= kPlaneClasses) return cudaErrorInvalidValue;
    PlaneKernel fn = plane_kernel(cls);
    cudaError_t e = set_max_smem((const void*)fn, smem);
    if (e != cudaSuccess) return e;
    if (cs == 1) {
        int bps = 0, dev = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, kPlaneThreads, smem);
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        *clusters = bps * sms;
        return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(kPlaneThreads);
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

cudaError_t launch_plane(const PlaneBatch& b, int cls, size_t smem, cudaStream_t st) {
    if (cls < 0 || cls >= kPlaneClasses) return cudaErrorInvalidValue;
    PlaneKernel fn = plane_kernel(cls);
    cudaError_t e = set_max_smem((const void*)fn, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[2];
    launch_config(cfg, attr, dim3((unsigned)(b.nclusters * b.cs)), dim3(kPlaneThreads), smem, st, b.cs);
    return cudaLaunchKernelEx(&cfg, fn, b);
}

}  // namespace zncc
