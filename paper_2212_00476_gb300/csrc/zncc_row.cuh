// zncc_row.cuh -- ZNCC cost of one image row for a range of disparities, optionally fused
// with the first horizontal DT pass pair (Sec. V-C fuses the cost with L2R the same way) or
// with WTA (no aggregation). Instantiated once per window radius R in zncc_row.cu.
#pragma once

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace zncc {

// Block (row y, a run of spb disparity slices of 4*tq disparities): thread (chunk k, dq)
// computes the costs of pixels x in [16k, 16k+16) for the four disparities d0 + 4dq ..
// d0 + 4dq + 3 of each slice. The chunk count is padded to whole warps; pixels x >= W are
// computed from clamped reads and dropped.
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
// window sums P(x) = prefix(x+R) - prefix(x-R-1). The packed bands are staged once per
// block and serve all of its disparity slices; the window statistics of both images
// (Sec. IV-B-1, Eq. (sum1)) come from the same packed columns: a column's pixel sum is
// __dp4a(word, 0x01010101) and its sum of squares __dp4a(word, word), slid like P.
// Four packed columns xs .. xs+3 (all inside the row) of a band of l raw rows in shared memory
// (row j at raw + j * Wr, Wr a multiple of 16), xs = S (mod 4): per row one 32-bit word of the
// four pixels (two aligned words funnel-shifted when S > 0), then a 4 x 4 byte transpose per
// packed word.
template <int l, int S>
__device__ __forceinline__ void pack4_raw(const uint8_t* raw, int Wr, int xs, uint4 (&col)[4]) {
    constexpr int NW = (l + 3) / 4;
    const unsigned* r32 = reinterpret_cast<const unsigned*>(raw);
    const int a4 = (xs - S) >> 2, wr4 = Wr >> 2;
    unsigned w[4 * NW];
#pragma unroll
    for (int j = 0; j < 4 * NW; ++j) {
        if (j < l) {
            const unsigned lo = r32[j * wr4 + a4];
            w[j] = S ? __funnelshift_r(lo, r32[j * wr4 + a4 + 1], 8 * S) : lo;
        } else {
            w[j] = 0u;
        }
    }
    unsigned o[4][4] = {{0u, 0u, 0u, 0u}, {0u, 0u, 0u, 0u}, {0u, 0u, 0u, 0u}, {0u, 0u, 0u, 0u}};
#pragma unroll
    for (int k = 0; k < NW; ++k) {
        const unsigned t0 = __byte_perm(w[4 * k], w[4 * k + 1], 0x5140), t1 = __byte_perm(w[4 * k + 2], w[4 * k + 3], 0x5140);
        const unsigned t2 = __byte_perm(w[4 * k], w[4 * k + 1], 0x7362), t3 = __byte_perm(w[4 * k + 2], w[4 * k + 3], 0x7362);
        o[0][k] = __byte_perm(t0, t1, 0x5410);
        o[1][k] = __byte_perm(t0, t1, 0x7632);
        o[2][k] = __byte_perm(t2, t3, 0x5410);
        o[3][k] = __byte_perm(t2, t3, 0x7632);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) col[c] = make_uint4(o[c][0], o[c][1], o[c][2], o[c][3]);
}

// Centres per item of the window statistics. An item's column walk reads up to kStatsItem - 1
// columns past the last centre of the band, so the packed band planes hold kStatsItem spare
// entries.
constexpr int kStatsItem = 12;

// Bytes of the rows a visit stages by bulk copies: l rows of each image, Wr = W + 16 apart.
__host__ __device__ inline int bulk_row_stride(int W) { return W + 16; }

// One visit of the cost kernel: row y of one pair, disparity slices [s_begin, s_end).
// Threads beyond the pair's nch * tq (whole warps) only take part in the barriers. Returns
// false when a bulk copy of the image rows timed out (the fault is recorded; the block stops).
template <int R, typename T, int MODE>
__device__ __forceinline__ bool zncc_row_item(const RowArgs& a, int y, int s_begin, int s_end,
                                              uint4* smem_u4, unsigned long long* bar, unsigned& phase,
                                              unsigned* fault) {
    constexpr int l = 2 * R + 1;
    constexpr int NW = (l + 3) / 4;     // packed words per column
    const int tq = a.tq, ds = kG * tq, nch = a.nch, span = nch * kL;
    const int W = a.W, H = a.H;
    const int tid = threadIdx.x;
    const int nthr = nch * tq;
    const bool active = tid < nthr;
    const int k = active ? tid / tq : 0, dq = active ? tid - (tid / tq) * tq : 0;
    const int lane = tid & 31, wl = tid >> 5, nwl = nthr >> 5;
    // every lane's disparities lie in [blk_lo, blk_hi)
    const int blk_lo = a.d_lo + s_begin * ds, blk_hi = a.d_lo + s_end * ds;

    // ---- shared memory carve ----
    const int NLP = span + 2 * R;                      // left columns x' in [-R, span+R)
    const int NRP = span + 2 * R + (blk_hi - blk_lo) - 1;
    const int xr0 = -R - (blk_hi - 1);                 // right columns x'' in [xr0, xr0+NRP)
    const int NSR = span + (blk_hi - blk_lo) - 1;      // right centres c in [c0, c0+NSR)
    const int c0 = -(blk_hi - 1);
    const int pLP = plane_of(NLP + kStatsItem), pRP = plane_of(NRP + kStatsItem), pX = plane_of(span), pSR = plane_of(NSR);
    uint4* LP = smem_u4;
    uint4* RP = LP + 4 * pLP;
    int2* SL = reinterpret_cast<int2*>(RP + 4 * pRP);               // (S, 1/sigma bits) per x
    int2* SR = SL + 4 * pX;                                          // per right centre
    float4* co = reinterpret_cast<float4*>(SR + 4 * pSR);            // HPair, chunk-major
    float4* sb = co + nch * kCS;
    float* sa = reinterpret_cast<float*>(sb + 2 * nwl * tq);
    // FastDT codes (HPair): the row's output scales and the reference values v(d_arb = 0)
    constexpr bool kFast = std::is_same<T, uint8_t>::value;
    float* mrow = sa + 2 * nwl * tq;                                 // chunk-major (kCS)
    float* ref = mrow + nch * kCS;
    // (bulk) the guide row y for the coefficients, after everything else
    uint8_t* grow = reinterpret_cast<uint8_t*>(kFast ? ref + nch * kCS : mrow);

    // ---- stage the packed bands (and the DT coefficients) ----
    const bool bulk = MODE == kModeHPair && a.bulk;
    if (bulk) {
        // Bulk copies (the TMA unit) of the clamped rows y-R .. y+R of both images into the
        // region that the statistics and coefficients take once the bands are packed, and of
        // the guide row y; one thread issues them, every thread waits on the mbarrier.
        const int Wr = bulk_row_stride(W);
        uint8_t* rawL = reinterpret_cast<uint8_t*>(SL);
        uint8_t* rawR = rawL + l * Wr;
        fence_proxy_async_smem();                       // earlier accesses of the region, then the copies
        __syncthreads();
        if (tid == 0) {
            mbar_expect_tx(bar, (unsigned)((2 * l + 1) * W));
#pragma unroll
            for (int j = 0; j < l; ++j) {
                const size_t ro = (size_t)min(max(y - R + j, 0), H - 1) * a.pitch;
                bulk_copy_g2s(rawL + j * Wr, a.left + ro, (unsigned)W, bar);
                bulk_copy_g2s(rawR + j * Wr, a.right + ro, (unsigned)W, bar);
            }
            bulk_copy_g2s(grow, a.left + (size_t)y * a.pitch, (unsigned)W, bar);
        }
        bool ok = mbar_wait(bar, phase, kBulkWaitPolls);
        if (__syncthreads_or(!ok)) {                     // a copy did not land in time: record it,
            if (tid == 0) atomicOr(fault, kFaultBulkWait);
            ok = mbar_wait(bar, phase, kBulkWaitPolls);  // wait for the copies still in flight
            if (__syncthreads_or(!ok) && tid == 0) atomicOr(fault, kFaultBulkDrain);
            return false;
        }
        phase ^= 1u;
        // pack four columns per thread where they lie inside the row, single columns (clamped)
        // at the ends
        auto pack1 = [&](const uint8_t* raw, int xc) {
            unsigned w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int j = 0; j < l; ++j) w[j >> 2] |= (unsigned)raw[j * Wr + xc] << (8 * (j & 3));
            return make_uint4(w[0], w[1], w[2], w[3]);
        };
        constexpr int SLS = ((-R) % 4 + 4) % 4, SRS = ((1 - R) % 4 + 4) % 4;   // (-R) & 3, xr0 & 3
        const int ngl = (NLP + 3) >> 2, ngr = (NRP + 3) >> 2;
        for (int g = tid; g < ngl + ngr; g += blockDim.x) {
            const bool left = g < ngl;
            const int g4 = left ? g : g - ngl;
            const int xs = left ? 4 * g4 - R : xr0 + 4 * g4;   // image column of entry 4 g4
            const int nent = left ? NLP : NRP;
            uint4* dst = left ? LP : RP;
            const int pl = left ? pLP : pRP;
            const uint8_t* raw = left ? rawL : rawR;
            if (xs >= 0 && xs + 3 < W && 4 * g4 + 3 < nent) {
                uint4 col[4];
                if (left) pack4_raw<l, SLS>(raw, Wr, xs, col);
                else pack4_raw<l, SRS>(raw, Wr, xs, col);
#pragma unroll
                for (int c = 0; c < 4; ++c) dst[c * pl + g4] = col[c];
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (4 * g4 + c < nent) dst[c * pl + g4] = pack1(raw, min(max(xs + c, 0), W - 1));
            }
        }
        __syncthreads();                                 // the raw rows are consumed
    } else {
        size_t roff[l];                                 // the band's clamped rows
#pragma unroll
        for (int j = 0; j < l; ++j) roff[j] = (size_t)min(max(y - R + j, 0), H - 1) * a.pitch;
        auto pack = [&](const uint8_t* img, int xc) {
            unsigned w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int j = 0; j < l; ++j) w[j >> 2] |= (unsigned)img[roff[j] + xc] << (8 * (j & 3));
            return make_uint4(w[0], w[1], w[2], w[3]);
        };
        for (int t = tid; t < NLP; t += blockDim.x) LP[p4(t, pLP)] = pack(a.left, min(max(t - R, 0), W - 1));
        for (int t = tid; t < NRP; t += blockDim.x) RP[p4(t, pRP)] = pack(a.right, min(max(xr0 + t, 0), W - 1));
    }
    if constexpr (MODE == kModeHPair) {
        // the row's DT coefficients (w, chunk prefix product, next w, chunk suffix product),
        // computed here from the guide (the left image) as k_dt_coef computes them: 16
        // consecutive lanes hold one chunk (span and the block are whole warps)
        const uint8_t* g = bulk ? grow : a.left + (size_t)y * a.pitch;
        auto weight = [&](int q) -> float {      // the step q-1 -> q
            return (q >= 1 && q < W) ? a.K * expf(-fabsf((float)(g[q] - g[q - 1])) * a.inv_sr255) : 0.0f;
        };
        for (int t = tid; t < span; t += blockDim.x) {
            const int i = t & (kL - 1);
            const float w = weight(t);
            float wn = __shfl_down_sync(kFull, w, 1, kL);
            if (i == kL - 1) wn = weight(t + 1);
            float A = w, B = wn;
#pragma unroll
            for (int off = 1; off < kL; off <<= 1) {
                const float a2 = __shfl_up_sync(kFull, A, off, kL);
                const float b2 = __shfl_down_sync(kFull, B, off, kL);
                if (i >= off) A *= a2;
                if (i + off < kL) B *= b2;
            }
            co[cpos(t)] = t < W ? make_float4(w, A, wn, B) : make_float4(0.f, 0.f, 0.f, 0.f);
            if (a.coefH_out && s_begin == 0 && t < W) a.coefH_out[(size_t)y * W + t] = make_float4(w, A, wn, B);
            if constexpr (kFast)
                mrow[cpos(t)] = t < W ? __ldg(a.mulmap + (size_t)y * W + t).y : 0.0f;
        }
    }
    __syncthreads();

    // ---- window statistics: kSC consecutive centres per thread, left then right ----
    // Items of 12 centres start 12 columns apart, so the 16-byte column loads of the eight
    // lanes of a quarter warp fall in distinct bank groups (16 apart, they would share two).
    constexpr int kSC = kStatsItem;
    const unsigned n = (unsigned)(l * l);
    // A fused horizontal pair (F32, F16) in the scaled form multiplies its result by
    // s2 = (1-K)^2; the pair is linear, so the factor rides on the left 1/sigma instead
    // (FastDT codes take per-position scales in the pair).
    const float lscale = (MODE == kModeHPair && !kFast) ? a.s2 : 1.0f;
    const int nlc = (span + kSC - 1) / kSC, nrc = (NSR + kSC - 1) / kSC;
    for (int t = tid; t < nlc + nrc; t += blockDim.x) {
        const bool is_left = t < nlc;
        const int cs = is_left ? t * kSC : c0 + (t - nlc) * kSC;   // first centre
        const uint4* col = is_left ? LP : RP;
        const int pc = is_left ? pLP : pRP;
        const int ib = is_left ? cs : cs - R - xr0;                 // column index of cs - R
        // (ib = 12 t, or 12 (t - nlc) on the right: both multiples of 4)
        int Sx[kSC], Qx[kSC];
#pragma unroll
        for (int i = 0; i < kSC; ++i) Sx[i] = Qx[i] = 0;
        unsigned ps = 0u, pq = 0u;
#pragma unroll
        for (int u = 0; u < kSC + 2 * R; ++u) {
            const uint4 w = at4(col, ib, u, pc);
            ps = __dp4a(w.x, 0x01010101u, ps);
            pq = __dp4a(w.x, w.x, pq);
            if (NW > 1) { ps = __dp4a(w.y, 0x01010101u, ps); pq = __dp4a(w.y, w.y, pq); }
            if (NW > 2) { ps = __dp4a(w.z, 0x01010101u, ps); pq = __dp4a(w.z, w.z, pq); }
            if (NW > 3) { ps = __dp4a(w.w, 0x01010101u, ps); pq = __dp4a(w.w, w.w, pq); }
            if (u - 2 * R >= 0 && u - 2 * R < kSC) { Sx[u - 2 * R] += (int)ps; Qx[u - 2 * R] += (int)pq; }
            if (u + 1 < kSC) { Sx[u + 1] -= (int)ps; Qx[u + 1] -= (int)pq; }
        }
#pragma unroll
        for (int i = 0; i < kSC; ++i) {
            const int var = (int)(n * (unsigned)Qx[i] - (unsigned)Sx[i] * (unsigned)Sx[i]);
            const float is = var > 0 ? rsqrtf((float)var) : 0.0f;      // as k_window_stats
            const int2 st = make_int2(Sx[i], __float_as_int(is_left ? is * lscale : is));
            if (is_left) {
                if (cs + i < span) at4(SL, cs, i, pX) = st;
            } else if (cs + i - c0 < NSR) {
                at4(SR, cs - c0, i, pSR) = st;
            }
        }
    }
    __syncthreads();

    const int x0 = k * kL;
    T* out = reinterpret_cast<T*>(a.vol);
    const bool vec = a.vec != 0;
    WtaRegs wr;
    if constexpr (MODE == kModeWta) wr.reset();

    for (int sl = s_begin; sl < s_end; ++sl) {
        const int d_first = a.d_lo + sl * ds + dq * kG;
        const int nvalid = max(0, min(4, a.d_hi - d_first));
        float v[kL][4];
        if (active) {
            // ---- window sums of products, times n, for 16 pixels x 4 disparities ----
            // n P[i] = n prefix(i + 2R) - n prefix(i - 1): each entry is set at its first touch
            // (-n prefix(i - 1) at step i - 1; n P[0] at step 2R) and completed at step i + 2R;
            // the factor n of Eq. (2)'s numerator rides on those multiply-adds (mod 2^32)
            unsigned P[kL][4];
            // RP index of column x' - d_first - j at step t (x' = x0 - R + t) is rbase + t - j;
            // rbase + 1 = x0 - d_first + blk_hi is a multiple of 4 (as are x0, d_first and
            // blk_hi, d_lo being one), so every index below has a constant plane
            const int rbase = x0 - R - d_first - xr0;      // >= 3: d_first + 3 < blk_hi
            const int rb4 = rbase + 1;
            uint4 rp[4];
            rp[1] = at4(RP, rb4, -2, pRP);
            rp[2] = at4(RP, rb4, -3, pRP);
            rp[3] = at4(RP, rb4, -4, pRP);
            unsigned pre[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int t = 0; t < kL + 2 * R; ++t) {
                const uint4 lp = at4(LP, x0, t, pLP);
                rp[0] = at4(RP, rb4, t - 1, pRP);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    pre[j] = __dp4a(lp.x, rp[j].x, pre[j]);
                    if (NW > 1) pre[j] = __dp4a(lp.y, rp[j].y, pre[j]);
                    if (NW > 2) pre[j] = __dp4a(lp.z, rp[j].z, pre[j]);
                    if (NW > 3) pre[j] = __dp4a(lp.w, rp[j].w, pre[j]);
                    if (t == 2 * R) P[0][j] = n * pre[j];
                    else if (t - 2 * R > 0 && t - 2 * R < kL) P[t - 2 * R][j] += n * pre[j];
                    if (t + 1 < kL) P[t + 1][j] = (0u - n) * pre[j];
                }
                rp[3] = rp[2];
                rp[2] = rp[1];
                rp[1] = rp[0];
            }

            // ---- normalization, Eq. (2); the target statistics slide like the columns ----
            const int cb = x0 - d_first - c0;               // SR index of (i, j) is cb + i - j >= 3
            const int cb4 = cb + 1;                         // a multiple of 4, like rb4
            int2 sr[4];
            sr[1] = at4(SR, cb4, -2, pSR);
            sr[2] = at4(SR, cb4, -3, pSR);
            sr[3] = at4(SR, cb4, -4, pSR);
            auto normalize = [&](auto full) {
#pragma unroll
                for (int i = 0; i < kL; ++i) {
                    const int x = x0 + i;
                    const int2 st = at4(SL, x0, i, pX);
                    sr[0] = at4(SR, cb4, i - 1, pSR);
                    const float isl = __int_as_float(st.y);      // (times the pair's scale)
                    const unsigned nsl = 0u - (unsigned)st.x;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const unsigned num = nsl * (unsigned)sr[j].x + P[i][j];       // n P - S_R S_T
                        const float c = (float)(int)num * isl * __int_as_float(sr[j].y);
                        if constexpr (decltype(full)::value) v[i][j] = c;
                        else v[i][j] = (x < W && j < nvalid) ? c : 0.0f;
                    }
                    sr[3] = sr[2];
                    sr[2] = sr[1];
                    sr[1] = sr[0];
                }
            };
            // whole chunks of whole 4-disparity groups take the path without predicates
            if (x0 + kL <= W && nvalid == 4) normalize(std::true_type());
            else normalize(std::false_type());
        }

        if constexpr (MODE == kModeWta) {
            if (active) wr.fold(v, nvalid, d_first);
            continue;
        }
        if constexpr (MODE == kModeHPair && kFast)
            dt_pair(v, co + k * kCS, tq, dq, lane, wl, nwl, sa, sb, a.s2, mrow + k * kCS, NoHook(), active);
        else if constexpr (MODE == kModeHPair)       // s2 already folded into the costs
            dt_pair<false>(v, co + k * kCS, tq, dq, lane, wl, nwl, sa, sb, 1.0f, (const float2*)nullptr,
                           NoHook(), active);

        if constexpr (kFast) {
            // near-zero-mean codes against d_arb = 0, held by lane dq 0 in slice 0 (a visit covers
            // every slice of its row, in order)
            if (sl == 0) {
                if (dq == 0 && active)
#pragma unroll
                    for (int i = 0; i < kL; ++i) ref[k * kCS + i] = v[i][0];
                __syncthreads();
            }
            if (active && nvalid > 0) {
                T* q = out + ((size_t)y * W + x0) * a.dstride + (d_first - a.d_out0);
#pragma unroll
                for (int i = 0; i < kL; ++i) {
                    if (x0 + i < W) *reinterpret_cast<unsigned*>(q) = fastdt_pack(v[i], ref[k * kCS + i], nvalid);
                    q += a.dstride;
                }
            }
        } else if (active && nvalid > 0) {
            // ---- store [H][W][dstride] ----
            T* q = out + ((size_t)y * W + x0) * a.dstride + (d_first - a.d_out0);
            if (vec && nvalid == 4 && x0 + kL <= W) {        // a whole chunk of whole groups
#pragma unroll
                for (int i = 0; i < kL; ++i) st4(q + (size_t)i * a.dstride, 4, true, v[i]);
            } else {
#pragma unroll
                for (int i = 0; i < kL; ++i) {
                    if (x0 + i < W) st4(q, nvalid, vec, v[i]);
                    q += a.dstride;
                }
            }
        }
    }

    if constexpr (MODE == kModeWta) {
        if (active) {
            // the chunk's lanes merge their running bests; each lane writes its share of positions
            wr.merge(tq, lane, [&](int i, float best, int bd) {
                const int x = x0 + i;
                if (x < W) {
                    const size_t o = (size_t)y * W + x;
                    if (!a.wta.first) {                                // earlier launches: smaller d
                        const float pb = a.wta.bestv[o];
                        if (!(best > pb)) { best = pb; bd = a.wta.bestd[o]; }
                    }
                    if (a.wta.last) a.wta.disp[o] = (uint16_t)bd;
                    else {
                        a.wta.bestv[o] = best;
                        a.wta.bestd[o] = bd;
                    }
                }
            });
        }
    }
    return true;
}

// SINGLE: the launch holds one pair, whose arguments are then read at constant offsets of
// the parameter block instead of through a dynamic index.
// Work units: (row, disparity slice) in row-major order, pair by pair (Wta: whole rows, since
// a row's running best stays in registers; FastDT codes: whole rows, since every slice is
// coded against d = 0 of the first). Block b takes the units [b*total/G, (b+1)*total/G)
// and visits them row by row, at most spb slices per visit, so that the band of a row is
// staged once per visit and every block gets the same work within one unit.
template <int R, typename T, int MODE, int MINB, bool SINGLE>
__global__ void __launch_bounds__(MINB == 2 ? 320 : 512, MINB) k_zncc_row(const __grid_constant__ RowBatch b) {
    extern __shared__ uint4 smem_u4[];
    __shared__ unsigned long long bar;                  // bulk copies of the image rows (HPair)
    unsigned phase = 0;
    if (MODE == kModeHPair && threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    griddep_wait();
    const int i0 = (int)((long long)blockIdx.x * b.total_items / b.grid);
    const int i1 = (int)((long long)(blockIdx.x + 1) * b.total_items / b.grid);
    int pi = 0;
    for (int u = i0; u < i1;) {
        if (!SINGLE)
            while (u >= b.p[pi].item0 + b.p[pi].nitems) ++pi;
        const RowArgs& a = b.p[SINGLE ? 0 : pi];
        const int ds = kG * a.tq;
        const int nslices = (a.d_hi - a.d_lo + ds - 1) / ds;
        const int local = u - a.item0;
        int y, s_begin, s_end;
        if constexpr (MODE == kModeWta || std::is_same<T, uint8_t>::value) {     // whole rows
            y = local;
            s_begin = 0;
            s_end = nslices;
            u += 1;
        } else {
            y = local / nslices;
            s_begin = local - y * nslices;
            const int last = min(i1, a.item0 + (y + 1) * nslices);      // this block, this row
            s_end = min(s_begin + a.spb, s_begin + (last - u));
            u += s_end - s_begin;
        }
        if (u >= i1) griddep_launch_dependents();       // this block's last visit
        if (!zncc_row_item<R, T, MODE>(a, y, s_begin, s_end, smem_u4, &bar, phase, b.fault)) return;
        __syncthreads();                                 // the next visit restages shared memory
    }
}

// Shared-memory bytes of one item of k_zncc_row.
inline size_t zncc_row_smem(int R, int mode, int dtype, const RowArgs& a, int nthreads) {
    const int ds = kG * a.tq, span = a.nch * kL;
    const int nslices = (a.d_hi - a.d_lo + ds - 1) / ds;
    const int drange = std::min(a.spb, nslices) * ds;
    size_t b = 16ull * 4 * (plane_of(span + 2 * R + kStatsItem) + plane_of(span + 2 * R + drange - 1 + kStatsItem));
    const int pX = plane_of(span);
    b += 8ull * 4 * (pX + plane_of(span + drange - 1));
    if (mode == kModeHPair) b += 16ull * a.nch * kCS + dt_scan_bytes(nthreads / 32, a.tq);
    if (mode == kModeHPair && dtype == 2) b += 8ull * a.nch * kCS;       // FastDT: scales, references
    if (mode == kModeHPair && a.bulk) b += (size_t)(a.W + 15) / 16 * 16; // the guide row
    return b;
}

// Whether a visit's raw rows (both images, bulk_row_stride apart) fit in the shared memory that
// the statistics and the later per-visit arrays take (HPair): the region after the packed bands.
inline bool zncc_row_bulk_fits(int R, int dtype, const RowArgs& a, int nthreads) {
    const int ds = kG * a.tq, span = a.nch * kL;
    const int nslices = (a.d_hi - a.d_lo + ds - 1) / ds;
    const int drange = std::min(a.spb, nslices) * ds;
    size_t after = 8ull * 4 * (plane_of(span) + plane_of(span + drange - 1)) + 16ull * a.nch * kCS +
                   dt_scan_bytes(nthreads / 32, a.tq);
    if (dtype == 2) after += 8ull * a.nch * kCS;
    return 2ull * (2 * R + 1) * bulk_row_stride(a.W) <= after;
}

template <int R, int MINB, bool SINGLE>
static void (*row_fn_t(int mode, int dtype))(RowBatch) {
    if (mode == kModeRaw)
        return dtype == 0 ? k_zncc_row<R, float, kModeRaw, MINB, SINGLE> : k_zncc_row<R, __half, kModeRaw, MINB, SINGLE>;
    if (mode == kModeHPair)
        return dtype == 0 ? k_zncc_row<R, float, kModeHPair, MINB, SINGLE>
                          : dtype == 1 ? k_zncc_row<R, __half, kModeHPair, MINB, SINGLE>
                                       : k_zncc_row<R, uint8_t, kModeHPair, MINB, SINGLE>;
    return k_zncc_row<R, float, kModeWta, MINB, SINGLE>;
}

// Batched launches come from the fused path only (HPair, Wta); a batched Raw launch would
// use the single-pair variant's arguments and is never made.
template <int R>
static void (*row_fn(int mode, int dtype, bool minb2, bool single))(RowBatch) {
    if (single) return minb2 ? row_fn_t<R, 2, true>(mode, dtype) : row_fn_t<R, 1, true>(mode, dtype);
    if (mode == kModeRaw) return nullptr;
    return minb2 ? row_fn_t<R, 2, false>(mode, dtype) : row_fn_t<R, 1, false>(mode, dtype);
}

// The variant limited to 96 registers (two resident blocks per SM) serves blocks of up to
// 320 threads when minb2 is set; larger blocks use the 128-register one.
template <int R>
cudaError_t zncc_row_occupancy_impl(int mode, int dtype, int threads, size_t smem, bool minb2, bool single,
                                    int* bps) {
    void (*fn)(RowBatch) = row_fn<R>(mode, dtype, minb2 && threads <= 320, single);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = set_max_smem((const void*)fn, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, fn, threads, smem);
}

template <int R>
cudaError_t launch_zncc_row_impl(const RowBatch& b, int threads, size_t smem, int mode, int dtype,
                                 cudaStream_t st) {
    bool minb2 = true;
    for (int i = 0; i < b.npairs; ++i) minb2 = minb2 && b.p[i].minb2;
    void (*fn)(RowBatch) = row_fn<R>(mode, dtype, minb2 && threads <= 320, b.npairs == 1);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = set_max_smem((const void*)fn, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[2];
    launch_config(cfg, attr, dim3(b.grid), dim3(threads), smem, st, 1);
    return cudaLaunchKernelEx(&cfg, fn, b);
}

}  // namespace zncc
