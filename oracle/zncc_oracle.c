/*
 * zncc_oracle.c -- plain, slow, FP64 CPU oracle for ZNCC + DT + WTA stereo matching.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg may load this library. It shares no code with the CUDA
 * path and must never serve a product call.
 *
 * Method: arXiv 2212.00476, "Efficient stereo matching on embedded GPUs with zero-means
 * cross correlation".
 *   - window sums:      Sec. IV-B-1, Eq. (sum1) (Method 1) and the integral image (Method 2)
 *   - matching cost:    Sec. III-A, Eq. (1) (ZNCC, computed literally from its definition)
 *   - DT weights:       Sec. III-B, Eqs. (7)-(10) and the simplified Eq. (11)
 *   - DT aggregation:   Sec. III-B, Eqs. (3)-(6), boundary condition C_L(0,y,d) = C(0,y,d)
 *   - disparity (WTA):  Sec. III-C, Eq. (WTA1)
 *   - FastDT storage:   Sec. IV-C (near-zero-mean normalization, 16-bit values, 8-bit code)
 *
 * Readings of passages the paper leaves open or garbles:
 *   - reference image I_R = left, target I_T = right; I_R(x,y) is matched to I_T(x-d,y);
 *   - every pixel read is clamped to the image (clamp-to-edge), also for centres x-d < 0;
 *   - a window with zero variance gives cost 0;
 *   - the DT guide is the reference (left) image scaled to [0,1] (sigma_r in those units);
 *   - every pass starts from its own input at the first element of its scan direction;
 *   - "scaled" form: each pass multiplies its input term by (1-K), K = exp(-1/sigma_s).
 *     It equals the literal chain times (1-K)^(4*iters) and keeps |C| <= 1;
 *   - iterations repeat the 4-pass chain (L2R, R2L, U2D, D2U) with the same sigmas;
 *   - WTA returns the smallest d reaching the maximum aggregated value (argmin of 1-C);
 *   - FastDT: d_arb = 0 (the paper's choice); the store happens after every pass pair but
 *     the last (the last feeds WTA), on e = (C(d_arb) - C(d)) / A_hat with A_hat the same
 *     pass pairs applied to an all-ones plane (|C| <= A_hat, so e lies in [-2, 2]), scaled
 *     by T = 16383 (the largest T with 2T inside int16; the paper's T = 21 belongs to its
 *     unnormalised costs), rounded to nearest (ties to even) and clamped to int16; the
 *     decoded value -E/T * A_hat replaces C (the offset C(d_arb) is not added back: a
 *     per-pixel offset changes no argmax, and the paper's Eq. (DT_new) drops it too).
 *
 * Layouts: images uint8 [H][W] (row pitch = W); cost volumes double [H][W][nd], the
 * disparity axis fastest.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ENOMEM 2

/* ------------------------------------------------------------------------------------ */
/* a tiny parallel-for over [0, n) on plain pthreads                                      */

typedef void (*range_fn)(void* ctx, long begin, long end);

typedef struct {
    range_fn fn;
    void* ctx;
    long begin, end;
} range_job;

static void* range_thread(void* p) {
    range_job* j = (range_job*)p;
    j->fn(j->ctx, j->begin, j->end);
    return NULL;
}

static void parallel_for(long n, int nthreads, range_fn fn, void* ctx) {
    if (nthreads <= 1 || n < 2) {
        fn(ctx, 0, n);
        return;
    }
    if (nthreads > n) nthreads = (int)n;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    range_job jobs[256];
    long chunk = (n + nthreads - 1) / nthreads;
    int started = 0;
    for (int t = 0; t < nthreads; ++t) {
        long b = (long)t * chunk, e = b + chunk < n ? b + chunk : n;
        if (b >= e) break;
        jobs[t].fn = fn; jobs[t].ctx = ctx; jobs[t].begin = b; jobs[t].end = e;
        if (pthread_create(&th[t], NULL, range_thread, &jobs[t]) != 0) {
            fn(ctx, b, e);            /* could not start a thread: do the range here */
            jobs[t].fn = NULL;
        }
        started = t + 1;
    }
    for (int t = 0; t < started; ++t)
        if (jobs[t].fn) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------------------------------ */
/* pixel access with clamp-to-edge                                                        */

static inline int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

static inline int pix(const uint8_t* img, int W, int H, int x, int y) {
    return img[(long)clampi(y, 0, H - 1) * W + clampi(x, 0, W - 1)];
}

/* ------------------------------------------------------------------------------------ */
/* Window sums, Method 1 (Sec. IV-B-1, Eq. (sum1)): S = sum of the (2r+1)^2 pixels around  */
/* the centre, Q = sum of their squares. Centres x in [x_begin, x_end), every y.           */
/* Output layout [H][x_end - x_begin].                                                     */

int oracle_window_sums(const uint8_t* img, int W, int H, int r, int x_begin, int x_end,
                       int64_t* S, int64_t* Q) {
    if (!img || W < 1 || H < 1 || r < 0 || x_end < x_begin) return ORACLE_EINVAL;
    int nx = x_end - x_begin;
    for (int y = 0; y < H; ++y)
        for (int xi = 0; xi < nx; ++xi) {
            int x = x_begin + xi;
            int64_t s = 0, q = 0;
            for (int j = -r; j <= r; ++j)
                for (int i = -r; i <= r; ++i) {
                    int v = pix(img, W, H, x + i, y + j);
                    s += v;
                    q += (int64_t)v * v;
                }
            if (S) S[(long)y * nx + xi] = s;
            if (Q) Q[(long)y * nx + xi] = q;
        }
    return ORACLE_OK;
}

/* Window sums, Method 2 (Sec. IV-B-1): integral image B of the clamp-padded image, then   */
/* the four-corner lookup. B(u,v) = sum_{u'<=u, v'<=v} P(u',v'), with B(-1,.) = B(.,-1) = 0. */
/* The padded image P covers columns [x_begin - r, x_end + r) and rows [-r, H + r).        */

int oracle_window_sums_integral(const uint8_t* img, int W, int H, int r, int x_begin,
                                int x_end, int64_t* S, int64_t* Q) {
    if (!img || W < 1 || H < 1 || r < 0 || x_end < x_begin) return ORACLE_EINVAL;
    int nx = x_end - x_begin;
    int PW = nx + 2 * r, PH = H + 2 * r;
    /* B has one extra leading row and column of zeros: Bz[v+1][u+1] = B(u,v) */
    int64_t* B1 = (int64_t*)calloc((size_t)(PW + 1) * (PH + 1), sizeof(int64_t));
    int64_t* B2 = (int64_t*)calloc((size_t)(PW + 1) * (PH + 1), sizeof(int64_t));
    if (!B1 || !B2) { free(B1); free(B2); return ORACLE_ENOMEM; }
    /* step 1: integrate each row (B_H); step 2: integrate each column of B_H */
    for (int v = 0; v < PH; ++v) {
        int64_t run1 = 0, run2 = 0;
        for (int u = 0; u < PW; ++u) {
            int p = pix(img, W, H, x_begin - r + u, v - r);
            run1 += p;
            run2 += (int64_t)p * p;
            B1[(long)(v + 1) * (PW + 1) + (u + 1)] = run1;
            B2[(long)(v + 1) * (PW + 1) + (u + 1)] = run2;
        }
    }
    for (int u = 1; u <= PW; ++u)
        for (int v = 1; v <= PH; ++v) {
            B1[(long)v * (PW + 1) + u] += B1[(long)(v - 1) * (PW + 1) + u];
            B2[(long)v * (PW + 1) + u] += B2[(long)(v - 1) * (PW + 1) + u];
        }
    /* window of centre (xi, y) covers padded u in [xi, xi+2r], v in [y, y+2r] */
    for (int y = 0; y < H; ++y)
        for (int xi = 0; xi < nx; ++xi) {
            long a = (long)(y + 2 * r + 1) * (PW + 1) + (xi + 2 * r + 1); /* B(xi+2r, y+2r) */
            long b = (long)(y) * (PW + 1) + (xi);                         /* B(xi-1, y-1)   */
            long c = (long)(y) * (PW + 1) + (xi + 2 * r + 1);             /* B(xi+2r, y-1)  */
            long e = (long)(y + 2 * r + 1) * (PW + 1) + (xi);             /* B(xi-1, y+2r)  */
            if (S) S[(long)y * nx + xi] = B1[a] + B1[b] - B1[c] - B1[e];
            if (Q) Q[(long)y * nx + xi] = B2[a] + B2[b] - B2[c] - B2[e];
        }
    free(B1);
    free(B2);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Window mean and sigma of Eq. (1): mean = average of the window; sigma = sqrt(sum of     */
/* squared deviations) (a sum, not divided by the window size).                           */

static void window_mean_sigma(const uint8_t* img, int W, int H, int r, int cx, int cy,
                              double* mean, double* sigma) {
    int n = (2 * r + 1) * (2 * r + 1);
    double s = 0.0;
    for (int j = -r; j <= r; ++j)
        for (int i = -r; i <= r; ++i) s += pix(img, W, H, cx + i, cy + j);
    double m = s / n;
    double ss = 0.0;
    for (int j = -r; j <= r; ++j)
        for (int i = -r; i <= r; ++i) {
            double dv = pix(img, W, H, cx + i, cy + j) - m;
            ss += dv * dv;
        }
    *mean = m;
    *sigma = sqrt(ss);
}

/* ZNCC of Eq. (1) for one (x, y, d): the window around I_R(x,y) against the window around */
/* I_T(x-d,y). Zero variance on either side gives the fixed cost 0.                       */

static double zncc_one(const uint8_t* L, const uint8_t* R, int W, int H, int r,
                       double mL, double sL, double mR, double sR, int x, int y, int d) {
    if (sL == 0.0 || sR == 0.0) return 0.0;
    double num = 0.0;
    for (int j = -r; j <= r; ++j)
        for (int i = -r; i <= r; ++i)
            num += (pix(L, W, H, x + i, y + j) - mL) * (pix(R, W, H, x - d + i, y + j) - mR);
    return num / (sL * sR);
}

double oracle_zncc_at(const uint8_t* L, const uint8_t* R, int W, int H, int r, int x, int y,
                      int d) {
    double mL, sL, mR, sR;
    window_mean_sigma(L, W, H, r, x, y, &mL, &sL);
    window_mean_sigma(R, W, H, r, x - d, y, &mR, &sR);
    return zncc_one(L, R, W, H, r, mL, sL, mR, sR, x, y, d);
}

typedef struct {
    const uint8_t *L, *R;
    int W, H, D, r, nd;
    const int* planes;
    double* C;
} zncc_job;

static void zncc_rows(void* p, long y0, long y1) {
    zncc_job* j = (zncc_job*)p;
    int W = j->W, H = j->H, D = j->D, r = j->r, nd = j->nd;
    int ext = W + D - 1;                        /* target centres x-d in [-(D-1), W) */
    double* mR = (double*)malloc(sizeof(double) * 2 * ext);
    double* mL = (double*)malloc(sizeof(double) * 2 * W);
    if (!mR || !mL) { free(mR); free(mL); return; }
    double* sR = mR + ext;
    double* sL = mL + W;
    for (long y = y0; y < y1; ++y) {
        for (int x = 0; x < W; ++x) window_mean_sigma(j->L, W, H, r, x, (int)y, &mL[x], &sL[x]);
        for (int t = 0; t < ext; ++t)
            window_mean_sigma(j->R, W, H, r, t - (D - 1), (int)y, &mR[t], &sR[t]);
        for (int x = 0; x < W; ++x)
            for (int k = 0; k < nd; ++k) {
                int d = j->planes ? j->planes[k] : k;
                int t = x - d + (D - 1);
                j->C[((long)y * W + x) * nd + k] =
                    zncc_one(j->L, j->R, W, H, r, mL[x], sL[x], mR[t], sR[t], x, (int)y, d);
            }
    }
    free(mR);
    free(mL);
}

/* Cost volume C(x,y,d) of Eq. (1) for d in [0, D) (planes == NULL, nd == D) or for the   */
/* listed planes only (planes[k] in [0, D), output plane k). Layout [H][W][nd].            */

int oracle_zncc_volume(const uint8_t* L, const uint8_t* R, int W, int H, int D, int r,
                       const int* planes, int nd, int nthreads, double* C) {
    if (!L || !R || !C || W < 1 || H < 1 || D < 1 || r < 0 || nd < 1) return ORACLE_EINVAL;
    if (!planes && nd != D) return ORACLE_EINVAL;
    if (planes)
        for (int k = 0; k < nd; ++k)
            if (planes[k] < 0 || planes[k] >= D) return ORACLE_EINVAL;
    zncc_job job = {L, R, W, H, D, r, nd, planes, C};
    parallel_for(H, nthreads, zncc_rows, &job);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------------------ */
/* DT weights. form 0: Eq. (11), W = K * exp(-|dI| / sigma_r), K = exp(-1/sigma_s).        */
/* form 1: Eqs. (7)-(10), W = a^(1 + sigma_s/sigma_r * |dI|), a = exp(-1/sigma_s).          */
/* dI is the difference of the guide (uint8 / 255) between the pixel and its neighbour:    */
/* W_L: (x-1,y), W_R: (x+1,y), W_U: (x,y-1), W_D: (x,y+1). Undefined borders are set to 0  */
/* (they are never used: each pass starts from its boundary condition there).             */

static double dt_weight(double gdiff, double sigma_s, double sigma_r, int form) {
    if (form == 1) {
        double a = exp(-1.0 / sigma_s);
        return pow(a, 1.0 + sigma_s / sigma_r * fabs(gdiff));
    }
    double K = exp(-1.0 / sigma_s);
    return K * exp(-fabs(gdiff) / sigma_r);
}

int oracle_dt_weights(const uint8_t* guide, int W, int H, double sigma_s, double sigma_r,
                      int form, double* WL, double* WR, double* WU, double* WD) {
    if (!guide || W < 1 || H < 1 || !(sigma_s > 0) || !(sigma_r > 0)) return ORACLE_EINVAL;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double g = guide[(long)y * W + x] / 255.0;
            long i = (long)y * W + x;
            WL[i] = x > 0 ? dt_weight(g - guide[i - 1] / 255.0, sigma_s, sigma_r, form) : 0.0;
            WR[i] = x < W - 1 ? dt_weight(g - guide[i + 1] / 255.0, sigma_s, sigma_r, form) : 0.0;
            WU[i] = y > 0 ? dt_weight(g - guide[i - W] / 255.0, sigma_s, sigma_r, form) : 0.0;
            WD[i] = y < H - 1 ? dt_weight(g - guide[i + W] / 255.0, sigma_s, sigma_r, form) : 0.0;
        }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------------------ */
/* DT aggregation, Eqs. (3)-(6), in place on C [H][W][nd]. One iteration runs, in order:   */
/*   C_L(x) = s*C(x)   + C_L(x-1) * W_L(x),   C_L(0)   = s*C(0)                            */
/*   C_R(x) = s*C_L(x) + C_R(x+1) * W_R(x),   C_R(W-1) = s*C_L(W-1)                        */
/*   C_U(y) = s*C_R(y) + C_U(y-1) * W_U(y),   C_U(0)   = s*C_R(0)                          */
/*   C_D(y) = s*C_U(y) + C_D(y+1) * W_D(y),   C_D(H-1) = s*C_U(H-1)                        */
/* and C := C_D. s = 1 is the paper's literal form; s = 1-K the scaled form.               */

typedef struct {
    double* C;
    int W, H, nd;
    const double* w;
    double s;
} pass_job;

static void pass_l2r(void* p, long y0, long y1) {
    pass_job* j = (pass_job*)p;
    for (long y = y0; y < y1; ++y)
        for (int x = 0; x < j->W; ++x) {
            double* c = j->C + ((long)y * j->W + x) * j->nd;
            double wgt = j->w[(long)y * j->W + x];
            for (int k = 0; k < j->nd; ++k)
                c[k] = x == 0 ? j->s * c[k] : j->s * c[k] + c[k - j->nd] * wgt;
        }
}

static void pass_r2l(void* p, long y0, long y1) {
    pass_job* j = (pass_job*)p;
    for (long y = y0; y < y1; ++y)
        for (int x = j->W - 1; x >= 0; --x) {
            double* c = j->C + ((long)y * j->W + x) * j->nd;
            double wgt = j->w[(long)y * j->W + x];
            for (int k = 0; k < j->nd; ++k)
                c[k] = x == j->W - 1 ? j->s * c[k] : j->s * c[k] + c[k + j->nd] * wgt;
        }
}

static void pass_u2d(void* p, long x0, long x1) {
    pass_job* j = (pass_job*)p;
    long row = (long)j->W * j->nd;
    for (long x = x0; x < x1; ++x)
        for (int y = 0; y < j->H; ++y) {
            double* c = j->C + ((long)y * j->W + x) * j->nd;
            double wgt = j->w[(long)y * j->W + x];
            for (int k = 0; k < j->nd; ++k)
                c[k] = y == 0 ? j->s * c[k] : j->s * c[k] + c[k - row] * wgt;
        }
}

static void pass_d2u(void* p, long x0, long x1) {
    pass_job* j = (pass_job*)p;
    long row = (long)j->W * j->nd;
    for (long x = x0; x < x1; ++x)
        for (int y = j->H - 1; y >= 0; --y) {
            double* c = j->C + ((long)y * j->W + x) * j->nd;
            double wgt = j->w[(long)y * j->W + x];
            for (int k = 0; k < j->nd; ++k)
                c[k] = y == j->H - 1 ? j->s * c[k] : j->s * c[k] + c[k + row] * wgt;
        }
}

int oracle_dt_aggregate(double* C, int W, int H, int nd, const double* WL, const double* WR,
                        const double* WU, const double* WD, double sigma_s, int iters,
                        int scaled, int nthreads) {
    if (!C || !WL || !WR || !WU || !WD || W < 1 || H < 1 || nd < 1 || iters < 0 ||
        !(sigma_s > 0))
        return ORACLE_EINVAL;
    double s = scaled ? 1.0 - exp(-1.0 / sigma_s) : 1.0;
    for (int it = 0; it < iters; ++it) {
        pass_job jl = {C, W, H, nd, WL, s}, jr = {C, W, H, nd, WR, s};
        pass_job ju = {C, W, H, nd, WU, s}, jd = {C, W, H, nd, WD, s};
        parallel_for(H, nthreads, pass_l2r, &jl);
        parallel_for(H, nthreads, pass_r2l, &jr);
        parallel_for(W, nthreads, pass_u2d, &ju);
        parallel_for(W, nthreads, pass_d2u, &jd);
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------------------ */
/* WTA, Eq. (WTA1): D_map(x,y) = argmin_d (1 - C(x,y,d)); the smallest such d on ties.     */
/* Also returns the winning value and the gap to the best value at any other d (the gap is */
/* +inf when nd == 1).                                                                    */

int oracle_wta(const double* C, int W, int H, int nd, uint16_t* disp, double* best,
               double* gap) {
    if (!C || !disp || W < 1 || H < 1 || nd < 1 || nd > 65535) return ORACLE_EINVAL;
    for (long p = 0; p < (long)W * H; ++p) {
        const double* c = C + p * nd;
        int bd = 0;
        double bcost = 1.0 - c[0];
        for (int d = 1; d < nd; ++d)
            if (1.0 - c[d] < bcost) { bcost = 1.0 - c[d]; bd = d; }
        double second = INFINITY;
        for (int d = 0; d < nd; ++d)
            if (d != bd && 1.0 - c[d] < second) second = 1.0 - c[d];
        disp[p] = (uint16_t)bd;
        if (best) best[p] = c[bd];
        if (gap) gap[p] = second - bcost;
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------------------ */
/* FastDT storage (Sec. IV-C): cost-value normalization with nearly zero mean, 16-bit      */
/* integers, and the 8-bit code of a 6-bit value and a 2-bit position flag.                */
/*                                                                                        */
/* Encoding of a 16-bit two's-complement value: values >= 0 give the code 0. A negative    */
/* value keeps six bits next to its leading ones: bits 14..9 with flag 01 unless bits     */
/* 14..11 are all ones; else bits 10..5 with flag 10 unless bits 10..7 are all ones; else */
/* bits 6..1 with flag 11. The code is (six bits << 2) | flag.                            */
/* Decoding: code 0 gives 0; otherwise the six bits go back to their position, every bit   */
/* above them is set to one and every bit below them to zero.                             */

uint8_t oracle_fastdt_encode(int16_t value) {
    if (value >= 0) return 0;
    unsigned v = (unsigned)(uint16_t)value;
    unsigned hi4 = (v >> 11) & 0xF, mid4 = (v >> 7) & 0xF;
    if (hi4 != 0xF) return (uint8_t)((((v >> 9) & 0x3F) << 2) | 1u);
    if (mid4 != 0xF) return (uint8_t)((((v >> 5) & 0x3F) << 2) | 2u);
    return (uint8_t)((((v >> 1) & 0x3F) << 2) | 3u);
}

int16_t oracle_fastdt_decode(uint8_t code) {
    if (code == 0) return 0;
    unsigned flag = code & 3u, six = code >> 2;
    int low = flag == 1 ? 9 : (flag == 2 ? 5 : 1);      /* position of the six bits */
    if (flag == 0) low = 1;                              /* not produced by the encoder */
    unsigned v = six << low;
    for (int b = low + 6; b < 16; ++b) v |= 1u << b;      /* ones above, zeros below */
    return (int16_t)(uint16_t)v;
}

/* One FastDT store of a [H][W][nd] volume in place, after a pass pair whose all-ones      */
/* response is ahat [H][W] (the per-pixel bound of |C|): per pixel, the near-zero-mean     */
/* normalization against disparity d_arb, e = (C(d_arb) - C(d)) / ahat (e < 0 where d does */
/* better than d_arb under the argmax), the 16-bit value E = rint(T e) clamped to int16,   */
/* its 8-bit code, and back: C(d) = -decode(code) / T * ahat. Values that do no better     */
/* than d_arb come back as 0, like C(d_arb) itself.                                        */
int oracle_fastdt_store(double* C, const double* ahat, int W, int H, int nd, int d_arb, double T) {
    if (!C || !ahat || W < 1 || H < 1 || nd < 1 || d_arb < 0 || d_arb >= nd || !(T > 0)) return ORACLE_EINVAL;
    for (long p = 0; p < (long)W * H; ++p) {
        double* c = C + p * nd;
        const double ref = c[d_arb], a = ahat[p];
        for (int d = 0; d < nd; ++d) {
            double e = rint(T * (ref - c[d]) / a);
            if (e < -32768.0) e = -32768.0;
            if (e > 32767.0) e = 32767.0;
            const int16_t E = oracle_fastdt_decode(oracle_fastdt_encode((int16_t)e));
            c[d] = -(double)E / T * a;
        }
    }
    return ORACLE_OK;
}

/* The DT chain with FastDT storage between pass pairs: after every pass pair but the last */
/* (the last feeds WTA directly) the volume goes through oracle_fastdt_store with the      */
/* all-ones response after the same number of pairs.                                       */
int oracle_dt_aggregate_fastdt(double* C, const uint8_t* guide, int W, int H, int nd, double sigma_s,
                               double sigma_r, int iters, int d_arb, double T, int nthreads) {
    if (!C || !guide || W < 1 || H < 1 || nd < 1 || iters < 0 || !(sigma_s > 0) || !(sigma_r > 0))
        return ORACLE_EINVAL;
    size_t n = (size_t)W * H;
    double* w = (double*)malloc(sizeof(double) * n * 5);
    if (!w) return ORACLE_ENOMEM;
    double* ones = w + 4 * n;
    int rc = oracle_dt_weights(guide, W, H, sigma_s, sigma_r, 0, w, w + n, w + 2 * n, w + 3 * n);
    for (size_t i = 0; i < n; ++i) ones[i] = 1.0;
    const double s = 1.0 - exp(-1.0 / sigma_s);
    for (int pair = 1; rc == ORACLE_OK && pair <= 2 * iters; ++pair) {
        const int horiz = pair % 2;
        pass_job a = {C, W, H, nd, horiz ? w : w + 2 * n, s}, b = {C, W, H, nd, horiz ? w + n : w + 3 * n, s};
        pass_job oa = {ones, W, H, 1, horiz ? w : w + 2 * n, s}, ob = {ones, W, H, 1, horiz ? w + n : w + 3 * n, s};
        if (horiz) {
            parallel_for(H, nthreads, pass_l2r, &a);
            parallel_for(H, nthreads, pass_r2l, &b);
            parallel_for(H, nthreads, pass_l2r, &oa);
            parallel_for(H, nthreads, pass_r2l, &ob);
        } else {
            parallel_for(W, nthreads, pass_u2d, &a);
            parallel_for(W, nthreads, pass_d2u, &b);
            parallel_for(W, nthreads, pass_u2d, &oa);
            parallel_for(W, nthreads, pass_d2u, &ob);
        }
        if (pair < 2 * iters) rc = oracle_fastdt_store(C, ones, W, H, nd, d_arb, T);
    }
    free(w);
    return rc;
}

/* ------------------------------------------------------------------------------------ */
/* The whole path on one pair: ZNCC volume, DT (scaled form, guide = left), WTA.           */
/* iters == 0 skips the aggregation. C (optional, [H][W][D]) receives the aggregated cost. */

int oracle_run(const uint8_t* L, const uint8_t* R, int W, int H, int D, int r,
               double sigma_s, double sigma_r, int iters, int nthreads, uint16_t* disp,
               double* gap, double* C_out) {
    if (!L || !R || !disp || W < 1 || H < 1 || D < 1 || r < 0 || iters < 0) return ORACLE_EINVAL;
    size_t n = (size_t)W * H;
    double* C = C_out ? C_out : (double*)malloc(sizeof(double) * n * D);
    if (!C) return ORACLE_ENOMEM;
    int rc = oracle_zncc_volume(L, R, W, H, D, r, NULL, D, nthreads, C);
    if (rc == ORACLE_OK && iters > 0) {
        double* w = (double*)malloc(sizeof(double) * n * 4);
        if (!w) rc = ORACLE_ENOMEM;
        else {
            rc = oracle_dt_weights(L, W, H, sigma_s, sigma_r, 0, w, w + n, w + 2 * n, w + 3 * n);
            if (rc == ORACLE_OK)
                rc = oracle_dt_aggregate(C, W, H, D, w, w + n, w + 2 * n, w + 3 * n, sigma_s,
                                         iters, 1, nthreads);
            free(w);
        }
    }
    if (rc == ORACLE_OK) rc = oracle_wta(C, W, H, D, disp, NULL, gap);
    if (!C_out) free(C);
    return rc;
}
