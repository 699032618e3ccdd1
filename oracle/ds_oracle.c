/*
 * ds_oracle.c -- CPU oracle (TEST INFRASTRUCTURE ONLY; see ds_oracle.h).
 *
 * A literal loop nest over the Array-OL tilers of the downscaler's
 * horizontal and vertical filters (paper Sec. 3 and Sec. 3.A).  No blocking,
 * no fusion, no reordering: for every repetition index the input pattern is
 * gathered through the tiler (origin + paving * r + fitting * i, clamped to
 * the frame), then the elementary task turns that pattern into p outputs.
 *
 * Built with -ffp-contract=off so that every FP64 product and sum is rounded
 * as written.
 */
#include "ds_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define DSO_PI 3.14159265358979323846

/* ---------------------------------------------------------------------- */
/* Shapes                                                                   */
/* ---------------------------------------------------------------------- */

/* Output extent: floor(n_in * p / q).  352 -> 132 at 3/8 (paper Sec. 3). */
long dso_out_extent(long n_in, int p, int q) {
    if (n_in < 0 || p <= 0 || q <= 0) return -1;
    return (n_in * (long)p) / (long)q;
}

static int gcd_int(int a, int b) {
    while (b) { int t = a % b; a = b; b = t; }
    return a;
}

static int check_filter_args(int p, int q, int K) {
    if (p <= 0 || q <= 0 || p >= q) return -1;
    if (gcd_int(p, q) != 1) return -1;
    if (K < 2 || K > 16 || (K % 2) != 0) return -1;
    return 0;
}

/* floor(a / b) for b > 0 */
static long floor_div(long a, long b) {
    long d = a / b;
    if ((a % b) != 0 && a < 0) d -= 1;
    return d;
}

/* ---------------------------------------------------------------------- */
/* Phase windows and taps                                                   */
/* ---------------------------------------------------------------------- */

/*
 * Phase j of a block (j < p): centre c_j = (j + 1/2) q / p - 1/2 in input
 * coordinates relative to the block start r*q; the K-tap window starts at
 * b_j = floor(c_j) - K/2 + 1.  floor(c_j) is taken with integers:
 * c_j = ((2j+1) q - p) / (2p).
 */
int dso_phase_windows(int p, int q, int K, int* b, double* c) {
    if (check_filter_args(p, q, K)) return -1;
    for (int j = 0; j < p; ++j) {
        long num = (long)(2 * j + 1) * q - p;
        long den = 2L * p;
        if (c) c[j] = (double)num / (double)den;
        if (b) b[j] = (int)(floor_div(num, den) - K / 2 + 1);
    }
    return 0;
}

/* sinc(x) = sin(pi x) / (pi x), sinc(0) = 1 */
static double sinc(double x) {
    if (x == 0.0) return 1.0;
    double px = DSO_PI * x;
    return sin(px) / px;
}

/* Lanczos-3 kernel: sinc(x) sinc(x/3) on |x| < 3, zero elsewhere. */
static double lanczos3(double x) {
    if (fabs(x) >= 3.0) return 0.0;
    return sinc(x) * sinc(x / 3.0);
}

/*
 * w_j[t] = L(sigma (b_j + t - c_j)) / sum_t L(...), sigma = 6/K: the
 * Lanczos-3 support (|x| < 3) stretched over the K-tap window.
 */
int dso_taps_f64(int p, int q, int K, double* w) {
    if (check_filter_args(p, q, K) || !w) return -1;
    int b[64];
    double c[64];
    if (p > 64) return -1;
    dso_phase_windows(p, q, K, b, c);
    double sigma = 6.0 / (double)K;
    for (int j = 0; j < p; ++j) {
        double sum = 0.0;
        for (int t = 0; t < K; ++t) {
            double v = lanczos3(sigma * ((double)(b[j] + t) - c[j]));
            w[j * K + t] = v;
            sum += v;
        }
        for (int t = 0; t < K; ++t) w[j * K + t] /= sum;
    }
    return 0;
}

/*
 * Q14: q = floor(w * 16384 + 1/2); the residual 16384 - sum(q) goes to the
 * tap with the largest w (lowest index on ties), so a constant frame is
 * reproduced exactly.
 */
int dso_taps_q14(int p, int q, int K, int32_t* qt) {
    if (check_filter_args(p, q, K) || !qt) return -1;
    if (p > 64) return -1;
    double w[64 * 16];
    dso_taps_f64(p, q, K, w);
    return dso_quantize_q14(w, p, K, qt);
}

/*
 * Q14 of any tap table w[p][K]: q = floor(w * 16384 + 1/2), then the
 * residual floor(16384 * sum(w) + 1/2) - sum(q) goes to the tap with the
 * largest w (lowest index on ties).  For rows that sum to 1 this is the
 * rule above: each row of q sums to 16384 exactly.
 */
int dso_quantize_q14(const double* w, int p, int K, int32_t* qt) {
    if (!w || !qt || p < 1 || K < 1) return -1;
    for (int j = 0; j < p; ++j) {
        long sum = 0;
        double wsum = 0.0;
        int big = 0;
        for (int t = 0; t < K; ++t) {
            qt[j * K + t] = (int32_t)floor(w[j * K + t] * 16384.0 + 0.5);
            sum += qt[j * K + t];
            wsum += w[j * K + t];
            if (w[j * K + t] > w[j * K + big]) big = t;
        }
        qt[j * K + big] += (int32_t)((long)floor(wsum * 16384.0 + 0.5) - sum);
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Array-OL tiler along one axis                                            */
/* ---------------------------------------------------------------------- */

/*
 * Input tiler of one filter pass along an axis of length n (Sec. 3.A): the
 * pattern of repetition r has `pattern` elements, element i read at
 * origin + paving * r + fitting * i, clamped to [0, n-1].  The output
 * tiler writes p elements per repetition at paving p.
 */
typedef struct {
    int origin;      /* b_0: first tap offset of phase 0                */
    int paving;      /* q: input step between repetitions               */
    int fitting;     /* 1: step between pattern elements                */
    int pattern;     /* b_{p-1} + K - b_0: elements one task reads      */
    long repetition; /* ceil(n_out / p): tasks along the axis           */
    long n_in;
    long n_out;
    int wrap;        /* 0: clamp to the array; 1: modulo its extent     */
} dso_tiler;

static void make_tiler(dso_tiler* tl, long n_in, int p, int q, int K, const int* b, int wrap) {
    tl->origin = b[0];
    tl->paving = q;
    tl->fitting = 1;
    tl->pattern = b[p - 1] + K - b[0];
    tl->n_in = n_in;
    tl->n_out = dso_out_extent(n_in, p, q);
    tl->repetition = (tl->n_out + p - 1) / p;
    tl->wrap = wrap;
}

static long clamp_index(long i, long n) {
    if (i < 0) return 0;
    if (i > n - 1) return n - 1;
    return i;
}

/* Array-OL tilers index modulo the array's shape (the toroidal reading). */
static long wrap_index(long i, long n) {
    long m = i % n;
    return m < 0 ? m + n : m;
}

static long tiler_index(const dso_tiler* tl, long r, int i) {
    long k = (long)tl->origin + (long)tl->paving * r + (long)tl->fitting * i;
    return tl->wrap ? wrap_index(k, tl->n_in) : clamp_index(k, tl->n_in);
}

/* ---------------------------------------------------------------------- */
/* FP64 filter                                                              */
/* ---------------------------------------------------------------------- */

/*
 * One pass over a 2-D array a[rows][cols] (channels C interleaved) along
 * either the row direction (horizontal: axis = 1) or the column direction
 * (vertical: axis = 0).  For every repetition index (line, r) the pattern
 * is gathered through the tiler and the elementary task emits, for each
 * phase j with r*p + j < n_out, sum_t w_j[t] * pattern[b_j - b_0 + t].
 */
static void pass_f64(const double* a, double* out, long rows, long cols, int C, int axis,
                     int p, int K, const int* b, const double* w, const dso_tiler* tl) {
    long lines = axis == 1 ? rows : cols;
    double* pattern = (double*)malloc(sizeof(double) * (size_t)tl->pattern);
    long out_cols = axis == 1 ? tl->n_out : cols;
    for (long line = 0; line < lines; ++line) {
        for (int ch = 0; ch < C; ++ch) {
            for (long r = 0; r < tl->repetition; ++r) {
                for (int i = 0; i < tl->pattern; ++i) {
                    long k = tiler_index(tl, r, i);
                    pattern[i] = axis == 1 ? a[(line * cols + k) * C + ch]
                                           : a[(k * cols + line) * C + ch];
                }
                for (int j = 0; j < p; ++j) {
                    long o = r * p + j;
                    if (o >= tl->n_out) break;
                    double acc = 0.0;
                    for (int t = 0; t < K; ++t) acc += w[j * K + t] * pattern[b[j] - b[0] + t];
                    if (axis == 1) out[(line * out_cols + o) * C + ch] = acc;
                    else           out[(o * out_cols + line) * C + ch] = acc;
                }
            }
        }
    }
    free(pattern);
}

int dso_filter_f64(const double* x, double* y, long n_frames, int H, int W, int C,
                   int p, int q, int K, int n_threads) {
    if (check_filter_args(p, q, K) || !x || !y) return -1;
    if (n_frames < 0 || H < 1 || W < 1 || C < 1 || p > 64) return -1;
    int b[64];
    double w[64 * 16];
    dso_phase_windows(p, q, K, b, NULL);
    dso_taps_f64(p, q, K, w);
    dso_tiler th, tv;
    make_tiler(&th, W, p, q, K, b, 0);
    make_tiler(&tv, H, p, q, K, b, 0);
    long OW = th.n_out, OH = tv.n_out;
    if (OW < 1 || OH < 1) return -1;
#ifdef _OPENMP
    int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
    for (long f = 0; f < n_frames; ++f) {
        const double* xf = x + f * (long)H * W * C;
        double* yf = y + f * OH * OW * C;
        double* h = (double*)malloc(sizeof(double) * (size_t)H * (size_t)OW * (size_t)C);
        pass_f64(xf, h, H, W, C, 1, p, K, b, w, &th);   /* horizontal filter */
        pass_f64(h, yf, H, OW, C, 0, p, K, b, w, &tv);  /* vertical filter   */
        free(h);
    }
    (void)n_threads;
    return 0;
}

/* ---------------------------------------------------------------------- */
/* uint8 filter (Q14 taps, integer accumulation)                            */
/* ---------------------------------------------------------------------- */

/* (acc + 2^13) >> 14 with a floor shift, clamped to [0, 255] */
static uint8_t q14_to_u8(int64_t acc) {
    int64_t v = floor_div(acc + 8192, 16384);
    if (v < 0) v = 0;
    if (v > 255) v = 255;
    return (uint8_t)v;
}

static void pass_u8(const uint8_t* a, uint8_t* out, long rows, long cols, int C, int axis,
                    int p, int K, const int* b, const int32_t* qt, const dso_tiler* tl) {
    long lines = axis == 1 ? rows : cols;
    int64_t* pattern = (int64_t*)malloc(sizeof(int64_t) * (size_t)tl->pattern);
    long out_cols = axis == 1 ? tl->n_out : cols;
    for (long line = 0; line < lines; ++line) {
        for (int ch = 0; ch < C; ++ch) {
            for (long r = 0; r < tl->repetition; ++r) {
                for (int i = 0; i < tl->pattern; ++i) {
                    long k = tiler_index(tl, r, i);
                    pattern[i] = axis == 1 ? a[(line * cols + k) * C + ch]
                                           : a[(k * cols + line) * C + ch];
                }
                for (int j = 0; j < p; ++j) {
                    long o = r * p + j;
                    if (o >= tl->n_out) break;
                    int64_t acc = 0;
                    for (int t = 0; t < K; ++t) acc += (int64_t)qt[j * K + t] * pattern[b[j] - b[0] + t];
                    uint8_t v = q14_to_u8(acc);
                    if (axis == 1) out[(line * out_cols + o) * C + ch] = v;
                    else           out[(o * out_cols + line) * C + ch] = v;
                }
            }
        }
    }
    free(pattern);
}

int dso_filter_u8(const uint8_t* x, uint8_t* y, long n_frames, int H, int W, int C,
                  int p, int q, int K, int n_threads) {
    if (check_filter_args(p, q, K) || !x || !y) return -1;
    if (n_frames < 0 || H < 1 || W < 1 || C < 1 || p > 64) return -1;
    int b[64];
    int32_t qt[64 * 16];
    dso_phase_windows(p, q, K, b, NULL);
    dso_taps_q14(p, q, K, qt);
    dso_tiler th, tv;
    make_tiler(&th, W, p, q, K, b, 0);
    make_tiler(&tv, H, p, q, K, b, 0);
    long OW = th.n_out, OH = tv.n_out;
    if (OW < 1 || OH < 1) return -1;
#ifdef _OPENMP
    int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
    for (long f = 0; f < n_frames; ++f) {
        const uint8_t* xf = x + f * (long)H * W * C;
        uint8_t* yf = y + f * OH * OW * C;
        uint8_t* h = (uint8_t*)malloc((size_t)H * (size_t)OW * (size_t)C);
        pass_u8(xf, h, H, W, C, 1, p, K, b, qt, &th);   /* horizontal filter */
        pass_u8(h, yf, H, OW, C, 0, p, K, b, qt, &tv);  /* vertical filter   */
        free(h);
    }
    (void)n_threads;
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Extended filter: each axis its own ratio, taps and tap table; boundary   */
/* ---------------------------------------------------------------------- */

typedef struct {
    int p, K;
    int b[64];
    double w[64 * 16];
    int32_t qt[64 * 16];
} dso_axis;

/* Windows of one axis and its taps: Lanczos-3 (the reading above) when
 * `user` is NULL, else the given FP64 table [p][K] as it is. */
static int make_axis(dso_axis* a, int p, int q, int K, const double* user) {
    if (check_filter_args(p, q, K) || p > 64) return -1;
    a->p = p;
    a->K = K;
    dso_phase_windows(p, q, K, a->b, NULL);
    if (user) {
        for (int i = 0; i < p * K; ++i) {
            if (!isfinite(user[i])) return -1;
            a->w[i] = user[i];
        }
    } else {
        dso_taps_f64(p, q, K, a->w);
    }
    return dso_quantize_q14(a->w, p, K, a->qt);
}

static int check_ex(const dso_axes* ax, dso_axis* h, dso_axis* v) {
    if (!ax || (ax->boundary != 0 && ax->boundary != 1)) return -1;
    if (make_axis(h, ax->ph, ax->qh, ax->Kh, ax->taps_h)) return -1;
    if (make_axis(v, ax->pv, ax->qv, ax->Kv, ax->taps_v)) return -1;
    return 0;
}

int dso_filter_ex_f64(const double* x, double* y, long n_frames, int H, int W, int C, const dso_axes* ax,
                      int n_threads) {
    dso_axis ah, av;
    if (!x || !y || check_ex(ax, &ah, &av)) return -1;
    if (n_frames < 0 || H < 1 || W < 1 || C < 1) return -1;
    dso_tiler th, tv;
    make_tiler(&th, W, ah.p, ax->qh, ah.K, ah.b, ax->boundary);
    make_tiler(&tv, H, av.p, ax->qv, av.K, av.b, ax->boundary);
    long OW = th.n_out, OH = tv.n_out;
    if (OW < 1 || OH < 1) return -1;
#ifdef _OPENMP
    int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
    for (long f = 0; f < n_frames; ++f) {
        const double* xf = x + f * (long)H * W * C;
        double* yf = y + f * OH * OW * C;
        double* hbuf = (double*)malloc(sizeof(double) * (size_t)H * (size_t)OW * (size_t)C);
        pass_f64(xf, hbuf, H, W, C, 1, ah.p, ah.K, ah.b, ah.w, &th);   /* horizontal filter */
        pass_f64(hbuf, yf, H, OW, C, 0, av.p, av.K, av.b, av.w, &tv);  /* vertical filter   */
        free(hbuf);
    }
    (void)n_threads;
    return 0;
}

int dso_filter_ex_u8(const uint8_t* x, uint8_t* y, long n_frames, int H, int W, int C, const dso_axes* ax,
                     int n_threads) {
    dso_axis ah, av;
    if (!x || !y || check_ex(ax, &ah, &av)) return -1;
    if (n_frames < 0 || H < 1 || W < 1 || C < 1) return -1;
    dso_tiler th, tv;
    make_tiler(&th, W, ah.p, ax->qh, ah.K, ah.b, ax->boundary);
    make_tiler(&tv, H, av.p, ax->qv, av.K, av.b, ax->boundary);
    long OW = th.n_out, OH = tv.n_out;
    if (OW < 1 || OH < 1) return -1;
#ifdef _OPENMP
    int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
    for (long f = 0; f < n_frames; ++f) {
        const uint8_t* xf = x + f * (long)H * W * C;
        uint8_t* yf = y + f * OH * OW * C;
        uint8_t* hbuf = (uint8_t*)malloc((size_t)H * (size_t)OW * (size_t)C);
        pass_u8(xf, hbuf, H, W, C, 1, ah.p, ah.K, ah.b, ah.qt, &th);   /* horizontal filter */
        pass_u8(hbuf, yf, H, OW, C, 0, av.p, av.K, av.b, av.qt, &tv);  /* vertical filter   */
        free(hbuf);
    }
    (void)n_threads;
    return 0;
}

int dso_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 0;
#endif
}
