/*
 * ds_oracle.h -- CPU oracle for the separable decimating FIR ("downscaler")
 * filter stage of Rodrigues, Guyomarc'h and Dekeyser, "Programming Massively
 * Parallel Architectures using MARTE: a Case Study" (arXiv:1103.4881).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain reference that
 * the CUDA library is checked against.  Only the test-suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or helper with the CUDA library under paper_1103_4881_b300/.
 *
 * What it computes (paper Sec. 3 "Case Study: H.263 Video Downscaling"):
 * a horizontal filter followed by a vertical filter, each one mapping
 * packets of q input pixels to p output pixels; every output is a K-tap
 * dot product over a window of the line (Sec. 3, first paragraph).  The
 * windows are described with an Array-OL tiler -- origin, paving, fitting
 * -- over a repetition space of independent elementary tasks (Sec. 3.A,
 * "Downscaler Model": task yhfk, repetition [288,44]).
 *
 * The paper gives no coefficients, no window placement and no boundary rule;
 * the readings used here are:
 *   - output extent per axis  n_out = floor(n_in * p / q);
 *   - phase j of block r: centre c_j = (j + 1/2) q / p - 1/2 (pixel-centre
 *     alignment), window start b_j = floor(c_j) - K/2 + 1 relative to r*q;
 *   - weights: Lanczos-3, L(x) = sinc(x) sinc(x/3) for |x| < 3, stretched by
 *     sigma = 6/K so the support fills the K-tap window, normalised to sum 1;
 *   - clamp-to-edge at the frame border;
 *   - uint8 path: Q14 taps (round half up, residual to the largest tap),
 *     integer accumulation, (acc + 2^13) >> 14 with a floor shift, clamp to
 *     [0,255], after each pass.
 *
 * Floating point: FP64 throughout, inputs given already decoded to double.
 * Integer: int64 accumulation.
 *
 * Errors: every function returns 0 on success and a negative value on a bad
 * argument (nothing is written in that case).
 */
#ifndef DS_ORACLE_H
#define DS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* floor(n_in * p / q) */
long dso_out_extent(long n_in, int p, int q);

/* Phase windows: b[j] (window start offset from r*q) and c[j] (centre), j<p. */
int dso_phase_windows(int p, int q, int K, int* b, double* c);

/* FP64 taps, row-major [p][K]; each row sums to 1. */
int dso_taps_f64(int p, int q, int K, double* w);

/* Q14 taps, row-major [p][K]; each row sums to 16384 exactly. */
int dso_taps_q14(int p, int q, int K, int32_t* qt);

/* Separable filter, H pass then V pass, FP64.
 * x: n_frames x H x W x C doubles (row-major, channels interleaved);
 * y: n_frames x floor(H p/q) x floor(W p/q) x C doubles.
 * n_threads <= 0: all OpenMP threads; 1: single thread. */
int dso_filter_f64(const double* x, double* y, long n_frames, int H, int W, int C,
                   int p, int q, int K, int n_threads);

/* Separable filter on uint8 with Q14 taps and a uint8 intermediate. */
int dso_filter_u8(const uint8_t* x, uint8_t* y, long n_frames, int H, int W, int C,
                  int p, int q, int K, int n_threads);

/* Q14 of any tap table w[p][K]: round half up, the residual
 * floor(16384 * row sum + 1/2) - sum(q) on the largest tap of the row. */
int dso_quantize_q14(const double* w, int p, int K, int32_t* qt);

/* Extended filter: a ratio, tap count and (optionally) tap table per axis,
 * and the boundary of the tilers: 0 = clamp-to-edge, 1 = modular (Array-OL
 * tilers index modulo the array's shape).  taps_h / taps_v NULL: the
 * Lanczos-3 taps above; else FP64 tables [p][K] used as given. */
typedef struct {
    int ph, qh, Kh;
    int pv, qv, Kv;
    int boundary;
    const double* taps_h;
    const double* taps_v;
} dso_axes;

int dso_filter_ex_f64(const double* x, double* y, long n_frames, int H, int W, int C,
                      const dso_axes* ax, int n_threads);
int dso_filter_ex_u8(const uint8_t* x, uint8_t* y, long n_frames, int H, int W, int C,
                     const dso_axes* ax, int n_threads);

/* Number of OpenMP threads a parallel region would use (0 if built without). */
int dso_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
