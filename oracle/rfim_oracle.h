/*
 * rfim_oracle.h -- CPU oracle for the time- and frequency-domain sigma cuts.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, single-threaded
 * reference that the GPU library is checked against.  Only the test suite,
 * the package smoke check and the CPU-baseline leg of the benchmark may load
 * it.  It shares no code, header, table or constant with the CUDA library.
 *
 * Method (Sclocco, Vohl, van Nieuwpoort, "Real-Time RFI Mitigation for the
 * Apertif Radio Transient System", arXiv:2001.03389):
 *   TDSC  Sec. IV, TDSC paragraph and Fig. 2: per (beam, channel), compare every
 *         time sample of the batch with the batch mean and standard deviation;
 *         |x - mu| > k sigma (symmetric, Fig. 2 caption) flags the sample,
 *         which is replaced by the batch mean.
 *   FDSC  Sec. IV, FDSC paragraph and Fig. 3: per (beam, time sample), subtract
 *         from each channel the mean of its channel bin, compare the corrected
 *         value with the mean and standard deviation of the corrected values of
 *         all channels, and replace an outlier's ORIGINAL value by its bin mean.
 *   Replacement strategy parameter (mean or median): Sec. IV, last paragraph.
 *   Iterations: Sec. V-A (three iterations in production) and Sec. V-B.
 *
 * Readings taken where the paper is silent (all listed in the design notes):
 *   - sigma is the population standard deviation (divide by the count);
 *   - statistics of each iteration are taken over all current values of the
 *     row/column, including values replaced by earlier iterations;
 *   - uint8 decisions use exact integers and a single IEEE rounding:
 *       TDSC: flag iff (double)((T*x - S)^2) > fl(k2 * (double)(T*Q - S^2)),
 *       FDSC: flag iff (double)(C*D^2) > fl(k2 * (double)sum(D^2)), with
 *             D = (L/G_g)(G_g*x - S_g), L = lcm of the bin sizes,
 *     where k2 = fl(k*k);
 *   - uint8 mean replacement rounds half up: floor((2S + n) / (2n));
 *   - median replacement is the lower median (rank floor((n-1)/2), 0-based)
 *     of the current values, taken over all of them;
 *   - FDSC bins are contiguous groups of `bin` channels, the last one may be
 *     shorter; bin == C is the single-bin (bandpass-corrected) case;
 *   - the combined cleaner runs all TDSC iterations on every row, then all
 *     FDSC iterations on every column of the TDSC output;
 *   - flags: one byte per sample, bit 0 = TDSC, bit 1 = FDSC, OR-ed over
 *     iterations.
 *   - float32 inputs must be finite; the float median orders -0 before +0.
 */
#ifndef RFIM_ORACLE_H
#define RFIM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* layout: 0 = beam x channel x time (time fastest), 1 = beam x time x channel */
#define ORC_LAYOUT_BCT 0
#define ORC_LAYOUT_BTC 1
/* replacement strategy */
#define ORC_REPLACE_MEAN 0
#define ORC_REPLACE_MEDIAN 1
#define ORC_REPLACE_RANDOM 2 /* a random unflagged sample of the same row / bin */
/* return codes */
#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_RANGE 2

/* One cut's parameters. enabled == 0 skips the method in orc_clean_*. */
typedef struct {
  int enabled;
  double k;        /* threshold in units of sigma, > 0 */
  int iterations;  /* 1..16 */
  int replace;     /* ORC_REPLACE_* */
  int bin;         /* FDSC channel-bin size, 1..C (ignored for TDSC) */
} orc_cut;

/* in and out may alias exactly (in-place).  flags: B*C*T bytes, nullable. */
int orc_clean_u8(const uint8_t* in, uint8_t* out, uint8_t* flags,
                 int64_t B, int64_t C, int64_t T, int layout,
                 const orc_cut* tdsc, const orc_cut* fdsc);
int orc_clean_f32(const float* in, float* out, uint8_t* flags,
                  int64_t B, int64_t C, int64_t T, int layout,
                  const orc_cut* tdsc, const orc_cut* fdsc);

/* Single-row / single-column primitives (exported for the pinning tests). */
void orc_tdsc_row_u8(uint8_t* x, uint8_t* f, int64_t n, double k, int iters, int replace);
void orc_fdsc_col_u8(uint8_t* x, uint8_t* f, int64_t n, double k, int iters, int replace, int64_t bin);
void orc_tdsc_row_f32(float* x, uint8_t* f, int64_t n, double k, int iters, int replace);
void orc_fdsc_col_f32(float* x, uint8_t* f, int64_t n, double k, int iters, int replace, int64_t bin);

/* Random replacement: SplitMix64 output function, and the position in
 * [0, n) of attempt `attempt` for (method 1 = TDSC / 2 = FDSC, iteration,
 * beam, line, index) -- line/index = channel/time for TDSC, time/channel for
 * FDSC (where the position is within the bin). */
uint64_t orc_mix64(uint64_t z);
int64_t orc_draw(int method, int it, int64_t beam, int64_t line, int64_t index, int attempt, int64_t n);
/* the row/column cuts with the beam and line that key the random draws, and
 * it0, the index of their first iteration (iteration i draws with it0 + i) */
void orc_tdsc_row_u8x(uint8_t* x, uint8_t* f, int64_t n, double k, int iters, int replace, int64_t beam,
                      int64_t line, int it0);
void orc_fdsc_col_u8x(uint8_t* x, uint8_t* f, int64_t n, double k, int iters, int replace, int64_t bin,
                      int64_t beam, int64_t line, int it0);
void orc_tdsc_row_f32x(float* x, uint8_t* f, double* margin, int64_t n, double k, int iters, int replace,
                       int64_t beam, int64_t line, int it0);
void orc_fdsc_col_f32x(float* x, uint8_t* f, double* margin, int64_t n, double k, int iters, int replace,
                       int64_t bin, int64_t beam, int64_t line, int it0);

/* The combined cleaner in interleaved order: round i applies TDSC iteration i
 * to every row, then FDSC iteration i to every column (single-iteration cuts
 * on the current values, random draws keyed by iteration i), for
 * max(iterations) rounds -- the method with more iterations runs alone in the
 * last rounds; flags OR over rounds. */
int orc_clean_u8_interleaved(const uint8_t* in, uint8_t* out, uint8_t* flags,
                             int64_t B, int64_t C, int64_t T, int layout,
                             const orc_cut* tdsc, const orc_cut* fdsc);
int orc_clean_f32_interleaved(const float* in, float* out, uint8_t* flags,
                              int64_t B, int64_t C, int64_t T, int layout,
                              const orc_cut* tdsc, const orc_cut* fdsc);

/* The same float32 cuts with a diagnostic output (nullable): margin[i] is the
 * minimum over the sample's decisions of |(|x - mu| - k sigma)| / (k sigma),
 * its relative distance from the nearest threshold (INFINITY where sigma = 0). */
int orc_clean_f32m(const float* in, float* out, uint8_t* flags, double* margin,
                   int64_t B, int64_t C, int64_t T, int layout,
                   const orc_cut* tdsc, const orc_cut* fdsc);
void orc_tdsc_row_f32m(float* x, uint8_t* f, double* margin, int64_t n, double k, int iters, int replace);
void orc_fdsc_col_f32m(float* x, uint8_t* f, double* margin, int64_t n, double k, int iters, int replace,
                       int64_t bin);
uint8_t orc_lower_median_u8(const uint8_t* x, int64_t n);
float orc_lower_median_f32(const float* x, int64_t n);

#ifdef __cplusplus
}
#endif
#endif
