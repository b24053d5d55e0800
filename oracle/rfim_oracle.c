/*
 * rfim_oracle.c -- plain single-threaded CPU oracle for TDSC and FDSC.
 *
 * TEST INFRASTRUCTURE ONLY (see rfim_oracle.h): loaded by the tests, the smoke
 * check and the benchmark's CPU-baseline leg, never by the library.  Every
 * function below is a literal loop over the definitions of Sec. IV of the
 * paper; a library sort (qsort) is the only primitive used, to pick medians.
 * Build with -ffp-contract=off so that no multiply-add is fused: every
 * floating-point operation below is one IEEE-754 rounding.
 */
#include "rfim_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define TWO53 9007199254740992LL /* 2^53: integers below it are exact doubles */

/* ------------------------------------------------------------------ */
/* Medians (replacement strategy "median", Sec. IV last paragraph).    */
/* The lower median is the element of rank floor((n-1)/2) of the       */
/* sorted values.                                                     */
/* ------------------------------------------------------------------ */
static int cmp_u8(const void* a, const void* b) {
  return (int)*(const uint8_t*)a - (int)*(const uint8_t*)b;
}

/* Total order on finite floats: numeric order, and -0 before +0. */
static int cmp_f32(const void* a, const void* b) {
  float x = *(const float*)a, y = *(const float*)b;
  if (x < y) return -1;
  if (x > y) return 1;
  int sx = signbit(x) ? 1 : 0, sy = signbit(y) ? 1 : 0;
  return sy - sx; /* equal values: the negative zero sorts first */
}

uint8_t orc_lower_median_u8(const uint8_t* x, int64_t n) {
  uint8_t* tmp = (uint8_t*)malloc((size_t)n);
  memcpy(tmp, x, (size_t)n);
  qsort(tmp, (size_t)n, 1, cmp_u8);
  uint8_t m = tmp[(n - 1) / 2];
  free(tmp);
  return m;
}

float orc_lower_median_f32(const float* x, int64_t n) {
  float* tmp = (float*)malloc((size_t)n * sizeof(float));
  memcpy(tmp, x, (size_t)n * sizeof(float));
  qsort(tmp, (size_t)n, sizeof(float), cmp_f32);
  float m = tmp[(n - 1) / 2];
  free(tmp);
  return m;
}

/* ------------------------------------------------------------------ */
/* TDSC on one (beam, channel) row of n time samples, uint8.           */
/* Sec. IV (TDSC): mu and sigma of the batch; |x - mu| > k sigma flags  */
/* the sample (symmetric test, Fig. 2 caption); flagged samples take   */
/* the replacement value.  With S = sum x, Q = sum x^2:                */
/*   |x - S/n| > k sqrt(Q/n - (S/n)^2)  <=>  (n x - S)^2 > k^2 (n Q - S^2) */
/* evaluated on exact integers with one rounding for k^2 * R.          */
/* ------------------------------------------------------------------ */
/* ------------------------------------------------------------------ */
/* Random replacement (Sec. IV, last paragraph: "random unflagged       */
/* samples"): a flagged sample takes the current value of an unflagged  */
/* sample of the same row (TDSC) or bin (FDSC), found by rejection      */
/* sampling -- attempt a = 0..31 draws a position and takes it if that   */
/* sample is unflagged in this iteration; after 32 misses the sample    */
/* keeps its value.  Draws come from a counter-based hash: the SplitMix64 */
/* output function (Steele, Lea, Flood 2014) of a key built from the    */
/* method, iteration, beam, line, index and attempt.                     */
/* ------------------------------------------------------------------ */
uint64_t orc_mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* position in [0, n) of attempt a; method 1 = TDSC (line = channel, index =
 * time sample), 2 = FDSC (line = time sample, index = channel) */
int64_t orc_draw(int method, int it, int64_t beam, int64_t line, int64_t index, int attempt, int64_t n) {
  const uint64_t h = orc_mix64(orc_mix64(orc_mix64(orc_mix64((uint64_t)beam) ^ (uint64_t)line) ^ (uint64_t)index) ^
                               ((uint64_t)method << 8 | (uint64_t)it << 16 | (uint64_t)attempt << 24));
  return (int64_t)(((h >> 32) * (uint64_t)n) >> 32);
}

#define ORC_ATTEMPTS 32

void orc_tdsc_row_u8(uint8_t* x, uint8_t* f, int64_t n, double k, int iters, int replace) {
  orc_tdsc_row_u8x(x, f, n, k, iters, replace, 0, 0, 0);
}

void orc_tdsc_row_u8x(uint8_t* x, uint8_t* f, int64_t n, double k, int iters, int replace, int64_t beam,
                      int64_t line, int it0) {
  const double k2 = k * k;
  uint8_t* fl = (uint8_t*)malloc((size_t)n);
  for (int it = 0; it < iters; it++) {
    int64_t S = 0, Q = 0;
    for (int64_t t = 0; t < n; t++) {
      S += x[t];
      Q += (int64_t)x[t] * x[t];
    }
    const int64_t R = n * Q - S * S; /* n^2 sigma^2, exact */
    const double thr = k2 * (double)R;
    uint8_t r = 0;
    if (replace == ORC_REPLACE_MEDIAN)
      r = orc_lower_median_u8(x, n);
    else if (replace == ORC_REPLACE_MEAN)
      r = (uint8_t)((2 * S + n) / (2 * n)); /* mean, rounded half up */
    for (int64_t t = 0; t < n; t++) {
      const int64_t d = n * (int64_t)x[t] - S; /* n (x - mu) */
      fl[t] = (double)(d * d) > thr;
    }
    for (int64_t t = 0; t < n; t++) {
      if (!fl[t]) continue;
      if (f) f[t] |= 1;
      if (replace != ORC_REPLACE_RANDOM) {
        x[t] = r;
        continue;
      }
      for (int a = 0; a < ORC_ATTEMPTS; a++) {
        const int64_t u = orc_draw(1, it0 + it, beam, line, t, a, n);
        if (!fl[u]) { /* unflagged samples are not changed in this iteration */
          x[t] = x[u];
          break;
        }
      }
    }
  }
  free(fl);
}

/* ------------------------------------------------------------------ */
/* FDSC on one (beam, time) column of n channels, uint8.               */
/* Sec. IV (FDSC), Fig. 3: step 1, channels are grouped into bins and   */
/* each value minus its bin mean is the mean-corrected sample d; step   */
/* 2, d is compared with the mean mu' and standard deviation sigma' of  */
/* the corrected samples of all channels; an outlier's ORIGINAL value   */
/* is replaced by its bin's replacement value (mean or median).        */
/* With G_g the size of bin g and S_g its sum, d_c = (G_g x_c - S_g)/G_g */
/* and sum_c d_c = 0, so mu' = 0.  Scaling by L = lcm of the bin sizes  */
/* makes D_c = L d_c an integer, and                                    */
/*   |d_c - mu'| > k sigma'  <=>  n D_c^2 > k^2 sum_c D_c^2.            */
/* ------------------------------------------------------------------ */
static int64_t gcd64(int64_t a, int64_t b) {
  while (b) {
    int64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

static int64_t fdsc_lcm(int64_t n, int64_t bin) {
  int64_t last = n - (n - 1) / bin * bin; /* size of the last bin */
  return bin / gcd64(bin, last) * last;
}

void orc_fdsc_col_u8(uint8_t* x, uint8_t* f, int64_t n, double k, int iters, int replace, int64_t bin) {
  orc_fdsc_col_u8x(x, f, n, k, iters, replace, bin, 0, 0, 0);
}

void orc_fdsc_col_u8x(uint8_t* x, uint8_t* f, int64_t n, double k, int iters, int replace, int64_t bin,
                      int64_t beam, int64_t line, int it0) {
  const double k2 = k * k;
  const int64_t nb = (n + bin - 1) / bin;
  const int64_t L = fdsc_lcm(n, bin);
  int64_t* S = (int64_t*)malloc((size_t)nb * sizeof(int64_t));
  int64_t* D = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  uint8_t* r = (uint8_t*)malloc((size_t)nb);
  uint8_t* fl = (uint8_t*)malloc((size_t)n);
  for (int it = 0; it < iters; it++) {
    for (int64_t g = 0; g < nb; g++) {
      const int64_t c0 = g * bin, c1 = (c0 + bin < n) ? c0 + bin : n, G = c1 - c0;
      S[g] = 0;
      for (int64_t c = c0; c < c1; c++) S[g] += x[c];
      if (replace == ORC_REPLACE_MEDIAN)
        r[g] = orc_lower_median_u8(x + c0, G);
      else
        r[g] = (uint8_t)((2 * S[g] + G) / (2 * G));
    }
    int64_t V = 0; /* L^2 * n * sigma'^2 */
    for (int64_t c = 0; c < n; c++) {
      const int64_t g = c / bin;
      const int64_t G = ((g + 1) * bin < n ? bin : n - g * bin);
      D[c] = (L / G) * (G * (int64_t)x[c] - S[g]);
      V += D[c] * D[c];
    }
    const double thr = k2 * (double)V;
    for (int64_t c = 0; c < n; c++) fl[c] = (double)(n * D[c] * D[c]) > thr;
    for (int64_t c = 0; c < n; c++) {
      if (!fl[c]) continue;
      if (f) f[c] |= 2;
      const int64_t g = c / bin, c0 = g * bin;
      if (replace != ORC_REPLACE_RANDOM) {
        x[c] = r[g];
        continue;
      }
      const int64_t G = ((g + 1) * bin < n ? bin : n - g * bin);
      for (int a = 0; a < ORC_ATTEMPTS; a++) {
        const int64_t u = c0 + orc_draw(2, it0 + it, beam, line, c, a, G);
        if (!fl[u]) {
          x[c] = x[u];
          break;
        }
      }
    }
  }
  free(S);
  free(D);
  free(r);
  free(fl);
}

/* ------------------------------------------------------------------ */
/* float32 versions: the same definitions evaluated in IEEE double,     */
/* two-pass statistics summed in index order.                          */
/* ------------------------------------------------------------------ */
/* Relative distance of one decision from its threshold, |(|x - mu| - thr)| / thr,
 * folded into *m as a minimum (diagnostic output for tolerance checks only). */
static void note_margin(double* m, double dist, double thr) {
  if (!m) return;
  const double r = thr > 0.0 ? fabs(dist - thr) / thr : INFINITY;
  if (r < *m) *m = r;
}

void orc_tdsc_row_f32(float* x, uint8_t* f, int64_t n, double k, int iters, int replace) {
  orc_tdsc_row_f32m(x, f, NULL, n, k, iters, replace);
}

void orc_tdsc_row_f32m(float* x, uint8_t* f, double* margin, int64_t n, double k, int iters, int replace) {
  orc_tdsc_row_f32x(x, f, margin, n, k, iters, replace, 0, 0, 0);
}

void orc_tdsc_row_f32x(float* x, uint8_t* f, double* margin, int64_t n, double k, int iters, int replace,
                       int64_t beam, int64_t line, int it0) {
  uint8_t* fl = (uint8_t*)malloc((size_t)n);
  for (int it = 0; it < iters; it++) {
    double s = 0.0;
    for (int64_t t = 0; t < n; t++) s += (double)x[t];
    const double mu = s / (double)n;
    double ss = 0.0;
    for (int64_t t = 0; t < n; t++) {
      const double d = (double)x[t] - mu;
      ss += d * d;
    }
    const double sigma = sqrt(ss / (double)n);
    const double thr = k * sigma;
    const float r = (replace == ORC_REPLACE_MEDIAN) ? orc_lower_median_f32(x, n) : (float)mu;
    for (int64_t t = 0; t < n; t++) {
      if (margin) note_margin(margin + t, fabs((double)x[t] - mu), thr);
      fl[t] = fabs((double)x[t] - mu) > thr;
    }
    for (int64_t t = 0; t < n; t++) {
      if (!fl[t]) continue;
      if (f) f[t] |= 1;
      if (replace != ORC_REPLACE_RANDOM) {
        x[t] = r;
        continue;
      }
      for (int a = 0; a < ORC_ATTEMPTS; a++) {
        const int64_t u = orc_draw(1, it0 + it, beam, line, t, a, n);
        if (!fl[u]) {
          x[t] = x[u];
          break;
        }
      }
    }
  }
  free(fl);
}

void orc_fdsc_col_f32(float* x, uint8_t* f, int64_t n, double k, int iters, int replace, int64_t bin) {
  orc_fdsc_col_f32m(x, f, NULL, n, k, iters, replace, bin);
}

void orc_fdsc_col_f32m(float* x, uint8_t* f, double* margin, int64_t n, double k, int iters, int replace,
                       int64_t bin) {
  orc_fdsc_col_f32x(x, f, margin, n, k, iters, replace, bin, 0, 0, 0);
}

void orc_fdsc_col_f32x(float* x, uint8_t* f, double* margin, int64_t n, double k, int iters, int replace,
                       int64_t bin, int64_t beam, int64_t line, int it0) {
  const int64_t nb = (n + bin - 1) / bin;
  double* m = (double*)malloc((size_t)nb * sizeof(double));
  double* d = (double*)malloc((size_t)n * sizeof(double));
  float* r = (float*)malloc((size_t)nb * sizeof(float));
  uint8_t* fl = (uint8_t*)malloc((size_t)n);
  for (int it = 0; it < iters; it++) {
    for (int64_t g = 0; g < nb; g++) {
      const int64_t c0 = g * bin, c1 = (c0 + bin < n) ? c0 + bin : n;
      double s = 0.0;
      for (int64_t c = c0; c < c1; c++) s += (double)x[c];
      m[g] = s / (double)(c1 - c0);
      r[g] = (replace == ORC_REPLACE_MEDIAN) ? orc_lower_median_f32(x + c0, c1 - c0) : (float)m[g];
    }
    double s = 0.0;
    for (int64_t c = 0; c < n; c++) {
      d[c] = (double)x[c] - m[c / bin];
      s += d[c];
    }
    const double mu = s / (double)n;
    double ss = 0.0;
    for (int64_t c = 0; c < n; c++) {
      const double e = d[c] - mu;
      ss += e * e;
    }
    const double thr = k * sqrt(ss / (double)n);
    for (int64_t c = 0; c < n; c++) {
      if (margin) note_margin(margin + c, fabs(d[c] - mu), thr);
      fl[c] = fabs(d[c] - mu) > thr;
    }
    for (int64_t c = 0; c < n; c++) {
      if (!fl[c]) continue;
      if (f) f[c] |= 2;
      const int64_t g = c / bin, c0 = g * bin;
      if (replace != ORC_REPLACE_RANDOM) {
        x[c] = r[g];
        continue;
      }
      const int64_t G = ((g + 1) * bin < n ? bin : n - g * bin);
      for (int a = 0; a < ORC_ATTEMPTS; a++) {
        const int64_t u = c0 + orc_draw(2, it0 + it, beam, line, c, a, G);
        if (!fl[u]) {
          x[c] = x[u];
          break;
        }
      }
    }
  }
  free(m);
  free(d);
  free(r);
  free(fl);
}

/* ------------------------------------------------------------------ */
/* Whole-block drivers: gather each row / column, run the cut, scatter. */
/* ------------------------------------------------------------------ */
static int check_cut(const orc_cut* c, int is_fdsc, int64_t C) {
  if (!c || !c->enabled) return ORC_OK;
  if (!(c->k > 0.0) || !isfinite(c->k)) return ORC_ERR_ARG;
  if (c->iterations < 1 || c->iterations > 16) return ORC_ERR_ARG;
  if (c->replace != ORC_REPLACE_MEAN && c->replace != ORC_REPLACE_MEDIAN && c->replace != ORC_REPLACE_RANDOM)
    return ORC_ERR_ARG;
  if (is_fdsc && (c->bin < 1 || c->bin > C)) return ORC_ERR_ARG;
  return ORC_OK;
}

static int check_block(int64_t B, int64_t C, int64_t T, int layout, const orc_cut* tdsc, const orc_cut* fdsc) {
  if (B < 1 || C < 1 || T < 1) return ORC_ERR_ARG;
  if (layout != ORC_LAYOUT_BCT && layout != ORC_LAYOUT_BTC) return ORC_ERR_ARG;
  int rc = check_cut(tdsc, 0, C);
  if (rc) return rc;
  return check_cut(fdsc, 1, C);
}

/* Exactness ranges of the integer forms: every product below 2^53. */
static int range_u8(int64_t C, int64_t T, const orc_cut* tdsc, const orc_cut* fdsc) {
  const int64_t lim = TWO53 / 65025; /* 255^2 = 65025 */
  if (tdsc && tdsc->enabled && T * T > lim) return ORC_ERR_RANGE;
  if (fdsc && fdsc->enabled) {
    const int64_t L = fdsc_lcm(C, fdsc->bin);
    if (L > 372181 || L * L > lim / C) return ORC_ERR_RANGE; /* C L^2 255^2 < 2^53 */
  }
  return ORC_OK;
}

/* element (b, c, t) */
static int64_t at(int64_t b, int64_t c, int64_t t, int64_t C, int64_t T, int layout) {
  return layout == ORC_LAYOUT_BCT ? (b * C + c) * T + t : (b * T + t) * C + c;
}

/* it0: index of the cuts' first iteration, which keys the random draws (the
 * interleaved order runs round r as single iterations with it0 = r) */
static int clean_u8_from(const uint8_t* in, uint8_t* out, uint8_t* flags, int64_t B, int64_t C, int64_t T,
                         int layout, const orc_cut* tdsc, const orc_cut* fdsc, int it0) {
  int rc = check_block(B, C, T, layout, tdsc, fdsc);
  if (rc) return rc;
  rc = range_u8(C, T, tdsc, fdsc);
  if (rc) return rc;
  const int64_t N = B * C * T;
  if (out != in) memmove(out, in, (size_t)N);
  if (flags) memset(flags, 0, (size_t)N);
  uint8_t* v = (uint8_t*)malloc((size_t)(C > T ? C : T));
  uint8_t* fl = (uint8_t*)malloc((size_t)(C > T ? C : T));
  if (tdsc && tdsc->enabled) {
    for (int64_t b = 0; b < B; b++)
      for (int64_t c = 0; c < C; c++) {
        for (int64_t t = 0; t < T; t++) {
          v[t] = out[at(b, c, t, C, T, layout)];
          fl[t] = 0;
        }
        orc_tdsc_row_u8x(v, fl, T, tdsc->k, tdsc->iterations, tdsc->replace, b, c, it0);
        for (int64_t t = 0; t < T; t++) {
          out[at(b, c, t, C, T, layout)] = v[t];
          if (flags) flags[at(b, c, t, C, T, layout)] |= fl[t];
        }
      }
  }
  if (fdsc && fdsc->enabled) {
    for (int64_t b = 0; b < B; b++)
      for (int64_t t = 0; t < T; t++) {
        for (int64_t c = 0; c < C; c++) {
          v[c] = out[at(b, c, t, C, T, layout)];
          fl[c] = 0;
        }
        orc_fdsc_col_u8x(v, fl, C, fdsc->k, fdsc->iterations, fdsc->replace, fdsc->bin, b, t, it0);
        for (int64_t c = 0; c < C; c++) {
          out[at(b, c, t, C, T, layout)] = v[c];
          if (flags) flags[at(b, c, t, C, T, layout)] |= fl[c];
        }
      }
  }
  free(v);
  free(fl);
  return ORC_OK;
}

int orc_clean_u8(const uint8_t* in, uint8_t* out, uint8_t* flags, int64_t B, int64_t C, int64_t T,
                 int layout, const orc_cut* tdsc, const orc_cut* fdsc) {
  return clean_u8_from(in, out, flags, B, C, T, layout, tdsc, fdsc, 0);
}

static int clean_f32_from(const float* in, float* out, uint8_t* flags, double* margin, int64_t B, int64_t C,
                          int64_t T, int layout, const orc_cut* tdsc, const orc_cut* fdsc, int it0);

int orc_clean_f32(const float* in, float* out, uint8_t* flags, int64_t B, int64_t C, int64_t T,
                  int layout, const orc_cut* tdsc, const orc_cut* fdsc) {
  return clean_f32_from(in, out, flags, NULL, B, C, T, layout, tdsc, fdsc, 0);
}

int orc_clean_f32m(const float* in, float* out, uint8_t* flags, double* margin, int64_t B, int64_t C, int64_t T,
                   int layout, const orc_cut* tdsc, const orc_cut* fdsc) {
  return clean_f32_from(in, out, flags, margin, B, C, T, layout, tdsc, fdsc, 0);
}

static int clean_f32_from(const float* in, float* out, uint8_t* flags, double* margin, int64_t B, int64_t C,
                          int64_t T, int layout, const orc_cut* tdsc, const orc_cut* fdsc, int it0) {
  int rc = check_block(B, C, T, layout, tdsc, fdsc);
  if (rc) return rc;
  const int64_t N = B * C * T;
  if (out != in) memmove(out, in, (size_t)N * sizeof(float));
  if (flags) memset(flags, 0, (size_t)N);
  if (margin)
    for (int64_t i = 0; i < N; i++) margin[i] = INFINITY;
  const int64_t M = C > T ? C : T;
  float* v = (float*)malloc((size_t)M * sizeof(float));
  uint8_t* fl = (uint8_t*)malloc((size_t)M);
  double* mg = margin ? (double*)malloc((size_t)M * sizeof(double)) : NULL;
  if (tdsc && tdsc->enabled) {
    for (int64_t b = 0; b < B; b++)
      for (int64_t c = 0; c < C; c++) {
        for (int64_t t = 0; t < T; t++) {
          v[t] = out[at(b, c, t, C, T, layout)];
          fl[t] = 0;
          if (mg) mg[t] = INFINITY;
        }
        orc_tdsc_row_f32x(v, fl, mg, T, tdsc->k, tdsc->iterations, tdsc->replace, b, c, it0);
        for (int64_t t = 0; t < T; t++) {
          out[at(b, c, t, C, T, layout)] = v[t];
          if (flags) flags[at(b, c, t, C, T, layout)] |= fl[t];
          if (mg && mg[t] < margin[at(b, c, t, C, T, layout)]) margin[at(b, c, t, C, T, layout)] = mg[t];
        }
      }
  }
  if (fdsc && fdsc->enabled) {
    for (int64_t b = 0; b < B; b++)
      for (int64_t t = 0; t < T; t++) {
        for (int64_t c = 0; c < C; c++) {
          v[c] = out[at(b, c, t, C, T, layout)];
          fl[c] = 0;
          if (mg) mg[c] = INFINITY;
        }
        orc_fdsc_col_f32x(v, fl, mg, C, fdsc->k, fdsc->iterations, fdsc->replace, fdsc->bin, b, t, it0);
        for (int64_t c = 0; c < C; c++) {
          out[at(b, c, t, C, T, layout)] = v[c];
          if (flags) flags[at(b, c, t, C, T, layout)] |= fl[c];
          if (mg && mg[c] < margin[at(b, c, t, C, T, layout)]) margin[at(b, c, t, C, T, layout)] = mg[c];
        }
      }
  }
  free(v);
  free(fl);
  free(mg);
  return ORC_OK;
}


/* ------------------------------------------------------------------ */
/* Interleaved order: round i runs TDSC iteration i on every row, then  */
/* FDSC iteration i on every column (each a single-iteration cut on the  */
/* current values, random draws keyed by iteration i); flags are OR-ed   */
/* over rounds.  With unequal iteration counts the method with more     */
/* iterations runs alone in the last rounds.  With one iteration of     */
/* each method this is the blocked order.                                */
/* ------------------------------------------------------------------ */
static int clean_interleaved(const void* in, void* out, uint8_t* flags, int64_t B, int64_t C, int64_t T,
                             int layout, const orc_cut* tdsc, const orc_cut* fdsc, int is_f32) {
  int rc = check_block(B, C, T, layout, tdsc, fdsc);
  if (rc) return rc;
  const int64_t N = B * C * T;
  const size_t es = is_f32 ? sizeof(float) : 1;
  if (out != in) memmove(out, in, (size_t)N * es);
  if (flags) memset(flags, 0, (size_t)N);
  uint8_t* fr = flags ? (uint8_t*)malloc((size_t)N) : NULL;
  const int it_t = (tdsc && tdsc->enabled) ? tdsc->iterations : 0;
  const int it_f = (fdsc && fdsc->enabled) ? fdsc->iterations : 0;
  const int rounds = it_t > it_f ? it_t : it_f;
  for (int r = 0; r < rounds && rc == ORC_OK; r++) {
    orc_cut t1 = {0, 0.0, 0, 0, 0}, f1 = {0, 0.0, 0, 0, 0};
    if (r < it_t) {
      t1 = *tdsc;
      t1.iterations = 1;
    }
    if (r < it_f) {
      f1 = *fdsc;
      f1.iterations = 1;
    }
    /* round r is iteration r of each method: its random draws are keyed by r */
    rc = is_f32 ? clean_f32_from((const float*)out, (float*)out, fr, NULL, B, C, T, layout, &t1, &f1, r)
                : clean_u8_from((const uint8_t*)out, (uint8_t*)out, fr, B, C, T, layout, &t1, &f1, r);
    if (flags)
      for (int64_t i = 0; i < N; i++) flags[i] |= fr[i];
  }
  free(fr);
  return rc;
}

int orc_clean_u8_interleaved(const uint8_t* in, uint8_t* out, uint8_t* flags, int64_t B, int64_t C, int64_t T,
                             int layout, const orc_cut* tdsc, const orc_cut* fdsc) {
  return clean_interleaved(in, out, flags, B, C, T, layout, tdsc, fdsc, 0);
}

int orc_clean_f32_interleaved(const float* in, float* out, uint8_t* flags, int64_t B, int64_t C, int64_t T,
                              int layout, const orc_cut* tdsc, const orc_cut* fdsc) {
  return clean_interleaved(in, out, flags, B, C, T, layout, tdsc, fdsc, 1);
}
