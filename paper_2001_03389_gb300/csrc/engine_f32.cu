// engine_f32.cu -- float32 TDSC and FDSC (Sec. IV of arXiv:2001.03389) on sm_103a.
//
// Same persistent work queue as the uint8 engine: TDSC items are whole rows
// (one CTA per (beam, channel) row, staged in shared memory), FDSC items are
// 32 time samples x all channels of a beam, processed in sub-slabs of ws
// samples held as a [channel][time] tile in shared memory.
//
// Precision.  The decision |x - mu| > k sigma must agree with an FP64
// evaluation except within ~1e-9 relative of the threshold, but an FP64 warp
// instruction costs ~20 SM cycles on this part.  So:
//  - sums and sums of squares are accumulated per thread in float-float
//    (TwoSum compensation, exact products by FMA) and merged in float-float;
//  - the finish (mean, variance, sqrt, k sigma) is float-float too (~2^-46
//    relative), computed by every thread of the row from the same merged sums,
//    so no thread waits for another to broadcast it;
//  - the variance is Q/n - mu^2 from those sums; when that cancels badly
//    (mu^2 > 1000 sigma^2) the row or column is redone with an FP64 two-pass;
//  - each sample is decided in FP32 against bounds widened by 2^-20 (and by
//    the rounding of the mean to float); a sample inside the band is decided
//    by the FP64 expression fabs((double)x - mu) > k * sigma.
#include <cuda_runtime.h>

#include "engine.h"

namespace rfim {

// ---------------------------------------------------------------------------
// float-float arithmetic (no contraction: explicit _rn intrinsics)
// ---------------------------------------------------------------------------
struct FF {
  float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

__device__ __forceinline__ void ff_acc(FF& a, float y) {
  float s, e;
  two_sum(a.hi, y, s, e);
  a.hi = s;
  a.lo = __fadd_rn(a.lo, e);
}

__device__ __forceinline__ void ff_acc_sq(FF& a, float y) {
  const float p = __fmul_rn(y, y);
  const float pe = __fmaf_rn(y, y, -p);  // y*y = p + pe exactly
  float s, e;
  two_sum(a.hi, p, s, e);
  a.hi = s;
  a.lo = __fadd_rn(a.lo, __fadd_rn(e, pe));
}

__device__ __forceinline__ FF ff_add(FF a, FF b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  FF r;
  r.hi = __fadd_rn(s, e);
  r.lo = __fsub_rn(e, __fsub_rn(r.hi, s));
  return r;
}

__device__ __forceinline__ FF ff_neg(FF a) { return FF{-a.hi, -a.lo}; }

// a * b for float-float a, b (error ~ u^2 relative)
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  FF r;
  r.hi = __fadd_rn(p, e);
  r.lo = __fsub_rn(e, __fsub_rn(r.hi, p));
  return r;
}

// a / g for a positive integer g
__device__ __forceinline__ FF ff_div_int(FF a, int g) {
  if ((g & (g - 1)) == 0) {  // power of two: exact scaling
    const float s = __frcp_rn((float)g);
    return FF{__fmul_rn(a.hi, s), __fmul_rn(a.lo, s)};
  }
  const float gf = (float)g;
  const float q1 = __fdiv_rn(a.hi, gf);
  const float p = __fmul_rn(q1, gf);
  const float pe = __fmaf_rn(q1, gf, -p);
  // remainder a - q1 * g: hi - p is exact (p is within one rounding of hi)
  const float rem = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), pe), a.lo);
  const float q2 = __fdiv_rn(rem, gf);
  FF r;
  r.hi = __fadd_rn(q1, q2);
  r.lo = __fsub_rn(q2, __fsub_rn(r.hi, q1));
  return r;
}

// a double as float-float (~2^-48 relative)
__device__ __forceinline__ FF ff_from_d(double v) {
  const float hi = __double2float_rn(v);
  return FF{hi, __double2float_rn(v - (double)hi)};
}

// sqrt of a float-float v >= 0 (0 otherwise): the float32 root refined by one
// Newton step, s = s0 + (v - s0^2) / (2 s0), with s0^2 formed exactly by FMA.
__device__ __forceinline__ FF ff_sqrt(FF v) {
  if (!(v.hi > 0.f)) return FF{0.f, 0.f};
  const float s0 = __fsqrt_rn(v.hi);
  const float p = __fmul_rn(s0, s0);
  const float pe = __fmaf_rn(s0, s0, -p);  // s0^2 = p + pe
  // v - s0^2: v.hi - p is exact (the two are within a rounding of each other)
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(v.hi, p), pe), v.lo);
  const float c = __fdiv_rn(r, __fmul_rn(2.f, s0));
  FF o;
  o.hi = __fadd_rn(s0, c);
  o.lo = __fsub_rn(c, __fsub_rn(o.hi, s0));
  return o;
}

__device__ __forceinline__ FF shfl_ff(FF a, int o) {
  return FF{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

__device__ __forceinline__ FF warp_ff(FF a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a = ff_add(a, shfl_ff(a, o));
  return a;
}

// sqrt(v) for v >= 0 to ~1e-14 relative: a float32 reciprocal square root
// refined by one Newton step in double (a double sqrt is ~30 slow FP64
// instructions on this part; one FMA-based step is four).
__device__ __forceinline__ double sqrt_fast(double v) {
  if (!(v > 0.0)) return 0.0;
  const float vf = (float)v;
  if (!(vf > 0.0f) || isinf(vf)) return sqrt(v);  // outside float range
  const double r = (double)rsqrtf(vf);  // ~2^-23 relative
  const double y = v * r;                // ~sqrt(v)
  return fma(0.5 * r, fma(-y, y, v), y);  // y + (v - y^2) / (2 sqrt v)
}

// ---------------------------------------------------------------------------
// Decisions
// ---------------------------------------------------------------------------
// One cut of one iteration of one row or (column, bin): samples y with
// |y - mu| > thr are flagged, mu and thr doubles.  mu_f = (float)mu; [lo_f, hi_f]
// is the band in which the float32 value |y - mu_f| cannot decide.  The
// doubles are read only inside the band: mu = mu_hi + mu_lo (exact), thr at *thr.
struct Cut32 {
  float mu_f, mu_lo, lo_f, hi_f;
  float thr_hi, thr_lo;  // thr as float-float
};

// thr and the rounding error dm = |mu - mu_f| (both >= 0) -> float32 bounds.
// |fl(y - mu_f)| = a satisfies |y - mu_f| in [a / (1 + u), a / (1 - u)], u = 2^-24,
// and | |y - mu| - |y - mu_f| | <= dm, so a > (thr + dm)(1 + 2^-20) proves a flag
// and a <= (thr - dm)(1 - 2^-20) proves a keep.  thr_lo <= thr <= thr_hi are
// float bounds of the double threshold.
__device__ __forceinline__ void band_bounds_f(float thr_lo, float thr_hi, float dm, float& lo_f, float& hi_f) {
  const float h = __fadd_ru(thr_hi, dm);
  hi_f = __fmul_ru(h, 1.0f + 0x1p-20f);
  const float l = __fsub_rd(thr_lo, dm);
  lo_f = __fmul_rd(l, 1.0f - 0x1p-20f);
}

// The double expression, kept out of line so that it runs only inside the band.
__device__ __noinline__ bool flag64(float y, float mu_hi, float mu_lo, float thr_hi, float thr_lo) {
  const double mu = (double)mu_hi + (double)mu_lo;
  return fabs((double)y - mu) > (double)thr_hi + (double)thr_lo;
}

__device__ __forceinline__ bool flag32(float y, const Cut32& c) {
  const float a = fabsf(__fsub_rn(y, c.mu_f));
  if (a > c.hi_f) return true;
  if (!(a > c.lo_f)) return false;
  return flag64(y, c.mu_f, c.mu_lo, c.thr_hi, c.thr_lo);
}

// flag32 on four samples at once, bit i for sample i: the float32 tests of all
// four first, and one branch to the FP64 expression when any lies in its band.
__device__ __forceinline__ unsigned flag32x4(const float4& v, const Cut32& c0, const Cut32& c1, const Cut32& c2,
                                             const Cut32& c3) {
  const float a0 = fabsf(__fsub_rn(v.x, c0.mu_f)), a1 = fabsf(__fsub_rn(v.y, c1.mu_f));
  const float a2 = fabsf(__fsub_rn(v.z, c2.mu_f)), a3 = fabsf(__fsub_rn(v.w, c3.mu_f));
  unsigned f = (a0 > c0.hi_f ? 1u : 0u) | (a1 > c1.hi_f ? 2u : 0u) | (a2 > c2.hi_f ? 4u : 0u) | (a3 > c3.hi_f ? 8u : 0u);
  const unsigned band =
      ((a0 > c0.lo_f ? 1u : 0u) | (a1 > c1.lo_f ? 2u : 0u) | (a2 > c2.lo_f ? 4u : 0u) | (a3 > c3.lo_f ? 8u : 0u)) & ~f;
  if (band) {
    if ((band & 1u) && flag64(v.x, c0.mu_f, c0.mu_lo, c0.thr_hi, c0.thr_lo)) f |= 1u;
    if ((band & 2u) && flag64(v.y, c1.mu_f, c1.mu_lo, c1.thr_hi, c1.thr_lo)) f |= 2u;
    if ((band & 4u) && flag64(v.z, c2.mu_f, c2.mu_lo, c2.thr_hi, c2.thr_lo)) f |= 4u;
    if ((band & 8u) && flag64(v.w, c3.mu_f, c3.mu_lo, c3.thr_hi, c3.thr_lo)) f |= 8u;
  }
  return f;
}

// The cut of mean mu and threshold thr (float-float, mu normalised so that
// |mu - mu.hi| = |mu.lo|).
__device__ __forceinline__ Cut32 make_cut32(FF mu, FF thr) {
  Cut32 c;
  c.mu_f = mu.hi;
  c.mu_lo = mu.lo;
  c.thr_hi = thr.hi;
  c.thr_lo = thr.lo;
  band_bounds_f(__fadd_rd(thr.hi, thr.lo), __fadd_ru(thr.hi, thr.lo), fabsf(mu.lo), c.lo_f, c.hi_f);
  return c;
}

// One TDSC iteration of a row as FDSC items replay it: the cut and the value
// that replaces the samples it flags.
__device__ __forceinline__ void store_prog(float* e, const Cut32& c, float r) {
  reinterpret_cast<float4*>(e)[0] = make_float4(c.mu_f, c.lo_f, c.hi_f, r);
  reinterpret_cast<float4*>(e)[1] = make_float4(c.mu_lo, c.thr_hi, c.thr_lo, 0.f);
}

// The value TDSC left in a sample of the input value y that one of its
// iterations flagged: the row's iterations replayed in order, y <- r_i where
// cut i flags y.  f: the first records' fast fields, loaded ahead.
__device__ __forceinline__ float replay_tdsc(float y, const float4* pe, const float4 (&f)[3], int I) {
#pragma unroll
  for (int i = 0; i < 3; i++) {
    if (i < I) {
      const float a = fabsf(__fsub_rn(y, f[i].x));
      bool fl = a > f[i].z;
      if (!fl && a > f[i].y) {
        const float4 sl = __ldcg(pe + 2 * i + 1);
        fl = flag64(y, f[i].x, sl.x, sl.y, sl.z);
      }
      if (fl) y = f[i].w;
    }
  }
  for (int i = 3; i < I; i++) {
    const float4 q = __ldcg(pe + 2 * i);
    const float a = fabsf(__fsub_rn(y, q.x));
    bool fl = a > q.z;
    if (!fl && a > q.y) {
      const float4 sl = __ldcg(pe + 2 * i + 1);
      fl = flag64(y, q.x, sl.x, sl.y, sl.z);
    }
    if (fl) y = q.w;
  }
  return y;
}

// Total order of floats as unsigned keys (-0 before +0).
__device__ __forceinline__ unsigned fkey(float f) {
  const unsigned b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_f(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// ---------------------------------------------------------------------------
// CTA reductions (NT threads)
// ---------------------------------------------------------------------------
struct Red32 {
  float f[2 * (NT / 32) * 2];
  double d[2 * (NT / 32)];
  int i[NT / 32];
  int flag;
};

// ---------------------------------------------------------------------------
// Thread groups of GN threads (a half CTA, or the whole CTA) that clean one
// row each; h = group index, synchronised by named barrier 1 + h.
// ---------------------------------------------------------------------------
template <int GN>
__device__ __forceinline__ void gsync(int h) {
  asm volatile("bar.sync %0, %1;" ::"r"(h + 1), "r"(GN) : "memory");
}

template <int GN>
__device__ __forceinline__ void grp_ff2(FF& a, FF& b, Red32* r, int t, int h) {
  const int lane = t & 31, warp = t >> 5;
  a = warp_ff(a);
  b = warp_ff(b);
  gsync<GN>(h);
  if (lane == 0) {
    r->f[4 * warp + 0] = a.hi;
    r->f[4 * warp + 1] = a.lo;
    r->f[4 * warp + 2] = b.hi;
    r->f[4 * warp + 3] = b.lo;
  }
  gsync<GN>(h);
  FF sa{0.f, 0.f}, sb{0.f, 0.f};
#pragma unroll
  for (int w = 0; w < GN / 32; w++) {
    sa = ff_add(sa, FF{r->f[4 * w + 0], r->f[4 * w + 1]});
    sb = ff_add(sb, FF{r->f[4 * w + 2], r->f[4 * w + 3]});
  }
  a = sa;
  b = sb;
}

template <int GN>
__device__ __forceinline__ double grp_dsum(double v, Red32* r, int t, int h) {
  const int lane = t & 31, warp = t >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  gsync<GN>(h);
  if (lane == 0) r->d[warp] = v;
  gsync<GN>(h);
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < GN / 32; w++) s += r->d[w];
  return s;
}

template <int GN>
__device__ __forceinline__ int grp_isum(int v, Red32* r, int t, int h) {
  const int lane = t & 31, warp = t >> 5;
  v = __reduce_add_sync(0xffffffffu, v);
  gsync<GN>(h);
  if (lane == 0) r->i[warp] = v;
  gsync<GN>(h);
  int s = 0;
#pragma unroll
  for (int w = 0; w < GN / 32; w++) s += r->i[w];
  return s;
}

__device__ __forceinline__ float f4_get(const float4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}
__device__ __forceinline__ void f4_set(float4& v, int i, float x) {
  if (i == 0) v.x = x;
  else if (i == 1) v.y = x;
  else if (i == 2) v.z = x;
  else v.w = x;
}

// Lower median (rank floor((n-1)/2)) of the valid elements of the staged row:
// bitwise search over the order keys, one bit per CTA-wide count.
template <int GN>
__device__ float row_median_f32(const float4* st, int nch, int head, int tail, int n, Red32* red, int t, int h) {
  const int rank = (n - 1) >> 1;
  unsigned prefix = 0;
  for (int b = 31; b >= 0; b--) {
    const unsigned test = prefix | (1u << b);
    int cnt = 0;
    for (int k = t; k < nch; k += GN) {
      const float4 v = st[k];
      const int lo = k == 0 ? head : 0, hi = k == nch - 1 ? tail : 4;
#pragma unroll
      for (int i = 0; i < 4; i++)
        if (i >= lo && i < hi) cnt += fkey(f4_get(v, i)) < test;
    }
    cnt = grp_isum<GN>(cnt, red, t, h);
    if (cnt <= rank) prefix = test;
  }
  return key_f(prefix);
}

// GN threads clean the row: t = thread in the group, h = group (its barrier is 1 + h)
// mbar: the group's staging mbarrier; bit `pb` of mpar is the parity of its next
// phase (tracked by every thread of the group).
template <int GN, bool RND>
__device__ void tdsc_row_f32(const Params& P, const Job& J, int row, unsigned char* smem, Red32* red, int t, int h,
                             unsigned long long* mbar, unsigned& mpar, int pb) {
  const CutDev& cut = P.td;
  const int T = J.T;
  const float* beam_in = static_cast<const float*>(J.in);
  const float* rin = beam_in + (size_t)row * T;
  float* rout = static_cast<float*>(J.out) + (size_t)row * T;
  const float* blo = static_cast<const float*>(J.src_lo);
  const float* bhi = static_cast<const float*>(J.src_hi);

  const int head = (int)(((uintptr_t)rin & 15) >> 2);
  const float* cb = rin - head;
  const int nch = (head + T + 3) >> 2;
  const int tail = head + T - 4 * (nch - 1);  // valid elements of the last chunk (1..4)

  float4* st = reinterpret_cast<float4*>(smem);
  unsigned char* fl4 = smem + 16 * nch;
  float* lst = reinterpret_cast<float*>(smem + 16 * nch + align16i(nch));
  __shared__ int s_cnt_g[2][2];  // per group: replaced-value counts of alternate iterations
  int* s_cnt = s_cnt_g[h];
  if (t == 0) {  // (published by the staging barrier)
    s_cnt[0] = 0;
    s_cnt[1] = 0;
  }

  // ---- stage the row: the interior chunks (inside the row) are one TMA bulk
  //      copy issued by the group's first thread, completing on the group's
  //      mbarrier; the edge chunks take guarded loads, padding zeroed
  const bool bulk = nch > 2;  // (the same in every thread of the group)
  if (bulk && t == 0) {
    fence_proxy_async_smem();  // earlier generic accesses of the stage come first
    mbar_arrive_expect_tx(mbar, 16u * (unsigned)(nch - 2));
    bulk_copy_g2s(st + 1, cb + 4, 16u * (unsigned)(nch - 2), mbar);
  }
  for (int k = t; k < nch; k += GN) {
    if (k == 0 || k == nch - 1) {
      const float* a = cb + 4 * k;
      const int lo = k == 0 ? head : 0, hi = k == nch - 1 ? tail : 4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int i = 0; i < 4; i++)
        if (i >= lo && i < hi && a + i >= blo && a + i < bhi) f4_set(v, i, a[i]);
      st[k] = v;
    }
    fl4[k] = 0;
  }
  if (bulk) {
    if (!mbar_wait_bounded(mbar, (mpar >> pb) & 1u, P.spin_limit_ns)) atomicExch(P.status, 5u);
    mpar ^= 1u << pb;
  }
  gsync<GN>(h);

  // ---- sums of the staged row (padding zeros add nothing)
  FF S{0.f, 0.f}, Q{0.f, 0.f};
  for (int k = t; k < nch; k += GN) {
    const float4 v = st[k];
    ff_acc(S, v.x);
    ff_acc_sq(Q, v.x);
    ff_acc(S, v.y);
    ff_acc_sq(Q, v.y);
    ff_acc(S, v.z);
    ff_acc_sq(Q, v.z);
    ff_acc(S, v.w);
    ff_acc_sq(Q, v.w);
  }
  grp_ff2<GN>(S, Q, red, t, h);
  // S, Q: running sums of the current values, the same in every thread of the
  // group (the merges above add in the same order everywhere)
  if (J.stats && t == 0) {  // statistics of the input row, for the caller's records
    J.stats[2 * (size_t)row] = (double)S.hi + (double)S.lo;
    J.stats[2 * (size_t)row + 1] = (double)Q.hi + (double)Q.lo;
  }
  const FF kff{cut.k_hi, cut.k_lo};
  const int I = cut.iterations;
  const bool rnd = RND && cut.replace == REP_RANDOM;  // (RND: the kernel build that holds random replacement)

  for (int it = 0; it < I; it++) {
    // statistics of the current values, finished in float-float by every thread
    FF mu = ff_div_int(S, T);
    const FF mq = ff_div_int(Q, T);
    FF var = ff_add(mq, ff_neg(ff_mul(mu, mu)));
    if (!(var.hi >= 1e-3f * mq.hi)) {  // (the same in every thread)
      // cancellation (or a constant row): FP64 two-pass over the current values
      double sd = 0.0;
      for (int k = t; k < nch; k += GN) {
        const float4 v = st[k];
        sd += ((double)v.x + (double)v.y) + ((double)v.z + (double)v.w);  // padding is 0
      }
      sd = grp_dsum<GN>(sd, red, t, h);
      const double rT = 1.0 / (double)T;  // (only on this rare path)
      const double m2 = sd * rT;
      double ss = 0.0;
      for (int k = t; k < nch; k += GN) {
        const float4 v = st[k];
        const int lo = k == 0 ? head : 0, hi = k == nch - 1 ? tail : 4;
#pragma unroll
        for (int i = 0; i < 4; i++)
          if (i >= lo && i < hi) {
            const double d = (double)f4_get(v, i) - m2;
            ss += d * d;
          }
      }
      ss = grp_dsum<GN>(ss, red, t, h);
      mu = ff_from_d(m2);
      var = ff_from_d(ss * rT);
      S = ff_from_d(sd);  // the two-pass sum carries on
    }
    const Cut32 c = make_cut32(mu, ff_mul(kff, ff_sqrt(var)));
    const float r = cut.replace == REP_MEDIAN ? row_median_f32<GN>(st, nch, head, tail, T, red, t, h) : c.mu_f;
    if (J.prog && t == 0) store_prog(J.prog + ((size_t)row * I + it) * PROG_FLOATS, c, r);

    // decide and replace; the replaced values go to a list for the statistics
    // update (its length counter was zeroed before the last barrier)
    int& s_nlist = s_cnt[it & 1];
    if (rnd) {
      // random replacement: this iteration's flags first (high nibble of fl4),
      // then each flagged sample copies the first drawn sample that is unflagged
      // (those are never written in this iteration)
      for (int k = t; k < nch; k += GN) {
        const float4 v = st[k];
        const int lo = k == 0 ? head : 0, hi = k == nch - 1 ? tail : 4;
        const unsigned nib = flag32x4(v, c, c, c, c) & (0xFu << lo) & (0xFu >> (4 - hi));
        fl4[k] = (unsigned char)((fl4[k] & 0xFu) | nib | (nib << 4));
      }
      gsync<GN>(h);
      const float* sf = reinterpret_cast<const float*>(st) + head;  // sample tt at sf[tt]
      const unsigned long long key = draw_key(J.beam, row);
      for (int k = t; k < nch; k += GN) {
        const unsigned nib = fl4[k] >> 4;
        if (!nib) continue;
        float4 v = st[k];
#pragma unroll
        for (int i = 0; i < 4; i++) {
          if (!((nib >> i) & 1u)) continue;
          const int tt = 4 * k + i - head;
          for (int a = 0; a < DRAW_ATTEMPTS; a++) {
            const unsigned u = draw_pos(key, tt, 1, cut.it0 + it, a, (unsigned)T);
            const unsigned pu = (unsigned)head + u;
            if (!((fl4[pu >> 2] >> (4 + (pu & 3))) & 1u)) {
              f4_set(v, i, sf[u]);
              break;
            }
          }
        }
        st[k] = v;
      }
    } else
    for (int k = t; k < nch; k += GN) {
      float4 v = st[k];
      const int lo = k == 0 ? head : 0, hi = k == nch - 1 ? tail : 4;
      const unsigned nib = flag32x4(v, c, c, c, c) & (0xFu << lo) & (0xFu >> (4 - hi));
      if (nib) {
#pragma unroll
        for (int i = 0; i < 4; i++) {
          if (!((nib >> i) & 1u)) continue;
          const int pos = atomicAdd(&s_nlist, 1);
          if (pos < TD32_LIST) lst[pos] = f4_get(v, i);
          f4_set(v, i, r);
        }
        st[k] = v;
        fl4[k] |= (unsigned char)nib;
      }
    }
    if (it == I - 1) break;
    if (t == 0) s_cnt[(it + 1) & 1] = 0;  // the next iteration's counter (last read before the previous merge)
    gsync<GN>(h);
    // statistics of the next iteration: S' = S - sum(replaced) + nf r (same for Q)
    const int nflag = rnd ? TD32_LIST + 1 : s_nlist;  // random: the replaced-with values vary, sum the row again
    FF rs{0.f, 0.f}, rq{0.f, 0.f};
    if (nflag <= TD32_LIST) {
      for (int i = t; i < nflag; i += GN) {
        ff_acc(rs, lst[i]);
        ff_acc_sq(rq, lst[i]);
      }
      grp_ff2<GN>(rs, rq, red, t, h);
      const float nf = (float)nflag;  // exact (nflag < 2^24)
      const float pr = __fmul_rn(nf, r);
      const float r2 = __fmul_rn(r, r);
      S = ff_add(ff_add(S, ff_neg(rs)), FF{pr, __fmaf_rn(nf, r, -pr)});
      Q = ff_add(ff_add(Q, ff_neg(rq)), ff_mul(FF{r2, __fmaf_rn(r, r, -r2)}, FF{nf, 0.f}));
    } else {
      // many replacements: sum the current row again
      for (int k = t; k < nch; k += GN) {
        const float4 v = st[k];
        ff_acc(rs, v.x);
        ff_acc_sq(rq, v.x);
        ff_acc(rs, v.y);
        ff_acc_sq(rq, v.y);
        ff_acc(rs, v.z);
        ff_acc_sq(rq, v.z);
        ff_acc(rs, v.w);
        ff_acc_sq(rq, v.w);
      }
      grp_ff2<GN>(rs, rq, red, t, h);
      S = rs;
      Q = rq;
    }
  }
  gsync<GN>(h);

  // ---- write the row (unless FDSC replays the recorded cuts) and its mask
  const bool same_align = (((uintptr_t)rout) & 15) == (((uintptr_t)rin) & 15);
  float* ob = rout - head;
  for (int k = t; k < (J.prog ? 0 : nch); k += GN) {
    const float4 v = st[k];
    const int lo = k == 0 ? head : 0, hi = k == nch - 1 ? tail : 4;
    if (same_align && lo == 0 && hi == 4) {
      *reinterpret_cast<float4*>(ob + 4 * k) = v;
    } else {
#pragma unroll
      for (int i = 0; i < 4; i++)
        if (i >= lo && i < hi) ob[4 * k + i] = f4_get(v, i);
    }
  }
  if (P.mask_kind == MASK_BITS && J.mask) {
    const int W32 = (T + 31) >> 5;
    unsigned* mrow = static_cast<unsigned*>(J.mask) + (size_t)row * W32;
    // word w covers chunk-grid positions head + 32 w ... head + 32 w + 31: chunks 8w .. 8w + 8
    for (int w = t; w < W32; w += GN) {
      unsigned long long bits = 0;
#pragma unroll
      for (int j = 0; j < 9; j++) {
        const int k = 8 * w + j;
        if (k < nch) bits |= (unsigned long long)(fl4[k] & 0xF) << (4 * j);
      }
      unsigned word = (unsigned)(bits >> head);
      const int valid = T - 32 * w;
      if (valid < 32) word &= (1u << valid) - 1u;
      mrow[w] = P.td_mask_or ? (mrow[w] | word) : word;
    }
  } else if (P.mask_kind == MASK_BYTES && J.mask) {
    unsigned char* mb = static_cast<unsigned char*>(J.mask) + (size_t)row * T;
    for (int tt = t; tt < T; tt += GN) {
      const int p = head + tt;
      const unsigned char f = (unsigned char)((fl4[p >> 2] >> (p & 3)) & 1u);
      mb[tt] = P.td_mask_or ? (unsigned char)(mb[tt] | f) : f;
    }
  }
  gsync<GN>(h);
}

// ---------------------------------------------------------------------------
// TDSC on one float32 row longer than the shared-memory stage (the whole CTA).
// Nothing is staged: every pass reads the row from memory and replays the
// decisions of the earlier iterations on the fly, y <- r_j where iteration j's
// cut flags y.  The same statistics, finish and decisions as tdsc_row_f32; the
// median is the same radix select, one pass per key bit.  Out of line, as such
// rows are rare.
// ---------------------------------------------------------------------------
__device__ __noinline__ void tdsc_row_f32_long(const Params& P, const Job& J, int row, Red32* red) {
  const CutDev& cut = P.td;
  const int T = J.T, t = threadIdx.x, lane = t & 31;
  const float* rin = static_cast<const float*>(J.in) + (size_t)row * T;
  float* rout = static_cast<float*>(J.out) + (size_t)row * T;
  const int I = cut.iterations;
  const FF kff{cut.k_hi, cut.k_lo};
  __shared__ Cut32 s_cut[16];
  __shared__ float s_rep[16];
  // value of sample i after iterations 0..n-1 (fl: flagged by any of them)
  auto cur = [&](int i, int n, bool& fl) -> float {
    float y = rin[i];
    for (int j = 0; j < n; j++)
      if (flag32(y, s_cut[j])) {
        y = s_rep[j];
        fl = true;
      }
    return y;
  };
  for (int it = 0; it < I; it++) {
    FF S{0.f, 0.f}, Q{0.f, 0.f};
    for (int i = t; i < T; i += NT) {
      bool fl = false;
      const float y = cur(i, it, fl);
      ff_acc(S, y);
      ff_acc_sq(Q, y);
    }
    grp_ff2<NT>(S, Q, red, t, 0);  // (the same in every thread)
    if (it == 0 && J.stats && t == 0) {  // statistics of the input row, for the caller's records
      J.stats[2 * (size_t)row] = (double)S.hi + (double)S.lo;
      J.stats[2 * (size_t)row + 1] = (double)Q.hi + (double)Q.lo;
    }
    FF mu = ff_div_int(S, T);
    const FF mq = ff_div_int(Q, T);
    FF var = ff_add(mq, ff_neg(ff_mul(mu, mu)));
    if (!(var.hi >= 1e-3f * mq.hi)) {
      // cancellation (or a constant row): FP64 two-pass
      double sd = 0.0;
      for (int i = t; i < T; i += NT) {
        bool fl = false;
        sd += (double)cur(i, it, fl);
      }
      sd = grp_dsum<NT>(sd, red, t, 0);
      const double rT = 1.0 / (double)T;  // (only on this rare path)
      const double m2 = sd * rT;
      double ss = 0.0;
      for (int i = t; i < T; i += NT) {
        bool fl = false;
        const double d = (double)cur(i, it, fl) - m2;
        ss += d * d;
      }
      ss = grp_dsum<NT>(ss, red, t, 0);
      mu = ff_from_d(m2);
      var = ff_from_d(ss * rT);
    }
    const Cut32 c = make_cut32(mu, ff_mul(kff, ff_sqrt(var)));
    float r = c.mu_f;
    if (cut.replace == REP_MEDIAN) {
      const int rank = (T - 1) >> 1;
      unsigned prefix = 0;
      for (int b = 31; b >= 0; b--) {
        const unsigned test = prefix | (1u << b);
        int cnt = 0;
        for (int i = t; i < T; i += NT) {
          bool fl = false;
          cnt += fkey(cur(i, it, fl)) < test;
        }
        cnt = grp_isum<NT>(cnt, red, t, 0);
        if (cnt <= rank) prefix = test;
      }
      r = key_f(prefix);
    }
    if (t == 0) {
      s_cut[it] = c;
      s_rep[it] = r;
      if (J.prog) store_prog(J.prog + ((size_t)row * I + it) * PROG_FLOATS, c, r);
    }
    gsync<NT>(0);
  }
  // ---- output and mask: a warp per 32-sample mask word
  const int W32 = (T + 31) >> 5;
  unsigned* mrow = (P.mask_kind == MASK_BITS && J.mask) ? static_cast<unsigned*>(J.mask) + (size_t)row * W32 : nullptr;
  unsigned char* mb =
      (P.mask_kind == MASK_BYTES && J.mask) ? static_cast<unsigned char*>(J.mask) + (size_t)row * T : nullptr;
  for (int w = t >> 5; w < W32; w += NT / 32) {
    const int i = 32 * w + lane;
    bool fl = false;
    if (i < T) {
      const float y = cur(i, I, fl);  // (read before the write: out may be in)
      if (!J.prog) rout[i] = y;
      if (mb) mb[i] = P.td_mask_or ? (unsigned char)(mb[i] | (fl ? 1u : 0u)) : (unsigned char)(fl ? 1u : 0u);
    }
    const unsigned bits = __ballot_sync(0xffffffffu, fl);
    if (mrow && lane == 0) mrow[w] = P.td_mask_or ? (mrow[w] | bits) : bits;
  }
  gsync<NT>(0);
}

// ---------------------------------------------------------------------------
// TDSC with random replacement on one float32 row longer than the stage (the
// whole CTA).  A draw's outcome is not a function of the value, so the row
// cannot be replayed as in tdsc_row_f32_long: iteration 0 reads the input row
// and writes every sample of the output row, later iterations read the output
// row and rewrite its flagged samples.  The flags are bitmaps over the sample
// index in shared memory (fcur: this iteration's, facc: the OR over the
// iterations), so a draw tests the flag of the very sample it would copy and an
// iteration writes only samples that no draw of it may read.  Statistics,
// finish and decisions as in tdsc_row_f32 (the row summed again every
// iteration, as its random path does).  A warp takes one 32-sample word at a
// time, lane i sample 32 w + i.
// ---------------------------------------------------------------------------
__device__ __noinline__ void tdsc_row_f32_long_rnd(const Params& P, const Job& J, int row, unsigned* bm, Red32* red) {
  const CutDev& cut = P.td;
  const int T = J.T, t = threadIdx.x, lane = t & 31;
  const float* rin = static_cast<const float*>(J.in) + (size_t)row * T;
  float* rout = static_cast<float*>(J.out) + (size_t)row * T;
  const int I = cut.iterations, NW = (T + 31) >> 5;
  const FF kff{cut.k_hi, cut.k_lo};
  unsigned* fcur = bm;
  unsigned* facc = bm + NW;
  for (int w = t; w < NW; w += NT) facc[w] = 0;
  const unsigned long long key = draw_key(J.beam, row);
  for (int it = 0; it < I; it++) {
    const float* src = it == 0 ? rin : rout;  // the current values
    FF S{0.f, 0.f}, Q{0.f, 0.f};
    for (int i = t; i < T; i += NT) {
      const float y = src[i];
      ff_acc(S, y);
      ff_acc_sq(Q, y);
    }
    grp_ff2<NT>(S, Q, red, t, 0);  // (the same in every thread)
    if (it == 0 && J.stats && t == 0) {  // statistics of the input row, for the caller's records
      J.stats[2 * (size_t)row] = (double)S.hi + (double)S.lo;
      J.stats[2 * (size_t)row + 1] = (double)Q.hi + (double)Q.lo;
    }
    FF mu = ff_div_int(S, T);
    const FF mq = ff_div_int(Q, T);
    FF var = ff_add(mq, ff_neg(ff_mul(mu, mu)));
    if (!(var.hi >= 1e-3f * mq.hi)) {
      // cancellation (or a constant row): FP64 two-pass
      double sd = 0.0;
      for (int i = t; i < T; i += NT) sd += (double)src[i];
      sd = grp_dsum<NT>(sd, red, t, 0);
      const double rT = 1.0 / (double)T;  // (only on this rare path)
      const double m2 = sd * rT;
      double ss = 0.0;
      for (int i = t; i < T; i += NT) {
        const double d = (double)src[i] - m2;
        ss += d * d;
      }
      ss = grp_dsum<NT>(ss, red, t, 0);
      mu = ff_from_d(m2);
      var = ff_from_d(ss * rT);
    }
    const Cut32 c = make_cut32(mu, ff_mul(kff, ff_sqrt(var)));
    for (int w = t >> 5; w < NW; w += NT / 32) {
      const int i = 32 * w + lane;
      const bool f = i < T && flag32(src[i], c);
      const unsigned bits = __ballot_sync(0xffffffffu, f);
      if (lane == 0) fcur[w] = bits;
    }
    gsync<NT>(0);
    for (int w = t >> 5; w < NW; w += NT / 32) {
      const int i = 32 * w + lane;
      const unsigned fw = fcur[w];
      if (i < T) {
        if ((fw >> lane) & 1u) {
          float y = src[i];
          for (int a = 0; a < DRAW_ATTEMPTS; a++) {
            const unsigned u = draw_pos(key, i, 1, cut.it0 + it, a, (unsigned)T);
            if (!((fcur[u >> 5] >> (u & 31)) & 1u)) {
              y = src[u];
              break;
            }
          }
          rout[i] = y;
        } else if (it == 0 && rout != rin) {
          rout[i] = rin[i];
        }
      }
      if (lane == 0) facc[w] |= fw;
    }
    gsync<NT>(0);  // (also publishes this iteration's writes of the output row)
  }
  // the mask: facc holds the row's bits word for word
  if (P.mask_kind == MASK_BITS && J.mask) {
    unsigned* mrow = static_cast<unsigned*>(J.mask) + (size_t)row * NW;
    for (int w = t; w < NW; w += NT) mrow[w] = P.td_mask_or ? (mrow[w] | facc[w]) : facc[w];
  } else if (P.mask_kind == MASK_BYTES && J.mask) {
    unsigned char* mb = static_cast<unsigned char*>(J.mask) + (size_t)row * T;
    for (int i = t; i < T; i += NT) {
      const unsigned char f = (unsigned char)((facc[i >> 5] >> (i & 31)) & 1u);
      mb[i] = P.td_mask_or ? (unsigned char)(mb[i] | f) : f;
    }
  }
  gsync<NT>(0);
}

// ---------------------------------------------------------------------------
// FDSC on one item: one sub-slab of ws time samples x C channels of a float32
// beam (16 bytes of each channel row for ws = 4).  Consecutive items, which
// share the 128-byte lines of the rows, run at the same time, so the lines in
// flight stay few and are read from DRAM once.
// ---------------------------------------------------------------------------
// Tile [c][t] (pitch ws floats).  Work units are (t, bin) pairs, one thread
// each, t fastest; a unit walks its bin starting at a rotation of (bin mod 32)
// channels so that the lanes of a warp hit distinct banks.
struct Fd32Layout {
  float* tile;    // C x ws
  unsigned* fm;   // C: FDSC flag bits of the item (bit = t - t_item)
  unsigned* tm;   // C: the TDSC mask word of the sub-slab (replay of TDSC's cut records)
  float2* um;     // units: bin mean as float-float
  float2* uv;     // units: sum of squared deviations as float-float
  float* uq;      // units: sum of squares (cancellation check)
  float2* thr;    // ws: column thresholds k * sigma' (float-float)
  float* thr_lo;  // ws
  float* thr_hi;  // ws
  unsigned* fcur; // C (random replacement only): flags of the iteration in progress (bit = t - t0)
};

__device__ __forceinline__ Fd32Layout fd32_layout(unsigned char* smem, int ws, int C, int nb, bool rnd) {
  const int U = ws * nb;
  Fd32Layout L;
  unsigned char* p = smem;
  L.tile = reinterpret_cast<float*>(p);
  p += align16i(ws * C * 4);
  L.fm = reinterpret_cast<unsigned*>(p);
  p += align16i(C * 4);
  L.um = reinterpret_cast<float2*>(p);
  p += align16i(U * 8);
  L.uv = reinterpret_cast<float2*>(p);
  p += align16i(U * 8);
  L.uq = reinterpret_cast<float*>(p);
  p += align16i(U * 4);
  L.thr = reinterpret_cast<float2*>(p);
  p += align16i(ws * 8);
  L.thr_lo = reinterpret_cast<float*>(p);
  p += align16i(ws * 4);
  L.thr_hi = reinterpret_cast<float*>(p);
  p += align16i(ws * 4);
  L.fcur = reinterpret_cast<unsigned*>(p);
  p += rnd ? align16i(C * 4) : 0;
  L.tm = reinterpret_cast<unsigned*>(p);
  return L;
}

// Lower median of the n values tile[(c0 + j) * ws + t], j < n (one thread).
__device__ float bin_median_f32(const float* tile, int c0, int n, int ws, int t) {
  const int rank = (n - 1) >> 1;
  unsigned prefix = 0;
  for (int b = 31; b >= 0; b--) {
    const unsigned test = prefix | (1u << b);
    int cnt = 0;
    for (int j = 0; j < n; j++) cnt += fkey(tile[(c0 + j) * ws + t]) < test;
    if (cnt <= rank) prefix = test;
  }
  return key_f(prefix);
}

// ---------------------------------------------------------------------------
// FDSC on float32 columns wider than the tile: the CTA cleans the item's time
// samples one column at a time.  The column is gathered into shared memory
// (read through L2), cleaned there and scattered back; the flags are bits per
// channel.  The column statistics are taken in FP64 (bin means, deviations
// from them, their mean and spread), the decisions |d - mu| > k sigma' in FP64
// as well.  A warp takes a bin for the means and the medians, 32 channels for
// the flags and replacements.  Out of line: such beams are rare.
// ---------------------------------------------------------------------------
template <bool RND>
__device__ __noinline__ void fdsc_wide_f32(const Params& P, const Job& J, int item, unsigned char* smem, Red32* red) {
  const CutDev& cut = P.fd;
  const int C = J.C, T = J.T, G = cut.bin, NB = J.nb;
  const int W = (C + 31) >> 5, W32 = (T + 31) >> 5, t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int t_item = item * FD_ITEM_T, t_end = min(t_item + FD_ITEM_T, T);
  const float* src = static_cast<const float*>(P.fd_reads_out ? J.out : J.in);
  float* dst = static_cast<float*>(J.out);
  unsigned char* p = smem;
  float* x = reinterpret_cast<float*>(p);  // the column
  p += align16i(C * 4);
  unsigned* fcur = reinterpret_cast<unsigned*>(p);  // flags of this iteration, bit c % 32 of word c / 32
  p += align16i(W * 4);
  unsigned* facc = reinterpret_cast<unsigned*>(p);  // flags of every iteration so far
  p += align16i(W * 4);
  double* mb = reinterpret_cast<double*>(p);  // per bin: mean
  p += align16i(NB * 8);
  float* rep = reinterpret_cast<float*>(p);  // replacement value
  const bool rnd = RND && cut.replace == REP_RANDOM;
  const double rC = 1.0 / (double)C;
  // this item's mask words start from zero unless they hold the beam's TDSC flags
  if (J.mask && P.mask_kind == MASK_BITS && !P.mask_or)
    for (int c = t; c < C; c += NT) static_cast<unsigned*>(J.mask)[(size_t)c * W32 + item] = 0u;
  for (int tc = t_item; tc < t_end; tc++) {
    for (int c = t; c < C; c += NT) x[c] = src[(size_t)c * T + tc];
    for (int w = t; w < W; w += NT) facc[w] = 0u;
    __syncthreads();
    const unsigned long long key = draw_key(J.beam, tc);
    for (int it = 0; it < cut.iterations; it++) {
      for (int g = warp; g < NB; g += NT / 32) {
        const int c0 = g * G, c1 = min(c0 + G, C);
        double s = 0.0;
        for (int c = c0 + lane; c < c1; c += 32) s += (double)x[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
          mb[g] = s / (double)(c1 - c0);
          rep[g] = (float)mb[g];  // (the mean; medians below)
        }
      }
      __syncthreads();
      double sd = 0.0;
      for (int c = t; c < C; c += NT) sd += (double)x[c] - mb[c / G];
      const double mu = grp_dsum<NT>(sd, red, t, 0) * rC;
      double ss = 0.0;
      for (int c = t; c < C; c += NT) {
        const double e = ((double)x[c] - mb[c / G]) - mu;
        ss += e * e;
      }
      const double thr = cut.k * sqrt(grp_dsum<NT>(ss, red, t, 0) * rC);
      for (int w = warp; w < W; w += NT / 32) {
        const int c = 32 * w + lane;
        const bool f = c < C && fabs(((double)x[c] - mb[c / G]) - mu) > thr;
        const unsigned bits = __ballot_sync(0xffffffffu, f);
        if (lane == 0) fcur[w] = bits;
      }
      __syncthreads();
      if (cut.replace == REP_MEDIAN) {
        // lower median of each bin with a flag: radix select on order-preserving keys
        for (int g = warp; g < NB; g += NT / 32) {
          const int c0 = g * G, c1 = min(c0 + G, C);
          bool any = false;
          for (int c = c0 + lane; c < c1; c += 32) any |= ((fcur[c >> 5] >> (c & 31)) & 1u) != 0u;
          if (!__any_sync(0xffffffffu, any)) continue;
          const int rank = (c1 - c0 - 1) >> 1;
          unsigned prefix = 0;
          for (int b = 31; b >= 0; b--) {
            const unsigned test = prefix | (1u << b);
            unsigned cnt = 0;
            for (int c = c0 + lane; c < c1; c += 32) cnt += fkey(x[c]) < test ? 1u : 0u;
            cnt = __reduce_add_sync(0xffffffffu, cnt);
            if ((int)cnt <= rank) prefix = test;
          }
          if (lane == 0) rep[g] = key_f(prefix);
        }
        __syncthreads();
      }
      // replace; a draw copies an unflagged value, which no thread writes in this iteration
      for (int w = warp; w < W; w += NT / 32) {
        const int c = 32 * w + lane;
        const unsigned fw = fcur[w];
        if (c < C && ((fw >> lane) & 1u)) {
          const int g = c / G;
          float y = x[c];
          if (rnd) {
            const int c0 = g * G;
            const unsigned gs = (unsigned)(min(c0 + G, C) - c0);
            for (int a = 0; a < DRAW_ATTEMPTS; a++) {
              const int u = c0 + (int)draw_pos(key, c, 2, cut.it0 + it, a, gs);
              if (!((fcur[u >> 5] >> (u & 31)) & 1u)) {
                y = x[u];
                break;
              }
            }
          } else {
            y = rep[g];
          }
          x[c] = y;
        }
        if (lane == 0) facc[w] |= fw;
      }
      __syncthreads();
    }
    for (int c = t; c < C; c += NT) {
      dst[(size_t)c * T + tc] = x[c];
      const bool f = ((facc[c >> 5] >> (c & 31)) & 1u) != 0u;
      if (!J.mask) continue;
      if (P.mask_kind == MASK_BITS) {
        if (f) atomicOr(static_cast<unsigned*>(J.mask) + (size_t)c * W32 + item, 1u << (tc - t_item));
      } else if (P.mask_kind == MASK_BYTES) {
        unsigned char* bp = static_cast<unsigned char*>(J.mask) + (size_t)c * T + tc;
        if (P.mask_or) {
          if (f) *bp = (unsigned char)(__ldcg(bp) | 2u);
        } else {
          *bp = (unsigned char)(f ? 2u : 0u);
        }
      }
    }
    __syncthreads();
  }
}

template <bool RND>
__device__ void fdsc_item_f32(const Params& P, const Job& J, int item, unsigned char* smem, Red32* red) {
  const CutDev& cut = P.fd;
  const int C = J.C, T = J.T, G = cut.bin, NB = J.nb, Gl = J.last_g;
  const int Ws = J.ws;
  const int t_item = item * Ws;
  const int t_end = min(t_item + Ws, T);
  const float* src = static_cast<const float*>(P.fd_reads_out ? J.out : J.in);
  float* dst = static_cast<float*>(J.out);
  const bool rnd = RND && cut.replace == REP_RANDOM;
  const Fd32Layout L = fd32_layout(smem, Ws, C, NB, rnd);
  const FF kff{cut.k_hi, cut.k_lo};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool vec = ((((uintptr_t)src) | ((uintptr_t)dst)) & 15) == 0 && (T & 3) == 0;

  for (int c = threadIdx.x; c < C; c += NT) L.fm[c] = 0;
  if (rnd)
    for (int c = threadIdx.x; c < C; c += NT) L.fcur[c] = 0;  // each unit clears its own bits after use

  for (int t0 = t_item; t0 < t_end; t0 += Ws) {
    const int w = min(Ws, t_end - t0);
    // ---- load the sub-slab: thread per channel; 16-byte asynchronous copies
    //      (all in flight at once, L1 bypassed) where rows allow them
    const int W32 = (T + 31) >> 5;
    const unsigned* mw = J.prog ? static_cast<const unsigned*>(J.mask) + (t0 >> 5) : nullptr;
    if (vec && w == Ws && Ws >= 4) {
      for (int c = threadIdx.x; c < C; c += NT) {
        const float* a = src + (size_t)c * T + t0;
        float* d = L.tile + c * Ws;
        for (int j = 0; j < Ws; j += 4) {
          const unsigned sdst = (unsigned)__cvta_generic_to_shared(d + j);
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sdst), "l"(a + j) : "memory");
        }
        if (mw) {  // with the tile: the TDSC mask word of this channel's sub-slab
          const unsigned sdst = (unsigned)__cvta_generic_to_shared(L.tm + c);
          asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sdst), "l"(mw + (size_t)c * W32) : "memory");
        }
      }
      asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
    } else {
      for (int c = threadIdx.x; c < C; c += NT) {
        const float* a = src + (size_t)c * T + t0;
        float* d = L.tile + c * Ws;
        for (int j = 0; j < w; j++) d[j] = a[j];
        if (mw) L.tm[c] = __ldcg(mw + (size_t)c * W32);
      }
    }
    if (J.prog) {
      // The tile holds the input.  A sample whose TDSC bit is set takes the
      // value TDSC gave it (replay_tdsc).  The TDSC rows of this beam are
      // published (the item waited for them); bits [t0 & 31, +w) of each word
      // are this item's own, so no FDSC bit is there yet.  Two channels of a
      // thread at a time load their records together.
      __syncthreads();  // (the tile and the mask words are complete)
      const int I = P.td.iterations, sh = t0 & 31;
      const unsigned wm = w >= 32 ? 0xFFFFFFFFu : (1u << w) - 1u;
      const float4* prog4 = reinterpret_cast<const float4*>(J.prog);
      for (int cA = threadIdx.x; cA < C; cA += 2 * NT) {
        const int cB = cA + NT;
        unsigned bA = (L.tm[cA] >> sh) & wm;
        unsigned bB = cB < C ? (L.tm[cB] >> sh) & wm : 0u;
        if (!(bA | bB)) continue;
        const float4* pA = prog4 + (size_t)cA * I * 2;
        const float4* pB = prog4 + (size_t)(bB ? cB : cA) * I * 2;
        float4 fA[3], fB[3];
#pragma unroll
        for (int i = 0; i < 3; i++) {
          fA[i] = (bA && i < I) ? __ldcg(pA + 2 * i) : make_float4(0.f, 0.f, 0.f, 0.f);
          fB[i] = (bB && i < I) ? __ldcg(pB + 2 * i) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float* dA = L.tile + cA * Ws;
        while (bA) {
          const int j = __ffs(bA) - 1;
          bA &= bA - 1;
          dA[j] = replay_tdsc(dA[j], pA, fA, I);
        }
        float* dB = L.tile + (size_t)(bB ? cB : cA) * Ws;
        while (bB) {
          const int j = __ffs(bB) - 1;
          bB &= bB - 1;
          dB[j] = replay_tdsc(dB[j], pB, fB, I);
        }
      }
    }
    __syncthreads();

    const int U = w * NB;
    // 4-sample sub-slabs of 32-channel bins, mean replacement: a thread owns half
    // a bin (16 channels) over the 4 samples, read as one float4 per channel
    const bool quad = w == 4 && Ws == 4 && G == 32 && (C & 31) == 0 && cut.replace == REP_MEAN;
    float4* tile4 = reinterpret_cast<float4*>(L.tile);
    for (int it = 0; it < cut.iterations; it++) {
      if (quad) {
        // whole warps take part in every round (the pair shuffle below needs all lanes)
        for (int ub = 0; ub < 2 * NB; ub += NT) {
          const int u = ub + threadIdx.x;
          const bool act = u < 2 * NB;
          const int g = u >> 1, c0 = 32 * g + 16 * (u & 1), rot = u & 7;
          FF s[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
          FF q[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 4
          for (int j = 0; j < (act ? 16 : 0); j++) {
            const float4 v = tile4[c0 + ((j + rot) & 15)];
            ff_acc(s[0], v.x);
            ff_acc_sq(q[0], v.x);
            ff_acc(s[1], v.y);
            ff_acc_sq(q[1], v.y);
            ff_acc(s[2], v.z);
            ff_acc_sq(q[2], v.z);
            ff_acc(s[3], v.w);
            ff_acc_sq(q[3], v.w);
          }
#pragma unroll
          for (int t = 0; t < 4; t++) {
            s[t] = ff_add(s[t], shfl_ff(s[t], 1));  // the other half of the bin
            q[t] = ff_add(q[t], shfl_ff(q[t], 1));
            if (act && (u & 1) == 0) {
              const FF m = ff_add(ff_div_int(s[t], 32), FF{0.f, 0.f});
              const FF m2 = ff_add(q[t], ff_neg(ff_mul(s[t], m)));
              L.um[g * 4 + t] = make_float2(m.hi, m.lo);
              L.uv[g * 4 + t] = make_float2(m2.hi, m2.lo);
              L.uq[g * 4 + t] = q[t].hi;
            }
          }
        }
      } else
      // ---- per (t, bin): float-float sum and sum of squares, bin mean, M2
      for (int u = threadIdx.x; u < U; u += NT) {
        const int t = u % w, g = u / w;
        const int c0 = g * G, n = g == NB - 1 ? Gl : G;
        const int rot = g % n;
        FF s{0.f, 0.f}, q{0.f, 0.f};
        for (int j = 0; j < n; j++) {
          int jj = j + rot;
          if (jj >= n) jj -= n;
          const float y = L.tile[(c0 + jj) * Ws + t];
          ff_acc(s, y);
          ff_acc_sq(q, y);
        }
        const FF m = ff_add(ff_div_int(s, n), FF{0.f, 0.f});  // normalised: m.hi = fl(mean)
        const FF m2 = ff_add(q, ff_neg(ff_mul(s, m)));  // sum (x - m)^2 = Q - S m
        L.um[u] = make_float2(m.hi, m.lo);
        L.uv[u] = make_float2(m2.hi, m2.lo);
        L.uq[u] = q.hi;
      }
      __syncthreads();
      // ---- per column: sigma' over all channels (mu' = 0: every bin's deviations
      //      sum to 0), finished in float-float; a column whose one-pass sums
      //      cancel (mu^2 > 1000 sigma^2) takes the FP64 two-pass of the definition
      for (int t = warp; t < w; t += NT / 32) {
        FF v{0.f, 0.f};
        float qs = 0.f;
        for (int g = lane; g < NB; g += 32) {
          const float2 a = L.uv[g * w + t];
          v = ff_add(v, FF{a.x, a.y});
          qs += L.uq[g * w + t];
        }
        v = warp_ff(v);  // (the same in every lane)
        qs = warp_sum(qs);
        FF thr;
        if (v.hi >= 1e-3f * qs) {
          thr = ff_mul(kff, ff_sqrt(ff_div_int(v, C)));
        } else {
          double sd = 0.0;
          for (int c = lane; c < C; c += 32) {
            const float2 m = L.um[(c / G) * w + t];
            sd += (double)L.tile[c * Ws + t] - ((double)m.x + (double)m.y);
          }
          sd = warp_sum(sd);
          const double rC = 1.0 / (double)C;  // (only on this rare path)
          const double mup = sd * rC;
          double ss = 0.0;
          for (int c = lane; c < C; c += 32) {
            const float2 m = L.um[(c / G) * w + t];
            const double e = ((double)L.tile[c * Ws + t] - ((double)m.x + (double)m.y)) - mup;
            ss += e * e;
          }
          ss = warp_sum(ss);
          thr = ff_from_d(cut.k * sqrt_fast(ss * rC));
        }
        if (lane == 0) {
          L.thr[t] = make_float2(thr.hi, thr.lo);
          L.thr_lo[t] = __fadd_rd(thr.hi, thr.lo);
          L.thr_hi[t] = __fadd_ru(thr.hi, thr.lo);
        }
      }
      __syncthreads();
      // ---- decide and replace
      if (quad) {
        // per half bin: its 16 channels over the 4 samples; a thread owns its
        // channels' flag words (fm) in every 4-sample sub-slab
        const int sh = t0 - t_item;
        for (int u = threadIdx.x; u < 2 * NB; u += NT) {
          const int g = u >> 1, c0 = 32 * g + 16 * (u & 1), rot = u & 7;
          Cut32 cc[4];
#pragma unroll
          for (int t = 0; t < 4; t++) {
            const float2 m = L.um[g * 4 + t];
            cc[t].mu_f = m.x;
            cc[t].mu_lo = m.y;
            cc[t].thr_hi = L.thr[t].x;
            cc[t].thr_lo = L.thr[t].y;
            band_bounds_f(L.thr_lo[t], L.thr_hi[t], fabsf(m.y), cc[t].lo_f, cc[t].hi_f);
          }
#pragma unroll 2
          for (int j = 0; j < 16; j++) {
            const int c = c0 + ((j + rot) & 15);
            float4 v = tile4[c];
            const unsigned nib = flag32x4(v, cc[0], cc[1], cc[2], cc[3]);
            if (nib) {
              if (nib & 1u) v.x = cc[0].mu_f;
              if (nib & 2u) v.y = cc[1].mu_f;
              if (nib & 4u) v.z = cc[2].mu_f;
              if (nib & 8u) v.w = cc[3].mu_f;
              tile4[c] = v;
              L.fm[c] |= nib << sh;
            }
          }
        }
      } else
      for (int u = threadIdx.x; u < U; u += NT) {
        const int t = u % w, g = u / w;
        const int c0 = g * G, n = g == NB - 1 ? Gl : G;
        const float2 m = L.um[u];
        Cut32 cc;
        cc.mu_f = m.x;
        cc.mu_lo = m.y;
        cc.thr_hi = L.thr[t].x;
        cc.thr_lo = L.thr[t].y;
        band_bounds_f(L.thr_lo[t], L.thr_hi[t], fabsf(m.y), cc.lo_f, cc.hi_f);
        const unsigned bit = 1u << (t0 + t - t_item);
        const int rot = g % n;
        if (rnd) {
          // random replacement: this iteration's flags of the bin go to fcur
          // first, so each draw tests the flag of the value it would copy
          const unsigned tb = 1u << t;
          for (int j = 0; j < n; j++)
            if (flag32(L.tile[(c0 + j) * Ws + t], cc)) {
              atomicOr(&L.fcur[c0 + j], tb);
              atomicOr(&L.fm[c0 + j], bit);
            }
          const unsigned long long key = draw_key(J.beam, t0 + t);
          for (int j = 0; j < n; j++) {
            if (!(L.fcur[c0 + j] & tb)) continue;
            for (int a = 0; a < DRAW_ATTEMPTS; a++) {
              const int uu = (int)draw_pos(key, c0 + j, 2, cut.it0 + it, a, (unsigned)n);
              if (!(L.fcur[c0 + uu] & tb)) {
                L.tile[(c0 + j) * Ws + t] = L.tile[(c0 + uu) * Ws + t];
                break;
              }
            }
          }
          for (int j = 0; j < n; j++)
            if (L.fcur[c0 + j] & tb) atomicAnd(&L.fcur[c0 + j], ~tb);
          continue;
        }
        float r = m.x;
        if (cut.replace == REP_MEDIAN) {
          // the median only where the bin has a flag
          bool any = false;
          for (int j = 0; j < n && !any; j++) any = flag32(L.tile[(c0 + j) * Ws + t], cc);
          if (!any) continue;
          r = bin_median_f32(L.tile, c0, n, Ws, t);
        }
        for (int j = 0; j < n; j++) {
          int jj = j + rot;
          if (jj >= n) jj -= n;
          float* p = L.tile + (c0 + jj) * Ws + t;
          if (flag32(*p, cc)) {
            *p = r;
            atomicOr(&L.fm[c0 + jj], bit);
          }
        }
      }
      __syncthreads();
    }

    // ---- store the sub-slab
    for (int c = threadIdx.x; c < C; c += NT) {
      float* a = dst + (size_t)c * T + t0;
      const float* d = L.tile + c * Ws;
      if (vec && w == Ws && Ws >= 4) {
#pragma unroll 2
        for (int j = 0; j < Ws; j += 4) *reinterpret_cast<float4*>(a + j) = *reinterpret_cast<const float4*>(d + j);
      } else {
        for (int j = 0; j < w; j++) a[j] = d[j];
      }
    }
    __syncthreads();
  }

  // ---- flags.  Items of ws samples share a mask word (ws divides 32): each
  //      ORs its flagged bits in; the word was written by the TDSC rows or zeroed.
  const int nt = t_end - t_item;
  const unsigned valid = (1u << nt) - 1u;  // nt <= 8
  if (P.mask_kind == MASK_BITS && J.mask) {
    const int W32 = (T + 31) >> 5;
    const int sh = t_item & 31;
    unsigned* mb = static_cast<unsigned*>(J.mask) + (t_item >> 5);
    for (int c = threadIdx.x; c < C; c += NT) {
      const unsigned f = (L.fm[c] & valid) << sh;
      if (f) atomicOr(mb + (size_t)c * W32, f);
    }
  } else if (P.mask_kind == MASK_BYTES && J.mask) {
    uint8_t* mb = static_cast<uint8_t*>(J.mask);
    for (int u = threadIdx.x; u < C * nt; u += NT) {
      const int c = u / nt, t = u % nt;
      const unsigned f = (L.fm[c] >> t) & 1u;
      uint8_t* bp = mb + (size_t)c * T + t_item + t;
      if (P.mask_or) {
        if (f) *bp = (uint8_t)(__ldcg(bp) | 2u);
      } else {
        *bp = (uint8_t)(f ? 2u : 0u);
      }
    }
  }
  __syncthreads();
  (void)red;
}

// ---------------------------------------------------------------------------
// persistent engine (float32)
// ---------------------------------------------------------------------------
__device__ bool wait_rows_f32(const Params& P, int job, unsigned need, int* flag) {
  if (threadIdx.x == 0) {
    int good = 1;
    const unsigned* ctr = P.counters + 1 + job;
    if (ld_acquire_u32(ctr) < need) {
      const unsigned long long t0 = globaltimer_ns();
      while (ld_acquire_u32(ctr) < need) {
        if (globaltimer_ns() - t0 > P.spin_limit_ns) {
          atomicExch(P.status, 5u);
          good = 0;
          break;
        }
        __nanosleep(128);
      }
    }
    *flag = good;
  }
  __syncthreads();
  const bool ok = *flag != 0;
  __syncthreads();
  return ok;
}

// RND: random replacement is compiled in (a separate build, so that the mean
// and median paths carry none of it)
template <bool RND>
__global__ void __launch_bounds__(NT, 2) k_engine_f32(const __grid_constant__ Params P) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Red32 red[2];
  // TDSC staging mbarriers: [0, 2) the half CTAs, 2 the CTA (one per group, so
  // that a barrier's phases are tracked by the same threads); mpar bits: 0 this
  // half's, 1 the CTA's
  __shared__ __align__(8) unsigned long long s_mbar[3];
  if (threadIdx.x < 3) mbar_init(&s_mbar[threadIdx.x], 1);
  mbar_init_fence();
  __syncthreads();
  unsigned mpar = 0;
  __shared__ int s_item, s_flag;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(P.counters, 1u);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= P.n_items) return;
    int lo = 0, hi = P.n_segs - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (P.segs[mid].start <= item) lo = mid;
      else hi = mid - 1;
    }
    const Seg sg = P.segs[lo];
    const int idx = item - sg.start;
    const Job& J = P.jobs[sg.job];
    if (sg.kind == 0) {
      unsigned done = 1;
      if (J.td_mode == 0) {
        // two rows per item, one per half CTA (each half synchronises on its own barrier)
        const int h = threadIdx.x / (NT / 2), t = threadIdx.x % (NT / 2);
        const int row = 2 * idx + h;
        if (row < J.rows)
          tdsc_row_f32<NT / 2, RND>(P, J, row, smem + h * td32_smem_bytes(J.T), &red[h], t, h, &s_mbar[h], mpar, 0);
        done = (unsigned)min(2, J.rows - 2 * idx);
      } else if (J.td_mode == 1) {
        tdsc_row_f32<NT, RND>(P, J, idx, smem, &red[0], threadIdx.x, 0, &s_mbar[2], mpar, 1);
      } else {
        if constexpr (RND) {
          if (P.td.replace == REP_RANDOM) tdsc_row_f32_long_rnd(P, J, idx, reinterpret_cast<unsigned*>(smem), &red[0]);
          else tdsc_row_f32_long(P, J, idx, &red[0]);
        } else {
          tdsc_row_f32_long(P, J, idx, &red[0]);
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        if (sg.job != P.withhold_job) atomicAdd(P.counters + 1 + sg.job, done);
      }
    } else {
      if (P.wait_tdsc && !wait_rows_f32(P, sg.job, (unsigned)J.rows, &s_flag)) continue;
      if (J.fd_wide) fdsc_wide_f32<RND>(P, J, idx, smem, &red[0]);
      else fdsc_item_f32<RND>(P, J, idx, smem, &red[0]);
    }
  }
}

int engine_smem_f32(const Params& p) {
  int s = 16;
  for (int j = 0; j < p.n_jobs; j++) {
    const Job& J = p.jobs[j];
    if (p.td.iterations > 0 && J.td_mode != 2) {
      const int td = (J.td_mode == 0 ? 2 : 1) * td32_smem_bytes(J.T);
      s = s > td ? s : td;
    } else if (p.td.iterations > 0 && p.td.replace == REP_RANDOM) {
      // mode 2 rows are not staged; with random replacement they keep two flag bitmaps
      const int td = td32_rnd_long_bytes(J.T);
      s = s > td ? s : td;
    }
    if (p.fd.iterations > 0) {
      const int fd = J.fd_wide ? fd_wide_smem_f32(J.C, J.nb)
                               : fd32_smem_bytes(J.ws, J.C, J.nb, p.fd.replace == REP_RANDOM, J.prog != nullptr);
      s = s > fd ? s : fd;
    }
  }
  return s;
}

void* engine_kernel_f32(const Params& p) {
  const bool rnd = (p.td.iterations > 0 && p.td.replace == REP_RANDOM) ||
                   (p.fd.iterations > 0 && p.fd.replace == REP_RANDOM);
  return rnd ? reinterpret_cast<void*>(&k_engine_f32<true>) : reinterpret_cast<void*>(&k_engine_f32<false>);
}

int launch_engine_f32(const Params& p, const LaunchCfg& cfg, void* stream) {
  void* args[] = {const_cast<Params*>(&p)};
  return (int)cudaLaunchKernel(engine_kernel_f32(p), dim3(cfg.grid), dim3(NT), args, (size_t)cfg.smem,
                               (cudaStream_t)stream);
}

}  // namespace rfim
