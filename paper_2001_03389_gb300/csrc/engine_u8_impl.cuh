// engine_u8_impl.cuh -- uint8 TDSC / FDSC device code and the persistent
// work-queue kernel, included by engine_u8.cu (the mean/median build) and
// engine_u8_rnd.cu (the build with random replacement), which compile in
// parallel.
//
// One persistent kernel serves every call.  CTAs of 256 threads dequeue work
// items in queue order:
//   TDSC rows  : rows of up to 200 16-byte chunks are processed by a quarter
//                warp each (32 rows per item), rows of up to 800 chunks by a
//                warp each (8 rows per item), longer rows (up to 6144 chunks)
//                one per item by the whole CTA; all are staged once in shared
//                memory (one TMA bulk copy per warp or CTA row) and every TDSC
//                iteration is a pass over the staged copy.  Rows longer still
//                (up to the exactness bound) are read from memory in every
//                pass.  The output row and its flags are written once.
//   FDSC item  : 32 time samples x all C channels of one beam, transposed into
//                a [t][c] shared-memory tile.  Each warp owns a set of columns
//                (LPC lanes per column), so the FDSC iterations run without CTA
//                barriers; bins holding a sample outside their keep interval
//                are compacted into a per-warp list and resolved one per lane.
// In the fused schedule the FDSC items of a beam wait (bounded) until its TDSC
// rows are published and read their output while it is still in L2.
// Layout: BCT (x[b][c][t], time fastest).
//
// Decision rule (exact, bit-identical to the reference definition):
//   TDSC keeps x iff |T x - S| <= A, A = max{a : (double)a^2 <= fl(k2 (T Q - S^2))};
//   FDSC keeps x iff |G x - S_g| <= A_g, A_g = max{a : (double)(C m_g^2 a^2) <= fl(k2 V)},
//   V = sum over channels of D^2 (see common.cuh).
// With median replacement every replaced value is the row's (bin's) lower
// median, which replacing values by it never changes; so the samples flagged
// by any of the I iterations are those outside the intersection of the I keep
// intervals, and they all end at the median.
#pragma once
#include <cstdint>
#include <cstdio>

#include "engine.h"

namespace rfim {
namespace {  // each including translation unit keeps its own copy

// ---------------------------------------------------------------------------
// memory access helpers
// ---------------------------------------------------------------------------

// 16 bytes at a 16-aligned address, not allocated in L1 (another SM may later
// write these addresses in place, and this SM must not keep a stale copy).
__device__ __forceinline__ uint4 ld16_na(const uint8_t* a) {
  uint4 v;
  asm volatile("ld.global.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(a));
  return v;
}

__device__ __forceinline__ uint8_t ld1_na(const uint8_t* a) {
  unsigned short v;
  asm volatile("ld.global.L1::no_allocate.u8 %0, [%1];" : "=h"(v) : "l"(a));
  return (uint8_t)v;
}

// 16 bytes at a 16-aligned address a; bytes outside [lo, hi) read as 0.
__device__ __forceinline__ uint4 load16_guarded(const uint8_t* a, const uint8_t* lo, const uint8_t* hi) {
  if (a >= lo && a + 16 <= hi) return ld16_na(a);
  uint32_t w[4] = {0, 0, 0, 0};
  for (int b = 0; b < 16; b++) {
    const uint8_t* p = a + b;
    if (p >= lo && p < hi) w[b >> 2] |= (uint32_t)ld1_na(p) << (8 * (b & 3));
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ __forceinline__ uint32_t word_of(const uint4& v, int i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// Store bytes [lo, hi) of a 16-byte chunk whose byte 0 goes to address dst.
__device__ __forceinline__ void store16_partial(uint8_t* dst, const uint4& v, int lo, int hi) {
  for (int b = lo; b < hi; b++) dst[b] = (uint8_t)(word_of(v, b >> 2) >> (8 * (b & 3)));
}

__device__ __forceinline__ void or16_partial(uint8_t* dst, const uint4& v, int lo, int hi) {
  for (int b = lo; b < hi; b++) dst[b] |= (uint8_t)(word_of(v, b >> 2) >> (8 * (b & 3)));
}

// ---------------------------------------------------------------------------
// exact keep intervals, computed by a group of lanes in parallel
// ---------------------------------------------------------------------------

// A = max{a in [0, amax] : mult a^2 <= F}, F = floor(fl(k2 R)) (thr_floor): the
// largest |d x - S| a kept sample may have.  The W lanes of an aligned group
// (W = 8 or 32) each test one candidate around a float estimate; the passing
// candidates form a prefix.  All lanes of the group return A.
template <int W>
__device__ __forceinline__ unsigned max_keep_grp(unsigned long long F, unsigned long long mult, unsigned amax,
                                                 float rcp_mult) {
  const int lane = threadIdx.x & 31;
  const int gl = lane & (W - 1);
  const int gshift = lane & ~(W - 1);
  const unsigned full = (W == 32) ? 0xffffffffu : ((1u << W) - 1u);
  const unsigned gmask = full << gshift;
  const float est = sqrtf((float)F * rcp_mult);  // rcp_mult ~ 1 / mult: an estimate, the candidates decide
  long long e = est < 4.0e9f ? (long long)est : (long long)amax;
  if (e > (long long)amax) e = amax;  // A never exceeds amax
  long long base = e - (W / 2 - 1);
  for (int round = 0; round < 1024; round++) {
    const long long a = base + gl;
    bool ok;
    if (a < 0) ok = true;
    else if (a > (long long)amax) ok = false;
    else ok = mult * (unsigned long long)a * (unsigned long long)a <= F;
    const unsigned b = (__ballot_sync(gmask, ok) >> gshift) & full;
    if (b == full) {
      if (base + (W - 1) >= (long long)amax) return amax;
      base += W;
      continue;
    }
    if (b == 0) {
      base -= W;
      continue;
    }
    return (unsigned)(base + __popc(b) - 1);
  }
  return 0;  // not reached: the float estimate lies within a few units of A
}

// keep interval [lo, hi] of |d x - S| <= A (S, A < 2^31, quotients <= 510)
__device__ __forceinline__ void keep_from(unsigned S, unsigned A, unsigned d, float rcp, int& lo, int& hi) {
  lo = S <= A ? 0 : (int)udiv_q(S - A + d - 1, d, rcp);
  const unsigned hv = udiv_q(S + A, d, rcp);
  hi = hv > 255 ? 255 : (int)hv;
}

// TDSC keep interval of a row; the lanes of the calling group (up to 32) cooperate.
template <int LANES>
__device__ __forceinline__ void tdsc_keep_warp(unsigned long long S, unsigned long long Q, int T, float rcpT,
                                               const ExactK2& k2, int& lo, int& hi) {
  const unsigned long long Tl = (unsigned long long)T;
  const unsigned long long R = Tl * Q - S * S;
  const unsigned A = max_keep_grp<(LANES < 32 ? LANES : 32)>(thr_floor(R, k2), 1ull, 255u * (unsigned)T, 1.0f);
  keep_from((unsigned)S, A, (unsigned)T, rcpT, lo, hi);
}

// bit 7 of each byte set iff the byte is outside a non-empty [lo, hi]
template <bool ODD>
__device__ __forceinline__ uint32_t outside_ne(uint32_t x, const ByteKeep& k) {
  const uint32_t d = absdiff4(x, k.m4);
  uint32_t g = ((d & 0x7F7F7F7Fu) + k.k4) | d;
  if (ODD) {
    const uint32_t e = x ^ k.hi4;
    g &= ((e & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | e;
  }
  return g & 0x80808080u;
}

__device__ __forceinline__ uint4 outside4(const uint4& w, const ByteKeep& k) {
  if (k.all) return make_uint4(0x80808080u, 0x80808080u, 0x80808080u, 0x80808080u);
  if (k.odd)
    return make_uint4(outside_ne<true>(w.x, k), outside_ne<true>(w.y, k), outside_ne<true>(w.z, k),
                      outside_ne<true>(w.w, k));
  return make_uint4(outside_ne<false>(w.x, k), outside_ne<false>(w.y, k), outside_ne<false>(w.z, k),
                    outside_ne<false>(w.w, k));
}

// 0xFF in every flagged byte (flags = 0x80 per byte), on the multiplier
__device__ __forceinline__ uint32_t wide8(uint32_t f) { return (f >> 7) * 0xFFu; }

// select r4 where flagged
__device__ __forceinline__ uint32_t sel8(uint32_t x, uint32_t r4, uint32_t F8) { return x ^ ((x ^ r4) & F8); }

// flags of a 16-byte chunk -> 16 bits (byte b -> bit b), multiplier-based
__device__ __forceinline__ uint32_t chunk_bits16(const uint4& f) {
  const uint32_t b0 = ((f.x >> 7) * 0x01020408u) >> 24, b1 = ((f.y >> 7) * 0x01020408u) >> 24;
  const uint32_t b2 = ((f.z >> 7) * 0x01020408u) >> 24, b3 = ((f.w >> 7) * 0x01020408u) >> 24;
  return b0 + 16u * (b1 + 16u * (b2 + 16u * b3));
}

__device__ __forceinline__ uint32_t sel_bytes(uint32_t x, uint32_t r4, uint32_t f) {
  const uint32_t F = widen80(f);
  return (x & ~F) | (r4 & F);
}

__device__ __forceinline__ uint4 and4(const uint4& a, const uint4& b) {
  return make_uint4(a.x & b.x, a.y & b.y, a.z & b.z, a.w & b.w);
}

// ---------------------------------------------------------------------------
// group reductions: LANES = 8 (a quarter warp per row), 32 (one warp per row)
// or NT (the CTA).  Groups of 8 are aligned lane octets; the four groups of a
// warp may diverge, so every group primitive names only its own lanes.
// ---------------------------------------------------------------------------
constexpr int GRP_SUM_MAX = 8;  // values one grp_sum may reduce (scratch: GRP_SUM_MAX * NT/32 words)

template <int LANES>
__device__ __forceinline__ unsigned grp_mask() {
  if constexpr (LANES >= 32) return 0xffffffffu;
  else return ((1u << LANES) - 1u) << ((threadIdx.x & 31) & ~(LANES - 1));
}

// sum over the lanes of a group of at most 32 lanes (every lane gets it)
template <int LANES, typename V>
__device__ __forceinline__ V grp_lane_sum(V v) {
  const unsigned m = grp_mask<LANES>();
#pragma unroll
  for (int o = 1; o < LANES; o <<= 1) v += __shfl_xor_sync(m, v, o);
  return v;
}

template <int LANES, int N>
__device__ __forceinline__ void grp_sum(unsigned long long (&v)[N], unsigned long long* scr) {
  static_assert(N <= GRP_SUM_MAX, "grp_sum scratch holds GRP_SUM_MAX values per warp");
  if constexpr (LANES <= 32) {
#pragma unroll
    for (int i = 0; i < N; i++) v[i] = grp_lane_sum<LANES>(v[i]);
  } else {
#pragma unroll
    for (int i = 0; i < N; i++) v[i] = warp_sum(v[i]);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < N; i++) scr[i * (NT / 32) + warp] = v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < N; i++) {
      unsigned long long s = 0;
#pragma unroll
      for (int w = 0; w < NT / 32; w++) s += scr[i * (NT / 32) + w];
      v[i] = s;
    }
  }
}

// grp_sum of non-negative row sums: a warp or quarter-warp row holds at most
// 12,769 samples (TD_WARP_CHUNKS), so every partial and total (at most
// 12,769 * 255^2 for sums of squares) fits 32 bits and the lanes reduce in
// 32-bit shuffles.
template <int LANES, int N>
__device__ __forceinline__ void grp_sum_row(unsigned long long (&v)[N], unsigned long long* scr) {
  static_assert(TD_WARP_CHUNKS * 16 * 255ull * 255ull < (1ull << 32), "warp-row sums fit 32 bits");
  if constexpr (LANES == 32) {
#pragma unroll
    for (int i = 0; i < N; i++) v[i] = __reduce_add_sync(0xffffffffu, (unsigned)v[i]);  // (whole warps only)
  } else if constexpr (LANES < 32) {
#pragma unroll
    for (int i = 0; i < N; i++) v[i] = grp_lane_sum<LANES>((unsigned)v[i]);
  } else {
    grp_sum<LANES, N>(v, scr);
  }
}

template <int LANES>
__device__ __forceinline__ void grp_sync() {
  if constexpr (LANES <= 32) __syncwarp(grp_mask<LANES>());
  else __syncthreads();
}

// ---------------------------------------------------------------------------
// TDSC on one row by a group of LANES threads; the row is staged in `st`.
// ---------------------------------------------------------------------------
struct RowGeom {
  const uint8_t* cb;  // 16-aligned base of the chunk grid of the input row
  int head;           // offset of the row start inside chunk 0
  int nch;            // chunks covering the row
  int tail;           // valid bytes in the last chunk (1..16)
};

__device__ __forceinline__ uint4 chunk_valid(const RowGeom& g, int k) {
  const int lo = k == 0 ? g.head : 0, hi = k == g.nch - 1 ? g.tail : 16;
  return chunk_keep_mask(lo, hi);
}

// Lower median of a staged row: m = min{p : #(x <= p) >= need}, need = floor((T+1)/2).
// With f(p) = sum |x - p| (SAD), #(x <= p) = (T + f(p+1) - f(p)) / 2 for p <= 254,
// and a median lies within one standard deviation of the mean.  The first pass
// counts at three consecutive points just below the mean, settling a median of
// floor(mu) - 1 or floor(mu) (bright interference lifts the mean of a row above
// its median); later passes split the remaining window in three.
struct MedSearch {
  int lo, hi;    // the median lies in [lo, hi]
  int pts[4];    // probe points of the current pass
  bool first;
};

// rcpT ~ 1 / T: the window and the first probes need the mean and the
// deviation to well within one unit only (the window has a unit of margin on
// each side, and the search is exact inside any window holding the median).
__device__ __forceinline__ void med_init(MedSearch& m, unsigned long long S, unsigned long long Q, float rcpT) {
  const float mu = (float)S * rcpT;
  float var = (float)Q * rcpT - mu * mu;
  var = var > 0.f ? var : 0.f;
  const float sd = var > 0.f ? var * rsqrtf(var) : 0.f;
  m.lo = max(0, (int)floorf(mu - sd) - 1);
  m.hi = min(255, (int)ceilf(mu + sd) + 1);
  int c = (int)floorf(mu) - 2;
  if (c > m.hi - 2) c = m.hi - 2;
  if (c < m.lo) c = m.lo;
  if (c < 0) c = 0;
  m.pts[0] = c;
  m.pts[1] = c + 1;
  m.pts[2] = c + 2;
  m.pts[3] = c + 3;
  m.first = true;
}

__device__ __forceinline__ uint32_t med_probe4(const MedSearch& m, int i) {
  return (uint32_t)(m.pts[i] > 255 ? 255 : m.pts[i]) * 0x01010101u;
}

// Narrow the window with the SAD sums f[i] = f(pts[i]) (padding already removed).
__device__ __forceinline__ void med_update(MedSearch& m, const unsigned long long (&f)[4], int T) {
  const int need = (T + 1) >> 1;
  auto count_at = [&](int i) -> long long {  // #(x <= pts[i])
    if (m.pts[i] >= 255) return T;
    return ((long long)T + (long long)f[i + 1] - (long long)f[i]) / 2;
  };
  if (m.first) {
    for (int i = 0; i < 3; i++) {
      const int p = m.pts[i];
      if (p < m.lo || p > m.hi) continue;
      if (count_at(i) >= need) {
        m.hi = p;
        break;
      }
      m.lo = p + 1;
    }
    m.first = false;
  } else {
    if (count_at(0) >= need) {
      m.hi = m.pts[0];
    } else {
      m.lo = m.pts[0] + 1;
      if (m.pts[2] <= m.hi) {
        if (count_at(2) >= need) m.hi = m.pts[2];
        else m.lo = m.pts[2] + 1;
      }
    }
  }
  const int a = m.lo + (m.hi - m.lo) / 3, b = m.lo + 2 * (m.hi - m.lo) / 3;
  m.pts[0] = a;
  m.pts[1] = a + 1;
  m.pts[2] = b > a ? b : a + 1;
  m.pts[3] = m.pts[2] + 1;
}

template <int LANES, typename Rd>
__device__ unsigned med_finish(MedSearch& m, const Rd& rd, int nch, int T, unsigned long long npad,
                               unsigned long long* scr, int gl) {
  while (m.lo < m.hi) {
    uint32_t p4[4];
#pragma unroll
    for (int i = 0; i < 4; i++) p4[i] = med_probe4(m, i);
    unsigned f32[4] = {0, 0, 0, 0};
    for (int k = gl; k < nch; k += LANES) {
      const uint4 w = rd(k);
#pragma unroll
      for (int i = 0; i < 4; i++) {
        f32[i] = sad4(w.x, p4[i], f32[i]);
        f32[i] = sad4(w.y, p4[i], f32[i]);
        f32[i] = sad4(w.z, p4[i], f32[i]);
        f32[i] = sad4(w.w, p4[i], f32[i]);
      }
    }
    unsigned long long f[4] = {f32[0], f32[1], f32[2], f32[3]};
    grp_sum_row<LANES, 4>(f, scr);
#pragma unroll
    for (int i = 0; i < 4; i++) f[i] -= npad * (unsigned long long)(m.pts[i] > 255 ? 255 : m.pts[i]);
    med_update(m, f, T);
  }
  return (unsigned)m.lo;
}

// One statistics pass over a staged row (single-replacement mode): sums of the
// kept samples, number of flagged samples and, with PROBE, the SAD sums of the
// median probes.  Padding bytes of the edge chunks are 0; the caller corrects
// the flagged count for them.
template <int LANES, bool ODD, bool PROBE, typename Rd>
__device__ __forceinline__ void td_stats_pass(const Rd& rd, int nch, int gl, const ByteKeep& kp,
                                              const uint32_t (&p4)[4], unsigned (&f32)[4], unsigned& s_in,
                                              unsigned long long& q_in, unsigned& n_out) {
  for (int k = gl; k < nch; k += LANES) {
    const uint4 w = rd(k);
    if (PROBE) {
#pragma unroll
      for (int i = 0; i < 4; i++) {
        f32[i] = sad4(w.x, p4[i], f32[i]);
        f32[i] = sad4(w.y, p4[i], f32[i]);
        f32[i] = sad4(w.z, p4[i], f32[i]);
        f32[i] = sad4(w.w, p4[i], f32[i]);
      }
    }
    const uint32_t f0 = outside_ne<ODD>(w.x, kp), f1 = outside_ne<ODD>(w.y, kp);
    const uint32_t f2 = outside_ne<ODD>(w.z, kp), f3 = outside_ne<ODD>(w.w, kp);
    const uint32_t i0 = w.x & ~wide8(f0), i1 = w.y & ~wide8(f1);
    const uint32_t i2 = w.z & ~wide8(f2), i3 = w.w & ~wide8(f3);
    s_in += dp4a_u(i0, 0x01010101u, 0u) + dp4a_u(i1, 0x01010101u, 0u) + dp4a_u(i2, 0x01010101u, 0u) +
            dp4a_u(i3, 0x01010101u, 0u);
    q_in += dp4a_u(i0, i0, 0u) + dp4a_u(i1, i1, 0u) + dp4a_u(i2, i2, 0u) + dp4a_u(i3, i3, 0u);
    n_out += (__popc(f0) + __popc(f1)) + (__popc(f2) + __popc(f3));
  }
}

// One statistics pass over a staged row of at most 32 chunks per lane (single-
// replacement mode): sums of the samples OUTSIDE [lo, hi] and their count, and
// with PROBE the SAD sums of the median probes.  Outliers are rare, so a sweep
// takes the probes and a cheap superset test of each chunk; each lane then sums
// its own chunks that hold an outlier, exactly.  Padding bytes of the edge
// chunks are 0; the caller corrects the count for them.
template <int LANES, bool ODD, bool PROBE, typename Rd>
__device__ __forceinline__ void td_outlier_pass(const Rd& rd, int nch, int gl, const ByteKeep& kp,
                                                const uint32_t (&p4)[4], unsigned (&f32)[4], unsigned& s_out,
                                                unsigned long long& q_out, unsigned& n_out) {
  uint32_t slow = 0;
  for (int k = gl, r = 0; k < nch; k += LANES, r++) {
    const uint4 w = rd(k);
    if (PROBE) {
#pragma unroll
      for (int i = 0; i < 4; i++) {
        f32[i] = sad4(w.x, p4[i], f32[i]);
        f32[i] = sad4(w.y, p4[i], f32[i]);
        f32[i] = sad4(w.z, p4[i], f32[i]);
        f32[i] = sad4(w.w, p4[i], f32[i]);
      }
    }
    const uint32_t t = outside_fast(w.x, kp) | outside_fast(w.y, kp) | outside_fast(w.z, kp) | outside_fast(w.w, kp);
    if (t & 0x80808080u) slow |= 1u << r;
  }
  while (slow) {
    const int r = __ffs(slow) - 1;
    slow &= slow - 1;
    const uint4 w = rd(gl + r * LANES);
    const uint32_t f0 = outside_ne<ODD>(w.x, kp), f1 = outside_ne<ODD>(w.y, kp);
    const uint32_t f2 = outside_ne<ODD>(w.z, kp), f3 = outside_ne<ODD>(w.w, kp);
    const uint32_t o0 = w.x & wide8(f0), o1 = w.y & wide8(f1), o2 = w.z & wide8(f2), o3 = w.w & wide8(f3);
    s_out += dp4a_u(o0, 0x01010101u, 0u) + dp4a_u(o1, 0x01010101u, 0u) + dp4a_u(o2, 0x01010101u, 0u) +
             dp4a_u(o3, 0x01010101u, 0u);
    q_out += dp4a_u(o0, o0, 0u) + dp4a_u(o1, o1, 0u) + dp4a_u(o2, o2, 0u) + dp4a_u(o3, o3, 0u);
    n_out += (__popc(f0) + __popc(f1)) + (__popc(f2) + __popc(f3));
  }
}

// STREAM: the row is longer than the shared-memory stage; every pass reads its
// 16-byte chunks from global memory (L2) instead, edge chunks masked as the
// staging would, and `st` only holds the output pass's flag words.
// mbar: the staging group's mbarrier; bit `pb` of mpar is the parity of its
// next phase (tracked by every thread of the group).
template <int LANES, bool RND, bool STREAM = false>
__device__ void tdsc_row_u8(const Params& P, const Job& J, int row, uint4* st, unsigned long long* scr, int gl,
                            unsigned long long* mbar, unsigned& mpar, int pb) {
  const CutDev& cut = P.td;
  const int T = J.T;
  const uint8_t* beam_in = static_cast<const uint8_t*>(J.in);
  const uint8_t* rin = beam_in + (size_t)row * T;
  uint8_t* rout = static_cast<uint8_t*>(J.out) + (size_t)row * T;
  const uint8_t* blo = beam_in;
  const uint8_t* bhi = beam_in + (size_t)J.C * T;

  RowGeom g;
  g.head = (int)((uintptr_t)rin & 15);
  g.cb = rin - g.head;
  g.nch = (g.head + T + 15) >> 4;
  g.tail = g.head + T - ((g.nch - 1) << 4);

  // chunk k of the row (edge chunks with their padding bytes zeroed)
  auto rd = [&](int k) -> uint4 {
    if (!STREAM) return st[k];
    const uint8_t* a = g.cb + 16 * k;
    if (k > 0 && k < g.nch - 1) return ld16_na(a);  // interior chunks lie inside the row
    return and4(load16_guarded(a, blo, bhi), chunk_valid(g, k));
  };

  // ---- pass 1: stage the row.  Warp and CTA rows: the run of chunks inside the
  //      beam buffer is one TMA bulk copy issued by the group's first lane,
  //      completing on the group's mbarrier.  Quarter-warp rows (at most 200
  //      chunks) issue 16-byte asynchronous copies from every lane instead:
  //      for them one copy's round trip costs more than it saves.  A chunk that
  //      crosses the buffer's ends takes guarded loads.  Then the edge chunks
  //      are fixed up, and S and Q taken.
  if (!STREAM && LANES < 32) {
    for (int k = gl; k < g.nch; k += LANES) {
      const uint8_t* a = g.cb + 16 * k;
      if (a >= blo && a + 16 <= bhi) {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(st + k)), "l"(a) : "memory");
      } else {
        st[k] = load16_guarded(a, blo, bhi);
      }
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
    grp_sync<LANES>();
  } else if (!STREAM) {
    const int k0 = g.cb >= blo ? 0 : 1;
    const int k1 = g.cb + 16 * g.nch <= bhi ? g.nch : g.nch - 1;
    const bool bulk = k1 > k0;  // (the same in every lane of the group)
    if (bulk && gl == 0) {
      fence_proxy_async_smem();  // earlier generic accesses of the stage come first
      mbar_arrive_expect_tx(mbar, 16u * (unsigned)(k1 - k0));
      bulk_copy_g2s(st + k0, g.cb + 16 * k0, 16u * (unsigned)(k1 - k0), mbar);
    }
    // the chunks the bulk copy leaves out: at most the first and the last
    if (k0 == 1 && gl == 0) st[0] = load16_guarded(g.cb, blo, bhi);
    if (k1 == g.nch - 1 && gl == (g.nch - 1) % LANES)
      st[g.nch - 1] = load16_guarded(g.cb + 16 * (g.nch - 1), blo, bhi);
    if (bulk) {
      if (!mbar_wait_bounded(mbar, (mpar >> pb) & 1u, P.spin_limit_ns)) atomicExch(P.status, 5u);
      mpar ^= 1u << pb;
    }
    grp_sync<LANES>();
  }
  unsigned long long sq[2];
  {
    if (!STREAM) {
      // the bytes of the edge chunks outside the row are zeroed in the stage
      // (by the lane that reads that chunk below)
      if (gl == 0) st[0] = and4(st[0], chunk_valid(g, 0));
      const int kl = g.nch - 1;
      if (kl > 0 && gl == kl % LANES) st[kl] = and4(st[kl], chunk_valid(g, kl));
    }
    // A lane sums at most 372,181 / 16 / 256 + 2 chunks (rows read from memory
    // by the whole CTA; 25 for staged rows), so its partial sums fit 32 bits.
    unsigned s0 = 0, s1 = 0, q0 = 0, q1 = 0;
    for (int k = gl; k < g.nch; k += LANES) {
      const uint4 w = rd(k);
      s0 = dp4a_u(w.x, 0x01010101u, s0);
      q0 = dp4a_u(w.x, w.x, q0);
      s1 = dp4a_u(w.y, 0x01010101u, s1);
      q1 = dp4a_u(w.y, w.y, q1);
      s0 = dp4a_u(w.z, 0x01010101u, s0);
      q0 = dp4a_u(w.z, w.z, q0);
      s1 = dp4a_u(w.w, 0x01010101u, s1);
      q1 = dp4a_u(w.w, w.w, q1);
    }
    sq[0] = (unsigned long long)s0 + s1;
    sq[1] = (unsigned long long)q0 + q1;
  }
  if (LANES <= 32) __syncwarp(grp_mask<LANES>());
  grp_sum_row<LANES, 2>(sq, scr);  // (the CTA variant's barriers also publish the staged row)
  unsigned long long S = sq[0], Q = sq[1];
  if (J.stats && gl == 0) {  // statistics of the input row, for the caller's records (exact in double)
    J.stats[2 * (size_t)row] = (double)S;
    J.stats[2 * (size_t)row + 1] = (double)Q;
  }

  // single: every flagged sample ends at one value (the median, or the mean of a
  // one-iteration cut), so one keep interval (the intersection) decides everything
  const bool median = cut.replace == REP_MEDIAN;
  // (RND: the build that holds random replacement; it runs on warp or CTA rows)
  const bool random = RND && !STREAM && LANES >= 32 && cut.replace == REP_RANDOM;
  const bool single = !random && (median || cut.iterations == 1);
  const unsigned long long npad = 16ull * (unsigned)g.nch - (unsigned)T;  // zero bytes in the chunk grid
  const int I = cut.iterations;
  const float rcpT = __frcp_rn((float)T), rcp2T = 0.5f * rcpT;  // (= 1.0f / T, 0.5f / T)
  unsigned r_med = 0;
  int lo_i[16], hi_i[16];
  ByteKeep kp_i[16];
  uint32_t r4_i[16];
  int klo = 0, khi = 255;  // intersection of the keep intervals so far

  if (single) {
    // Every replaced value is the median m, so after iteration i a sample holds
    // x if x lies in every keep interval so far, else m: S_{i+1} = s_in + n_out m,
    // with s_in = S0 - (sum of the samples outside), S0 the sum of the input row.
    const unsigned long long S0 = S, Q0 = Q;
    MedSearch ms;
    med_init(ms, S, Q, rcpT);
    for (int it = 0; it < I; it++) {
      int lo, hi;
      tdsc_keep_warp<LANES>(S, Q, T, rcpT, cut.k2, lo, hi);
      klo = lo > klo ? lo : klo;
      khi = hi < khi ? hi : khi;
      if (it == I - 1) break;
      // statistics of the kept samples (and, in the first pass, the median probes)
      const ByteKeep kp = make_keep(klo, khi);
      const bool probe = (it == 0);
      uint32_t p4[4];
#pragma unroll
      for (int i = 0; i < 4; i++) p4[i] = med_probe4(ms, i);
      unsigned f32[4] = {0, 0, 0, 0};
      unsigned s_in = 0, n_out = 0;
      unsigned long long q_in = 0;
      if (kp.all) {
        // empty keep interval: every sample is flagged
        if (probe) td_stats_pass<LANES, false, true>(rd, g.nch, gl, make_keep(0, 255), p4, f32, s_in, q_in, n_out);
        s_in = 0;
        q_in = 0;
        n_out = (gl == 0) ? (unsigned)T : 0u;
      } else if (STREAM) {
        if (kp.odd) {
          if (probe) td_stats_pass<LANES, true, true>(rd, g.nch, gl, kp, p4, f32, s_in, q_in, n_out);
          else td_stats_pass<LANES, true, false>(rd, g.nch, gl, kp, p4, f32, s_in, q_in, n_out);
        } else {
          if (probe) td_stats_pass<LANES, false, true>(rd, g.nch, gl, kp, p4, f32, s_in, q_in, n_out);
          else td_stats_pass<LANES, false, false>(rd, g.nch, gl, kp, p4, f32, s_in, q_in, n_out);
        }
      } else {
        // staged rows (at most 32 chunks per lane): sums of the outliers, subtracted below
        unsigned s_out = 0;
        unsigned long long q_out = 0;
        if (kp.odd) {
          if (probe) td_outlier_pass<LANES, true, true>(rd, g.nch, gl, kp, p4, f32, s_out, q_out, n_out);
          else td_outlier_pass<LANES, true, false>(rd, g.nch, gl, kp, p4, f32, s_out, q_out, n_out);
        } else {
          if (probe) td_outlier_pass<LANES, false, true>(rd, g.nch, gl, kp, p4, f32, s_out, q_out, n_out);
          else td_outlier_pass<LANES, false, false>(rd, g.nch, gl, kp, p4, f32, s_out, q_out, n_out);
        }
        s_in = s_out;  // (kept sums taken from the totals after the reduction)
        q_in = q_out;
      }
      unsigned long long red[7] = {s_in, q_in, n_out, f32[0], f32[1], f32[2], f32[3]};
      grp_sum_row<LANES, 7>(red, scr);
      if (!STREAM && !kp.all) {
        red[0] = S0 - red[0];
        red[1] = Q0 - red[1];
      }
      if (!kp.all && klo > 0) red[2] -= npad;  // the zero padding bytes were counted as flagged
      if (probe) {
        unsigned long long f[4] = {red[3], red[4], red[5], red[6]};
#pragma unroll
        for (int i = 0; i < 4; i++) f[i] -= npad * (unsigned long long)(ms.pts[i] > 255 ? 255 : ms.pts[i]);
        med_update(ms, f, T);
        r_med = med_finish<LANES>(ms, rd, g.nch, T, npad, scr, gl);
      }
      S = red[0] + red[2] * r_med;
      Q = red[1] + red[2] * r_med * r_med;
    }
    if (I == 1)
      r_med = median ? med_finish<LANES>(ms, rd, g.nch, T, npad, scr, gl)
                     : udiv_q((unsigned)(2 * S + (unsigned long long)T), 2u * (unsigned)T, rcp2T);
  } else if (random) {
    // Each iteration records its flags per chunk first (fcur), then replaces a
    // flagged byte by the first drawn byte that fcur marks unflagged: those are
    // never written in this iteration, so the draws see the values they test.
    uint16_t* fcur = reinterpret_cast<uint16_t*>(st + g.nch);
    uint16_t* facc = fcur + g.nch;  // flags OR-ed over the iterations
    const uint8_t* sb = reinterpret_cast<const uint8_t*>(st) + g.head;  // row byte t at sb[t]
    const unsigned long long key = draw_key(J.beam, row);
    for (int k = gl; k < g.nch; k += LANES) facc[k] = 0;
    for (int it = 0; it < I; it++) {
      int lo, hi;
      tdsc_keep_warp<LANES>(S, Q, T, rcpT, cut.k2, lo, hi);
      const ByteKeep kp = make_keep(lo, hi);
      for (int k = gl; k < g.nch; k += LANES) {
        const uint4 w = st[k];
        const uint4 vm = (k == 0 || k == g.nch - 1) ? chunk_valid(g, k) : make_uint4(~0u, ~0u, ~0u, ~0u);
        const uint4 f = make_uint4(outside_exact(w.x, kp) & vm.x, outside_exact(w.y, kp) & vm.y,
                                   outside_exact(w.z, kp) & vm.z, outside_exact(w.w, kp) & vm.w);
        fcur[k] = (uint16_t)chunk_bits16(f);
      }
      grp_sync<LANES>();
      long long dS = 0, dQ = 0;
      for (int k = gl; k < g.nch; k += LANES) {
        const uint32_t fb = fcur[k];
        if (!fb) continue;
        uint4 w = st[k];
        uint32_t rem = fb;
        while (rem) {
          const int b = __ffs(rem) - 1;
          rem &= rem - 1;
          const int t = 16 * k + b - g.head;
          const uint32_t old = (word_of(w, b >> 2) >> (8 * (b & 3))) & 0xFFu;
          uint32_t nv = old;
          for (int a = 0; a < DRAW_ATTEMPTS; a++) {
            const unsigned u = draw_pos(key, t, 1, cut.it0 + it, a, (unsigned)T);
            const unsigned pu = (unsigned)g.head + u;
            if (!((fcur[pu >> 4] >> (pu & 15)) & 1u)) {
              nv = sb[u];
              break;
            }
          }
          const uint32_t sh = 8 * (b & 3), msk = 0xFFu << sh;
          if (b < 4) w.x = (w.x & ~msk) | (nv << sh);
          else if (b < 8) w.y = (w.y & ~msk) | (nv << sh);
          else if (b < 12) w.z = (w.z & ~msk) | (nv << sh);
          else w.w = (w.w & ~msk) | (nv << sh);
          dS += (long long)nv - (long long)old;
          dQ += (long long)(nv * nv) - (long long)(old * old);
        }
        st[k] = w;
        facc[k] |= (uint16_t)fb;
      }
      unsigned long long d[2] = {(unsigned long long)dS, (unsigned long long)dQ};
      grp_sum<LANES, 2>(d, scr);  // (the CTA variant's barriers also publish the new row)
      if (LANES <= 32) __syncwarp(grp_mask<LANES>());
      S += d[0];
      Q += d[1];
    }
  } else {
    for (int it = 0; it < I; it++) {
      int lo, hi;
      tdsc_keep_warp<LANES>(S, Q, T, rcpT, cut.k2, lo, hi);
      const unsigned r = udiv_q((unsigned)(2 * S + (unsigned long long)T), 2u * (unsigned)T, rcp2T);
      lo_i[it] = lo;
      hi_i[it] = hi;
      kp_i[it] = make_keep(lo, hi);
      r4_i[it] = splat4(r);
      if (it == I - 1) break;
      // mean: replay iterations 0..it on every value
      unsigned s2 = 0;
      unsigned long long q2 = 0;
      for (int k = gl; k < g.nch; k += LANES) {
        const uint4 w = rd(k);
        const uint4 vm = (k == 0 || k == g.nch - 1) ? chunk_valid(g, k) : make_uint4(~0u, ~0u, ~0u, ~0u);
#pragma unroll
        for (int i = 0; i < 4; i++) {
          uint32_t y = word_of(w, i);
          const uint32_t m = word_of(vm, i);
          for (int j = 0; j <= it; j++) y = sel_bytes(y, r4_i[j], outside_exact(y, kp_i[j]) & m);
          s2 = dp4a_u(y, 0x01010101u, s2);
          q2 += dp4a_u(y, y, 0u);
        }
      }
      unsigned long long d[2] = {s2, q2};
      grp_sum_row<LANES, 2>(d, scr);
      S = d[0];
      Q = d[1];
    }
  }

  // ---- final pass: output and flags
  const bool same_align = (((uintptr_t)rout) & 15) == (uintptr_t)g.head;
  uint8_t* ob = rout - g.head;
  const int W32 = (T + 31) >> 5;
  uint32_t* mrow = (P.mask_kind == MASK_BITS && J.mask) ? static_cast<uint32_t*>(J.mask) + (size_t)row * W32 : nullptr;
  uint8_t* mrowb = (P.mask_kind == MASK_BYTES && J.mask) ? static_cast<uint8_t*>(J.mask) + (size_t)row * T : nullptr;
  const bool mb_align = mrowb && ((((uintptr_t)mrowb) & 15) == (uintptr_t)g.head);
  uint8_t* mbb = mrowb ? mrowb - g.head : nullptr;
  const ByteKeep kk = make_keep(klo, khi);
  const uint32_t rm4 = r_med * 0x01010101u;
  uint16_t* f16 = reinterpret_cast<uint16_t*>(st);  // flag bits of chunk k overwrite consumed staged bytes
  auto final_chunk = [&](const int k) -> uint32_t {
    uint32_t fb = 0;
      const uint4 w = rd(k);
      const bool edge = (k == 0 || k == g.nch - 1);
      const uint4 vm = (edge && !single) ? chunk_valid(g, k) : make_uint4(~0u, ~0u, ~0u, ~0u);
      uint4 y, f;
      if (random) {
        // the row already holds the output; the flags were kept per chunk
        y = w;
        const uint32_t a = reinterpret_cast<const uint16_t*>(st + g.nch)[g.nch + k];
        f = make_uint4(bytes_from_bits4(a) << 7, bytes_from_bits4(a >> 4) << 7, bytes_from_bits4(a >> 8) << 7,
                       bytes_from_bits4(a >> 12) << 7);
      } else if (single) {
        // padding bytes of edge chunks are never stored and their flag bits fall
        // outside the row's mask words, so no masking is needed here
        f = outside4(w, kk);
        y = make_uint4(sel8(w.x, rm4, wide8(f.x)), sel8(w.y, rm4, wide8(f.y)), sel8(w.z, rm4, wide8(f.z)),
                       sel8(w.w, rm4, wide8(f.w)));
      } else {
        uint32_t yy[4], ff[4];
#pragma unroll
        for (int i = 0; i < 4; i++) {
          uint32_t v = word_of(w, i), fl = 0;
          const uint32_t m = word_of(vm, i);
          for (int j = 0; j < I; j++) {
            const uint32_t fj = outside_exact(v, kp_i[j]) & m;
            v = sel_bytes(v, r4_i[j], fj);
            fl |= fj;
          }
          yy[i] = v;
          ff[i] = fl;
        }
        y = make_uint4(yy[0], yy[1], yy[2], yy[3]);
        f = make_uint4(ff[0], ff[1], ff[2], ff[3]);
      }
      fb = chunk_bits16(f);
      if (same_align && !edge) {
        *reinterpret_cast<uint4*>(ob + 16 * k) = y;
      } else {
        const int clo = k == 0 ? g.head : 0, chi = k == g.nch - 1 ? g.tail : 16;
        store16_partial(ob + 16 * k, y, clo, chi);
      }
      if (mrowb) {
        const uint4 fbytes = make_uint4(bytes_from_bits4(fb), bytes_from_bits4(fb >> 4), bytes_from_bits4(fb >> 8),
                                        bytes_from_bits4(fb >> 12));
        if (mb_align && !edge) {
          uint4* mp = reinterpret_cast<uint4*>(mbb + 16 * k);
          if (P.td_mask_or) {
            const uint4 o = *mp;
            *mp = make_uint4(o.x | fbytes.x, o.y | fbytes.y, o.z | fbytes.z, o.w | fbytes.w);
          } else {
            *mp = fbytes;
          }
        } else {
          const int clo = k == 0 ? g.head : 0, chi = k == g.nch - 1 ? g.tail : 16;
          if (P.td_mask_or) or16_partial(mbb + 16 * k, fbytes, clo, chi);
          else store16_partial(mbb + 16 * k, fbytes, clo, chi);
        }
      }
    return fb;
  };
  if (!STREAM && !random && same_align) {
    // A chunk whose bytes all lie inside every keep interval is neither changed
    // nor flagged.  The first sweep stores such chunks as they are (most of a
    // row); each lane then takes the exact path on its own remaining chunks.
    // The row's mask words are zeroed first (unless this pass ORs into an
    // earlier round's flags) and the exact path ORs its bits in with
    // reductions, so no flag word waits on another chunk.  (Rows here have
    // at most 32 chunks per lane: warp rows 800 / 32, quarter-warp rows
    // 200 / 8, CTA rows 6144 / 256.)
    int ilo = klo, ihi = khi;  // the intersection of the iterations' keep intervals
    if (!single)
      for (int j = 0; j < I; j++) {
        ilo = lo_i[j] > ilo ? lo_i[j] : ilo;
        ihi = hi_i[j] < ihi ? hi_i[j] : ihi;
      }
    const ByteKeep ki = make_keep(ilo, ihi);
    uint32_t slow = 0;  // bit r: chunk gl + r * LANES takes the exact path
    // the edge chunks always do; the sweep runs over the interior ones
    const int kend = g.nch - 1;
    if (gl == 0) slow = 1u;
    if (kend > 0 && gl == kend % LANES) slow |= 1u << (kend / LANES);
    const int kfirst = gl == 0 ? LANES : gl, rfirst = gl == 0 ? 1 : 0;
    if (mrowb && !P.td_mask_or) {
      for (int k = kfirst, r = rfirst; k < kend; k += LANES, r++) {
        const uint4 w = st[k];
        const uint32_t t = outside_fast(w.x, ki) | outside_fast(w.y, ki) | outside_fast(w.z, ki) | outside_fast(w.w, ki);
        if (t & 0x80808080u) {
          slow |= 1u << r;
          continue;
        }
        *reinterpret_cast<uint4*>(ob + 16 * k) = w;
        if (mb_align) *reinterpret_cast<uint4*>(mbb + 16 * k) = make_uint4(0u, 0u, 0u, 0u);
        else store16_partial(mbb + 16 * k, make_uint4(0u, 0u, 0u, 0u), 0, 16);
      }
    } else {
      for (int k = kfirst, r = rfirst; k < kend; k += LANES, r++) {
        const uint4 w = st[k];
        const uint32_t t = outside_fast(w.x, ki) | outside_fast(w.y, ki) | outside_fast(w.z, ki) | outside_fast(w.w, ki);
        if (t & 0x80808080u) {
          slow |= 1u << r;
          continue;
        }
        *reinterpret_cast<uint4*>(ob + 16 * k) = w;
      }
    }
    if (mrow && !P.td_mask_or)
      for (int wi = gl; wi < W32; wi += LANES) mrow[wi] = 0u;
    grp_sync<LANES>();  // (orders the zeroed words before the reductions)
    if (single && !mrowb) {
      // one keep interval and one replacement value, bit mask or none: the
      // exact path of final_chunk without its other cases
      while (slow) {
        const int r = __ffs(slow) - 1;
        slow &= slow - 1;
        const int k = gl + r * LANES;
        const uint4 w = st[k];
        const uint4 f = outside4(w, kk);
        const uint4 y = make_uint4(sel8(w.x, rm4, wide8(f.x)), sel8(w.y, rm4, wide8(f.y)), sel8(w.z, rm4, wide8(f.z)),
                                   sel8(w.w, rm4, wide8(f.w)));
        const bool edge = k == 0 || k == g.nch - 1;
        const int clo = k == 0 ? g.head : 0, chi = k == g.nch - 1 ? g.tail : 16;
        if (!edge) *reinterpret_cast<uint4*>(ob + 16 * k) = y;
        else store16_partial(ob + 16 * k, y, clo, chi);
        if (!mrow) continue;
        uint32_t fb = chunk_bits16(f);
        if (edge) fb &= (chi >= 16 ? 0xFFFFu : ((1u << chi) - 1u)) & ~((1u << clo) - 1u);  // not samples
        if (!fb) continue;
        const int s0 = 16 * k - g.head;  // chunk byte b is row sample s0 + b
        const unsigned long long v = s0 < 0 ? (unsigned long long)(fb >> (-s0)) : (unsigned long long)fb << (s0 & 31);
        const int w0 = s0 < 0 ? 0 : s0 >> 5;
        if ((uint32_t)v) atomicOr(mrow + w0, (uint32_t)v);
        if ((uint32_t)(v >> 32)) atomicOr(mrow + w0 + 1, (uint32_t)(v >> 32));
      }
      return;
    }
    while (slow) {
      const int r = __ffs(slow) - 1;
      slow &= slow - 1;
      const int k = gl + r * LANES;
      uint32_t fb = final_chunk(k);
      if (!mrow) continue;
      if (k == 0 || k == g.nch - 1) {  // bits of padding bytes are not samples
        const int clo = k == 0 ? g.head : 0, chi = k == g.nch - 1 ? g.tail : 16;
        fb &= (chi >= 16 ? 0xFFFFu : ((1u << chi) - 1u)) & ~((1u << clo) - 1u);
      }
      if (!fb) continue;
      // chunk byte b is row sample 16 k - head + b
      const int s0 = 16 * k - g.head;
      const unsigned long long v = s0 < 0 ? (unsigned long long)(fb >> (-s0)) : (unsigned long long)fb << (s0 & 31);
      const int w0 = s0 < 0 ? 0 : s0 >> 5;
      if ((uint32_t)v) atomicOr(mrow + w0, (uint32_t)v);
      if ((uint32_t)(v >> 32)) atomicOr(mrow + w0 + 1, (uint32_t)(v >> 32));
    }
    return;
  }
  for (int base = 0; base < g.nch; base += 2 * LANES) {
    const int ka = base + gl, kb = base + LANES + gl;
    uint32_t fa = 0, fbb = 0;
    if (ka < g.nch) fa = final_chunk(ka);
    if (kb < g.nch) fbb = final_chunk(kb);
    if (mrow) {
      grp_sync<LANES>();  // every chunk <= kb of this round has been read
      if (ka < g.nch) f16[ka] = (uint16_t)fa;
      if (kb < g.nch) f16[kb] = (uint16_t)fbb;
    }
  }
  if (mrow) {
    grp_sync<LANES>();
    // word w covers chunk-grid bytes [head + 32 w, head + 32 w + 32): chunks 2w .. 2w+2
    for (int wi = gl; wi < W32; wi += LANES) {
      const int k0 = 2 * wi;
      unsigned long long bits = f16[k0];
      if (k0 + 1 < g.nch) bits |= (unsigned long long)f16[k0 + 1] << 16;
      if (k0 + 2 < g.nch) bits |= (unsigned long long)f16[k0 + 2] << 32;
      uint32_t word = (uint32_t)(bits >> g.head);
      const int valid = T - 32 * wi;
      if (valid < 32) word &= (1u << valid) - 1u;
      mrow[wi] = P.td_mask_or ? (mrow[wi] | word) : word;
    }
  }
}

// ---------------------------------------------------------------------------
// FDSC on one item: 32 time samples x C channels, tile [t][c] in shared memory
//
// Tile addressing: row t holds the C channels of time sample t (pitch bytes,
// a multiple of 128).  Its 16-byte units are XOR-swizzled by (t >> 2) & 7, so
//  - the load/store units (4 channels x 4 samples, lanes along time so that
//    every global access is a contiguous 32-byte run of a row) write and read
//    32 distinct banks, and
//  - the 8 lanes of a column reading 32-byte bins (two 16-byte loads, halves
//    ordered by lane) touch 8 distinct bank groups.
// ---------------------------------------------------------------------------
struct FdLayout {
  uint8_t* tile;          // ws rows x pitch bytes
  unsigned* Sg;           // ws x nbp bin sums
  unsigned* Qg;           // ws x nbp bin sums of squares
  uint16_t* med;          // ws x nbp cached bin medians (0xFFFF unknown)
  uint16_t* mm;           // ws x nbp byte maximum (low byte) and minimum (high byte) of 32-channel bins
  unsigned long long* V;  // ws: sum of D^2 per column
  unsigned* A;            // ws x 2: keep half-widths per bin-size class
  unsigned* fmask;        // flag bits of the item: [FD_ITEM_T][nb | 1] words (bit j = channel 32 g + j) when
                          // bin_bits, else C words (bit = t - t_item)
  unsigned* list;         // ws x nb flagged (t, bin) pairs, one segment per warp
  unsigned* cnt;          // per-warp list lengths
  unsigned* fcur;         // C (random replacement only): flags of the iteration in progress (bit = tile row)
};

__device__ __forceinline__ FdLayout fd_layout(unsigned char* smem, int ws, int pitch, int nb, int C, bool bin_bits) {
  FdLayout L;
  const int nbp = fd_nbp(nb);
  unsigned char* p = smem;
  L.tile = p;
  p += ws * pitch;
  L.Sg = reinterpret_cast<unsigned*>(p);
  p += align16i(ws * nbp * 4);
  L.Qg = reinterpret_cast<unsigned*>(p);
  p += align16i(ws * nbp * 4);
  L.med = reinterpret_cast<uint16_t*>(p);
  p += align16i(ws * nbp * 2);
  L.mm = reinterpret_cast<uint16_t*>(p);
  p += align16i(ws * nbp * 2);
  L.V = reinterpret_cast<unsigned long long*>(p);
  p += align16i(ws * 8);
  L.A = reinterpret_cast<unsigned*>(p);
  p += align16i(ws * 8);
  L.fmask = reinterpret_cast<unsigned*>(p);
  p += fd_flag_bytes(C, nb, bin_bits);
  L.list = reinterpret_cast<unsigned*>(p);
  p += align16i(ws * nb * 4);
  L.cnt = reinterpret_cast<unsigned*>(p);
  p += 4 * (NT / 32);
  L.fcur = reinterpret_cast<unsigned*>(p);
  return L;
}

// byte offset of channel c of tile row r
__device__ __forceinline__ int toff(int r, int c, int pitch) {
  return r * pitch + ((((c >> 4) ^ ((r >> 2) & 7)) << 4) | (c & 15));
}

// Whole 32-sample items of rows on 4-byte boundaries with C % 16 == 0: units of
// 16 channels x 4 samples.  16 row words (lanes along time, so 8 lanes read 32
// contiguous bytes of a row), four 4x4 byte transposes, and one 16-byte shared
// store per sample row (the 16 channels are one swizzle unit).
// 4 bytes of a row at a (any alignment), reading only inside [lo, hi)
__device__ __forceinline__ uint32_t ld_row4(const uint8_t* a, const uint8_t* lo, const uint8_t* hi) {
  const int off = (int)((uintptr_t)a & 3);
  if (off == 0) return *reinterpret_cast<const uint32_t*>(a);
  const uint32_t* al = reinterpret_cast<const uint32_t*>(a - off);
  if ((const uint8_t*)(al + 2) <= hi) return __funnelshift_r(al[0], al[1], 8 * off);
  uint32_t w = 0;
  for (int b = 0; b < 4; b++)
    if (a + b < hi) w |= (uint32_t)a[b] << (8 * b);
  (void)lo;
  return w;
}

// 4 bytes of a row at a (any alignment)
__device__ __forceinline__ void st_row4(uint8_t* a, uint32_t w) {
  const int off = (int)((uintptr_t)a & 3);
  if (off == 0) {
    *reinterpret_cast<uint32_t*>(a) = w;
  } else if (off == 2) {
    reinterpret_cast<uint16_t*>(a)[0] = (uint16_t)w;
    reinterpret_cast<uint16_t*>(a)[1] = (uint16_t)(w >> 16);
  } else {
    for (int b = 0; b < 4; b++) a[b] = (uint8_t)(w >> (8 * b));
  }
}

template <int UPR, bool ALIGNED>  // units per round (their 16 x UPR row words are in flight together);
                                  // ALIGNED: rows start on 4-byte boundaries
__device__ __forceinline__ void fd_load_full(uint8_t* tile, const uint8_t* src, const uint8_t* src_end, int C, int T,
                                             int t0, int pitch) {
  const int nunits = (C >> 4) * 8;
  for (int u0 = threadIdx.x; u0 < nunits; u0 += UPR * NT) {
    uint32_t w[UPR][16];
#pragma unroll
    for (int k = 0; k < UPR; k++) {
      const int u = u0 + k * NT;
      if (u < nunits) {
        const uint8_t* a = src + (size_t)((u >> 3) * 16) * T + t0 + 4 * (u & 7);
        if (ALIGNED) {
#pragma unroll
          for (int i = 0; i < 16; i++) w[k][i] = *reinterpret_cast<const uint32_t*>(a + (size_t)i * T);
        } else {
#pragma unroll
          for (int i = 0; i < 16; i++) w[k][i] = ld_row4(a + (size_t)i * T, src, src_end);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < UPR; k++) {
      const int u = u0 + k * NT;
      if (u < nunits) {
        const int tq = u & 7, cg = u >> 3;
#pragma unroll
        for (int g = 0; g < 4; g++) transpose4x4(w[k][4 * g], w[k][4 * g + 1], w[k][4 * g + 2], w[k][4 * g + 3]);
#pragma unroll
        for (int r = 0; r < 4; r++) {
          const int t = 4 * tq + r;
          *reinterpret_cast<uint4*>(tile + t * pitch + ((cg ^ ((t >> 2) & 7)) << 4)) =
              make_uint4(w[k][r], w[k][4 + r], w[k][8 + r], w[k][12 + r]);
        }
      }
    }
  }
}

template <bool ALIGNED>
__device__ __forceinline__ void fd_store_full(const uint8_t* tile, uint8_t* dst, int C, int T, int t0, int pitch) {
  const int nunits = (C >> 4) * 8;
  for (int u = threadIdx.x; u < nunits; u += NT) {
    const int tq = u & 7, cg = u >> 3;
    uint32_t w[16];
#pragma unroll
    for (int r = 0; r < 4; r++) {
      const int t = 4 * tq + r;
      const uint4 v = *reinterpret_cast<const uint4*>(tile + t * pitch + ((cg ^ ((t >> 2) & 7)) << 4));
      w[r] = v.x;
      w[4 + r] = v.y;
      w[8 + r] = v.z;
      w[12 + r] = v.w;
    }
#pragma unroll
    for (int g = 0; g < 4; g++) transpose4x4(w[4 * g], w[4 * g + 1], w[4 * g + 2], w[4 * g + 3]);
    uint8_t* a = dst + (size_t)(cg * 16) * T + t0 + 4 * tq;
    if (ALIGNED) {
#pragma unroll
      for (int i = 0; i < 16; i++) *reinterpret_cast<uint32_t*>(a + (size_t)i * T) = w[i];
    } else {
#pragma unroll
      for (int i = 0; i < 16; i++) st_row4(a + (size_t)i * T, w[i]);
    }
  }
}

__device__ __forceinline__ unsigned long long fd_contrib(unsigned long long m, unsigned gsz, unsigned S, unsigned Q) {
  // sum over the bin of D^2 = m^2 * G * (G Q - S^2)
  return m * m * (unsigned long long)gsz * ((unsigned long long)gsz * Q - (unsigned long long)S * S);
}

// The same for a 32-channel bin when every bin has 32 channels (m = L / G = 1):
// 32 (32 Q - S^2) <= 32 * 32 * 32 * 255^2 < 2^32, so 32-bit arithmetic is exact.
__device__ __forceinline__ unsigned fd_contrib32(unsigned S, unsigned Q) { return 32u * (32u * Q - S * S); }

// Byte maximum (low byte of the result) and minimum (high byte) of the 32 bytes
// held in w.  The maximum (minimum) of two 16-bit lanes has the larger (smaller)
// high byte, so the 16-bit lane extremes (__vmaxu2 / __vminu2, one instruction
// each, where the byte-lane forms take several) of the words carry the extremes
// of bytes 1 and 3 in their high bytes, and those of the words shifted up one
// byte carry the extremes of bytes 0 and 2.
__device__ __forceinline__ unsigned bin_extremes32(const uint32_t (&w)[8]) {
  uint32_t hx = w[0], lx = w[0] << 8, hn = w[0], ln = w[0] << 8;
#pragma unroll
  for (int i = 1; i < 8; i++) {
    const uint32_t u = w[i] << 8;
    hx = __vmaxu2(hx, w[i]);
    lx = __vmaxu2(lx, u);
    hn = __vminu2(hn, w[i]);
    ln = __vminu2(ln, u);
  }
  const uint32_t x = __vmaxu2(hx, lx), n = __vminu2(hn, ln);  // bytes 1 and 3: the extremes of two halves
  const unsigned mx = max(x >> 24, (x >> 8) & 0xFFu), mn = min(n >> 24, (n >> 8) & 0xFFu);
  return mx | (mn << 8);
}

// Channels [c0, c0+n) of tile row r, read as words (c0 % 4 == 0; bytes past C are 0).
struct BinView {
  uint8_t* tile;
  int r, c0, n, pitch;
  __device__ __forceinline__ uint32_t& word(int i) const {
    return *reinterpret_cast<uint32_t*>(tile + toff(r, c0 + 4 * i, pitch));
  }
  __device__ __forceinline__ uint8_t& byte(int i) const { return tile[toff(r, c0 + i, pitch)]; }
};

// Lower median of a bin: counting search (SAD sums) over [lo, hi].
__device__ unsigned bin_median(const BinView& bv, bool words, int lo, int hi) {
  const int n = bv.n, need = (n + 1) >> 1;
  if (words) {
    const int nw = (n + 3) >> 2;
    const uint32_t tailmask = (n & 3) ? ((1u << (8 * (n & 3))) - 1u) : 0xffffffffu;
    const unsigned npad = 4u * nw - n;  // masked bytes count as 0
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      const uint32_t pa = splat4((uint32_t)mid), pb = splat4((uint32_t)(mid + 1));
      unsigned fa = 0, fb = 0;
      for (int i = 0; i < nw; i++) {
        const uint32_t x = (i == nw - 1) ? (bv.word(i) & tailmask) : bv.word(i);
        fa = sad4(x, pa, fa);
        fb = sad4(x, pb, fb);
      }
      fa -= npad * (unsigned)mid;
      fb -= npad * (unsigned)(mid + 1);
      const int cnt = (int)(((long long)n + (long long)fb - (long long)fa) / 2);
      if (cnt >= need) hi = mid;
      else lo = mid + 1;
    }
  } else {
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      int cnt = 0;
      for (int i = 0; i < n; i++) cnt += bv.byte(i) <= mid;
      if (cnt >= need) hi = mid;
      else lo = mid + 1;
    }
  }
  return (unsigned)lo;
}

// f(p) = sum over the 32 bytes held in w of |x - p| (p <= 255)
__device__ __forceinline__ unsigned sad32(const uint32_t (&w)[8], unsigned p) {
  const uint32_t p4 = splat4(p);
  unsigned a = 0, b = 0;
#pragma unroll
  for (int i = 0; i < 8; i += 2) {
    a = sad4(w[i], p4, a);
    b = sad4(w[i + 1], p4, b);
  }
  return a + b;
}

// Lower median m = min{p : #(x <= p) >= 16} of the 32 bytes held in w, known to
// lie in [lo, hi]: bisection, with #(x <= p) = (32 + f(p+1) - f(p)) / 2 for
// p <= 254, so #(x <= p) >= 16 iff f(p+1) >= f(p).  (Walking from the bin mean
// instead took more steps: in a bin holding an outlier the mean is off.)
__device__ __forceinline__ unsigned median32_regs(const uint32_t (&w)[8], int lo, int hi) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;  // mid < hi <= 255
    if (sad32(w, (unsigned)mid + 1) >= sad32(w, (unsigned)mid)) hi = mid;
    else lo = mid + 1;
  }
  return (unsigned)lo;
}

// The 8 words of 32-channel bin gi of tile row r (two 16-byte units).  With
// sw = 1 the halves are fetched in the other order (bank spreading).
__device__ __forceinline__ void load_bin32(const uint8_t* tile, int r, int gi, int pitch, int sw, uint32_t (&w)[8]) {
  const int s = (r >> 2) & 7;
  const uint8_t* row = tile + r * pitch;
  const uint4* p0 = reinterpret_cast<const uint4*>(row + (((2 * gi) ^ s) << 4));
  const uint4* p1 = reinterpret_cast<const uint4*>(row + (((2 * gi + 1) ^ s) << 4));
  uint4 lo, hi;
  if (sw) {
    hi = *p1;
    lo = *p0;
  } else {
    lo = *p0;
    hi = *p1;
  }
  w[0] = lo.x;
  w[1] = lo.y;
  w[2] = lo.z;
  w[3] = lo.w;
  w[4] = hi.x;
  w[5] = hi.y;
  w[6] = hi.z;
  w[7] = hi.w;
}

__device__ __forceinline__ void store_bin32(uint8_t* tile, int r, int gi, int pitch, const uint32_t (&w)[8]) {
  const int s = (r >> 2) & 7;
  uint8_t* row = tile + r * pitch;
  *reinterpret_cast<uint4*>(row + (((2 * gi) ^ s) << 4)) = make_uint4(w[0], w[1], w[2], w[3]);
  *reinterpret_cast<uint4*>(row + (((2 * gi + 1) ^ s) << 4)) = make_uint4(w[4], w[5], w[6], w[7]);
}

// 4 bytes of a row at global address a (n <= 4 valid), reads only inside [lo, hi)
__device__ __forceinline__ uint32_t load4_row(const uint8_t* a, int n, const uint8_t* lo, const uint8_t* hi) {
  const uintptr_t ia = (uintptr_t)a;
  if (n == 4 && a >= lo && a + 4 <= hi) {
    if ((ia & 3) == 0) return *reinterpret_cast<const uint32_t*>(a);
    const int off = (int)(ia & 3);
    const uint8_t* al = a - off;
    if (al + 8 <= hi) {
      const uint32_t* p = reinterpret_cast<const uint32_t*>(al);
      return __funnelshift_r(p[0], p[1], 8 * off);
    }
  }
  uint32_t w = 0;
  for (int b = 0; b < n; b++) {
    const uint8_t* p = a + b;
    if (p >= lo && p < hi) w |= (uint32_t)(*p) << (8 * b);
  }
  return w;
}

__device__ __forceinline__ void store4_row(uint8_t* a, uint32_t w, int n) {
  if (n == 4 && (((uintptr_t)a) & 3) == 0) {
    *reinterpret_cast<uint32_t*>(a) = w;
    return;
  }
  for (int b = 0; b < n; b++) a[b] = (uint8_t)(w >> (8 * b));
}

// 32 x 32 bit transpose across a warp: lane r holds row r (bit c = column c) and
// gets column r (bit c = row c).  Five butterfly stages; stage s swaps the
// off-diagonal s x s blocks between lanes r and r ^ s.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t v) {
  const int lane = threadIdx.x & 31;
  const uint32_t m[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int i = 0; i < 5; i++) {
    const int sh = 16 >> i;
    const uint32_t o = __shfl_xor_sync(0xffffffffu, v, sh);
    v = (lane & sh) ? ((v & ~m[i]) | ((o >> sh) & m[i])) : ((v & m[i]) | ((o << sh) & ~m[i]));
  }
  return v;
}

// bit b of the result: byte b of a 4-byte flag word (0x80 per flagged byte) is set
__device__ __forceinline__ uint32_t bits_of4(uint32_t f) { return (((f >> 7) * 0x01020408u) >> 24); }

// The FDSC flags of item `item` (nt samples) from the flag words fm into the
// mask (the forms other than bit masks from [t][bin] words, which the item
// writes inline).  Out of line: inlined, these paths raised the register
// pressure of the item loop into spills.
__device__ __noinline__ void fd_write_flags(const Params& P, const Job& J, const unsigned* fm, int item, int nt,
                                            int NB, bool bin_bits) {
  const int C = J.C, T = J.T, t_item = item * FD_ITEM_T, W32 = (T + 31) >> 5;
  const unsigned valid = nt >= 32 ? 0xFFFFFFFFu : ((1u << nt) - 1u);
  if (!J.mask || P.mask_kind == MASK_NONE) return;
  if (bin_bits) {
    // per-channel words from the [t][bin] words: a warp per bin, one transpose
    // each; lane j then holds the word of channel 32 gi + j
    const int lane = threadIdx.x & 31, NBO = NB | 1;
    for (int gi = threadIdx.x >> 5; gi < NB; gi += NT / 32) {
      const unsigned f = warp_transpose32(fm[lane * NBO + gi]) & valid;
      const int c = gi * 32 + lane;
      if (c >= C) continue;
      if (P.mask_kind == MASK_BITS) {
        unsigned* wp = static_cast<unsigned*>(J.mask) + (size_t)c * W32 + item;
        if (P.mask_or) {
          // the word holds this beam's TDSC flags (published before this item
          // started) and only this item writes its FDSC bits: a reduction that
          // returns nothing, so the item does not wait for the word
          if (f) atomicOr(wp, f);
        } else {
          *wp = f;
        }
      } else {
        uint8_t* bp = static_cast<uint8_t*>(J.mask) + (size_t)c * T + t_item;
        for (int t = 0; t < nt; t++) {
          if (P.mask_or) {
            if ((f >> t) & 1u) bp[t] = (uint8_t)(__ldcg(bp + t) | 2u);
          } else {
            bp[t] = (uint8_t)(((f >> t) & 1u) << 1);
          }
        }
      }
    }
  } else if (P.mask_kind == MASK_BITS) {
    unsigned* mb = static_cast<unsigned*>(J.mask) + item;
    for (int c = threadIdx.x; c < C; c += NT) {
      const unsigned f = fm[c] & valid;
      unsigned* wp = mb + (size_t)c * W32;
      if (P.mask_or) {
        if (f) atomicOr(wp, f);  // (as above)
      } else {
        *wp = f;
      }
    }
  } else {
    uint8_t* mb = static_cast<uint8_t*>(J.mask);
    for (int u = threadIdx.x; u < C * nt; u += NT) {
      const int c = u / nt, t = u % nt;
      const unsigned f = (fm[c] >> t) & 1u;
      uint8_t* bp = mb + (size_t)c * T + t_item + t;
      if (P.mask_or) {
        if (f) *bp = (uint8_t)(__ldcg(bp) | 2u);
      } else {
        *bp = (uint8_t)(f ? 2u : 0u);
      }
    }
  }
}

template <bool RND>
__device__ void fdsc_item_u8(const Params& P, const Job& J, int item, unsigned char* smem) {
  const CutDev& cut = P.fd;
  const int C = J.C, T = J.T, G = cut.bin, NB = J.nb, Gl = J.last_g;
  const int t_item = item * FD_ITEM_T;
  const int t_end = min(t_item + FD_ITEM_T, T);
  const int Ws = J.ws, pitch = J.pitch;
  const uint8_t* src = static_cast<const uint8_t*>(P.fd_reads_out ? J.out : J.in);
  uint8_t* dst = static_cast<uint8_t*>(J.out);
  const uint8_t* blo = src;
  const uint8_t* bhi = src + (size_t)C * T;
  const bool words = (G & 3) == 0;  // bins start on 4-byte boundaries of a tile row
  const unsigned long long mf = J.m_full, ml = J.m_last;
  const bool rnd = RND && cut.replace == REP_RANDOM;
  const bool bin_bits = fd_bin_bits(G, rnd);  // flag bits per (t, bin), see fd_flag_bytes
  const int NBO = NB | 1;
  FdLayout L = fd_layout(smem, Ws, pitch, NB, C, bin_bits);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // column ownership: LPC lanes per column, each warp owns 32 / LPC columns
  const int lsh = Ws == 32 ? 3 : (Ws == 16 ? 4 : 5);  // Ws in {32, 16, 8} -> 8, 16, 32 lanes per column
  const int LPC = 1 << lsh;
  const int cpw = 32 >> lsh;
  const int sl = lane & (LPC - 1);
  const int tcol = warp * cpw + (lane >> lsh);
  unsigned* wlist = L.list + warp * (cpw * NB);
  const float rcpG = __frcp_rn((float)G), rcpL = __frcp_rn((float)Gl);  // (= 1.0f / G, 1.0f / Gl)
  const int NBP = fd_nbp(NB);
  const bool fast32 = G == 32;  // whole bins are two 16-byte tile units
  const bool rows4 = ((((uintptr_t)src) | (uintptr_t)T) & 3) == 0;
  const bool out4 = ((((uintptr_t)dst) | (uintptr_t)T) & 3) == 0;
  const unsigned long long multF = (unsigned long long)C * mf * mf;
  const unsigned long long multL = (unsigned long long)C * ml * ml;
  const float rcpF = __frcp_rn((float)multF), rcpLm = __frcp_rn((float)multL);
  // In place (the item writes the buffer its tile was read from: the fused and
  // the separate schedules, or a caller's in-place call), the only samples that
  // differ from what the buffer holds are the flagged ones, and the per-(sample,
  // bin) flag words name them: the item writes back those bytes alone instead
  // of the whole tile.
  const bool sparse_store = bin_bits && static_cast<const void*>(src) == static_cast<const void*>(dst);
  // 32-channel bins keep their byte extremes (L.mm), taken in the statistics pass
  // and again whenever a bin changes, so that the flag pass decides a bin with
  // two comparisons: a byte x of a bin is flagged iff |32 x - S| > A, hence the
  // bin holds one iff 32 max - S > A or S - 32 min > A.  (Random replacement
  // changes bins outside the resolution path below and keeps the sum test.)
  const bool mm_ok = fast32 && !rnd;
  const bool unit_m = mf == 1ull && ml == 1ull;  // every bin has 32 channels (G = 32, C % 32 == 0)

  for (int i = threadIdx.x, n = bin_bits ? FD_ITEM_T * NBO : C; i < n; i += NT) L.fmask[i] = 0;
  if (rnd)
    for (int c = threadIdx.x; c < C; c += NT) L.fcur[c] = 0;  // each bin clears its own bits after use

  for (int t0 = t_item; t0 < t_end; t0 += Ws) {
    const int ws = min(Ws, t_end - t0);
    const int nt4 = (ws + 3) >> 2, nq = (C + 3) >> 2;
    const bool full = ws == 32 && (C & 15) == 0;
    // ---- load: units of 4 channels x 4 samples, lanes along time, transposed into [t][c];
    //      four units per thread are in flight at a time
    if (full && rows4) {
      fd_load_full<1, true>(L.tile, src, bhi, C, T, t0, pitch);
    } else if (full) {
      fd_load_full<1, false>(L.tile, src, bhi, C, T, t0, pitch);
    } else {
      const int nunits = nq * nt4;
      for (int ub = threadIdx.x; ub < nunits; ub += 4 * NT) {
        uint32_t a[4][4];
#pragma unroll
        for (int kk = 0; kk < 4; kk++) {
          const int u = ub + kk * NT;
          if (u < nunits) {
            const int tq = u % nt4, cq = u / nt4;
            const int c = 4 * cq, tt = 4 * tq;
            const int nv = min(4, ws - tt);
            const uint8_t* ap = src + (size_t)c * T + t0 + tt;
            if (nv == 4 && c + 3 < C && rows4) {
              a[kk][0] = *reinterpret_cast<const uint32_t*>(ap);
              a[kk][1] = *reinterpret_cast<const uint32_t*>(ap + T);
              a[kk][2] = *reinterpret_cast<const uint32_t*>(ap + 2 * (size_t)T);
              a[kk][3] = *reinterpret_cast<const uint32_t*>(ap + 3 * (size_t)T);
            } else {
              a[kk][0] = load4_row(ap, nv, blo, bhi);
              a[kk][1] = c + 1 < C ? load4_row(ap + T, nv, blo, bhi) : 0u;
              a[kk][2] = c + 2 < C ? load4_row(ap + 2 * (size_t)T, nv, blo, bhi) : 0u;
              a[kk][3] = c + 3 < C ? load4_row(ap + 3 * (size_t)T, nv, blo, bhi) : 0u;
            }
          }
        }
#pragma unroll
        for (int kk = 0; kk < 4; kk++) {
          const int u = ub + kk * NT;
          if (u < nunits) {
            const int tq = u % nt4, cq = u / nt4;
            const int c = 4 * cq, tt = 4 * tq;
            const int nv = min(4, ws - tt);
            uint32_t a0 = a[kk][0], a1 = a[kk][1], a2 = a[kk][2], a3 = a[kk][3];
            transpose4x4(a0, a1, a2, a3);
            *reinterpret_cast<uint32_t*>(L.tile + toff(tt, c, pitch)) = a0;
            if (nv > 1) *reinterpret_cast<uint32_t*>(L.tile + toff(tt + 1, c, pitch)) = a1;
            if (nv > 2) *reinterpret_cast<uint32_t*>(L.tile + toff(tt + 2, c, pitch)) = a2;
            if (nv > 3) *reinterpret_cast<uint32_t*>(L.tile + toff(tt + 3, c, pitch)) = a3;
          }
        }
      }
    }
    for (int i = threadIdx.x; i < Ws * NBP / 2; i += NT) reinterpret_cast<unsigned*>(L.med)[i] = 0xFFFFFFFFu;
    __syncthreads();

    // ---- per-warp column work, no CTA barrier until the store
    const bool own = tcol < ws;
    {
      unsigned long long v = 0;
      if (own && mm_ok && unit_m) {
        // every bin has 32 channels: sums, extremes and D^2 with no per-bin cases
        const int t = tcol;
        for (int gi = sl; gi < NB; gi += LPC) {
          uint32_t w[8];
          load_bin32(L.tile, t, gi, pitch, (sl >> 2) & 1, w);
          unsigned s0 = 0, q0 = 0, s1 = 0, q1 = 0;
#pragma unroll
          for (int i = 0; i < 8; i += 2) {
            s0 = dp4a_u(w[i], 0x01010101u, s0);
            q0 = dp4a_u(w[i], w[i], q0);
            s1 = dp4a_u(w[i + 1], 0x01010101u, s1);
            q1 = dp4a_u(w[i + 1], w[i + 1], q1);
          }
          const unsigned s = s0 + s1, q = q0 + q1;
          L.Sg[t * NBP + gi] = s;
          L.Qg[t * NBP + gi] = q;
          L.mm[t * NBP + gi] = (uint16_t)bin_extremes32(w);
          v += fd_contrib32(s, q);
        }
      } else if (own) {
        const int t = tcol;
        for (int gi = sl; gi < NB; gi += LPC) {
          const unsigned gsz = gi == NB - 1 ? (unsigned)Gl : (unsigned)G;
          unsigned s = 0, q = 0;
          if (fast32 && gsz == 32) {
            uint32_t w[8];
            load_bin32(L.tile, t, gi, pitch, (sl >> 2) & 1, w);
            unsigned s1 = 0, q1 = 0;
#pragma unroll
            for (int i = 0; i < 8; i += 2) {
              s = dp4a_u(w[i], 0x01010101u, s);
              q = dp4a_u(w[i], w[i], q);
              s1 = dp4a_u(w[i + 1], 0x01010101u, s1);
              q1 = dp4a_u(w[i + 1], w[i + 1], q1);
            }
            s += s1;
            q += q1;
            if (mm_ok) L.mm[t * NBP + gi] = (uint16_t)bin_extremes32(w);
          } else if (words) {
            const BinView bv{L.tile, t, gi * G, (int)gsz, pitch};
            const int nw = (gsz + 3) >> 2;  // bytes past C in the tile are zero
            for (int i = 0; i < nw; i++) {
              const uint32_t x = bv.word(i);
              s = dp4a_u(x, 0x01010101u, s);
              q = dp4a_u(x, x, q);
            }
          } else {
            const BinView bv{L.tile, t, gi * G, (int)gsz, pitch};
            for (unsigned i = 0; i < gsz; i++) {
              const unsigned x = bv.byte(i);
              s += x;
              q += x * x;
            }
          }
          L.Sg[t * NBP + gi] = s;
          L.Qg[t * NBP + gi] = q;
          v += unit_m && gsz == 32 ? (unsigned long long)fd_contrib32(s, q) : fd_contrib(gi == NB - 1 ? ml : mf, gsz, s, q);
        }
      }
      for (int o = 1; o < LPC; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (own && sl == 0) L.V[tcol] = v;
    }
    __syncwarp();

    for (int it = 0; it < cut.iterations; it++) {
      if (it > 0) {
        // sum of D^2 per column from the bin sums as the last iteration left them
        unsigned long long v = 0;
        if (own && unit_m && G == 32)
          for (int gi = sl; gi < NB; gi += LPC) v += fd_contrib32(L.Sg[tcol * NBP + gi], L.Qg[tcol * NBP + gi]);
        else if (own)
          for (int gi = sl; gi < NB; gi += LPC)
            v += fd_contrib(gi == NB - 1 ? ml : mf, gi == NB - 1 ? (unsigned)Gl : (unsigned)G, L.Sg[tcol * NBP + gi],
                            L.Qg[tcol * NBP + gi]);
        for (int o = 1; o < LPC; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (own && sl == 0) L.V[tcol] = v;
        __syncwarp();
      }
      // per-column keep half-widths (8-lane candidate groups)
      const unsigned long long Ft = thr_floor(own ? L.V[tcol] : 0ull, cut.k2);
      const unsigned Af = max_keep_grp<8>(Ft, multF, own ? 255u * (unsigned)G : 0u, rcpF);
      const unsigned Al = (Gl == G) ? Af : max_keep_grp<8>(Ft, multL, own ? 255u * (unsigned)Gl : 0u, rcpLm);
      if (own && sl == 0) {
        L.A[2 * tcol] = Af;
        L.A[2 * tcol + 1] = Al;
      }
      // pass B: bins with a byte outside their keep interval, compacted into this
      //        warp's list (the running length is the same in every lane)
      unsigned nlist = 0;
      const int nsteps = (NB + LPC - 1) >> lsh;
      if (mm_ok && unit_m) {
        // every bin has 32 channels and stored extremes: two comparisons per bin
        const int A = (int)Af;
        const unsigned* srow = L.Sg + tcol * NBP;
        const uint16_t* xrow = L.mm + tcol * NBP;
        const unsigned below = (1u << lane) - 1u;
        for (int stp = 0; stp < nsteps; stp++) {
          const int gi = sl + stp * LPC;
          bool any = false;
          if (own && gi < NB) {
            const int S = (int)srow[gi];
            const unsigned mm = xrow[gi];
            any = (int)(32u * (mm & 0xFFu)) - S > A || S - (int)(32u * (mm >> 8)) > A;
          }
          const unsigned b = __ballot_sync(0xffffffffu, any);
          if (any) wlist[nlist + __popc(b & below)] = ((unsigned)tcol << 16) | (unsigned)gi;
          nlist += __popc(b);
        }
      } else
      for (int stp = 0; stp < nsteps; stp++) {
        const int gi = sl + stp * LPC;
        bool any = false;
        if (own && gi < NB) {
          const bool lastbin = gi == NB - 1;
          const unsigned gsz = lastbin ? (unsigned)Gl : (unsigned)G;
          int lo, hi;
          const unsigned S = L.Sg[tcol * NBP + gi];
          if (mm_ok && gsz == 32) {
            const int A = (int)(lastbin ? Al : Af);
            const unsigned mm = L.mm[tcol * NBP + gi];
            any = (int)(32u * (mm & 0xFFu)) - (int)S > A || (int)S - (int)(32u * (mm >> 8)) > A;
            lo = 0;  // (decided)
            hi = 255;
          } else if (fast32 && gsz == 32) {
            const unsigned A = lastbin ? Al : Af;
            lo = S <= A ? 0 : (int)((S - A + 31) >> 5);
            const unsigned hv = (S + A) >> 5;
            hi = hv > 255 ? 255 : (int)hv;
          } else {
            keep_from(S, lastbin ? Al : Af, gsz, lastbin ? rcpL : rcpG, lo, hi);
          }
          if (!(lo == 0 && hi == 255)) {
            if (fast32 && gsz == 32) {
              // exact: sum over the bin of (x - hi)^+ is (f(hi) + S - 32 hi) / 2 and
              // of (lo - x)^+ is (f(lo) - S + 32 lo) / 2, f(p) the sum of |x - p|
              uint32_t w[8];
              load_bin32(L.tile, tcol, gi, pitch, (sl >> 2) & 1, w);
              const uint32_t h4 = splat4((uint32_t)hi), l4 = splat4((uint32_t)lo);
              unsigned fh0 = 0, fh1 = 0, fl0 = 0, fl1 = 0;
#pragma unroll
              for (int i = 0; i < 8; i += 2) {
                fh0 = sad4(w[i], h4, fh0);
                fh1 = sad4(w[i + 1], h4, fh1);
                fl0 = sad4(w[i], l4, fl0);
                fl1 = sad4(w[i + 1], l4, fl1);
              }
              any = (int)(fh0 + fh1) + (int)S > 32 * hi || (int)(fl0 + fl1) + 32 * lo > (int)S;
            } else if (words) {
              const BinView bv{L.tile, tcol, gi * G, (int)gsz, pitch};
              const ByteKeep kp = make_keep(lo, hi);
              const int nw = (gsz + 3) >> 2;
              uint32_t acc = 0;
              for (int i = 0; i < nw; i++) acc |= outside_fast(bv.word(i), kp);
              any = (acc & 0x80808080u) != 0;
            } else {
              const BinView bv{L.tile, tcol, gi * G, (int)gsz, pitch};
              for (unsigned i = 0; i < gsz; i++) any |= ((int)bv.byte(i) < lo) | ((int)bv.byte(i) > hi);
            }
          }
        }
        const unsigned b = __ballot_sync(0xffffffffu, any);
        if (any) wlist[nlist + __popc(b & ((1u << lane) - 1u))] = ((unsigned)tcol << 16) | (unsigned)gi;
        nlist += __popc(b);
      }
      __syncwarp();  // the list entries are visible to the whole warp
      const unsigned n = nlist;
      // resolve the flagged bins of this warp's columns, one per lane
      if (mm_ok && unit_m) {
        // every bin has 32 channels: the bin in registers, no per-bin cases
        const bool more = it + 1 < cut.iterations;
        const bool med = cut.replace == REP_MEDIAN;
        const int frow0 = t0 - t_item;
        for (unsigned e = lane; e < n; e += 32) {
          const int pair = (int)wlist[e];
          const int t = pair >> 16, gi = pair & 0xFFFF;  // (column, bin) packed by the flag pass
          uint32_t w[8];
          load_bin32(L.tile, t, gi, pitch, lane & 1, w);
          const int ix = t * NBP + gi;
          const unsigned s_old = L.Sg[ix];
          const unsigned A = L.A[2 * t];
          const int lo = s_old <= A ? 0 : (int)((s_old - A + 31) >> 5);
          const unsigned hv = (s_old + A) >> 5;
          const int hi = hv > 255 ? 255 : (int)hv;
          unsigned r;
          if (med) {
            unsigned m = L.med[ix];
            if (m == 0xFFFFu) {
              // the lower median lies within one standard deviation of the bin mean
              const float mu = (float)s_old * (1.0f / 32.0f);
              const float var = (float)L.Qg[ix] * (1.0f / 32.0f) - mu * mu;
              const float sd = sqrtf(var > 0.f ? var : 0.f);
              m = median32_regs(w, max(0, (int)floorf(mu - sd) - 1), min(255, (int)ceilf(mu + sd) + 1));
              L.med[ix] = (uint16_t)m;
            }
            r = m;
          } else {
            r = (s_old + 16) >> 5;  // floor((2 S + 32) / 64)
          }
          const ByteKeep kp = make_keep(lo, hi);
          const uint32_t r4 = splat4(r);
          uint32_t fbm = 0;  // flagged channels of the bin: bit j = channel 32 gi + j
#pragma unroll
          for (int i = 0; i < 8; i++) {
            const uint32_t f = outside_exact(w[i], kp);
            w[i] = sel8(w[i], r4, wide8(f));
            fbm |= (((f >> 7) * 0x01020408u) >> 24) << (4 * i);
          }
          if (fbm) {
            store_bin32(L.tile, t, gi, pitch, w);
            if (more) {  // later iterations start from the new sums and extremes
              unsigned s0 = 0, q0 = 0, s1 = 0, q1 = 0;
#pragma unroll
              for (int i = 0; i < 8; i += 2) {
                s0 = dp4a_u(w[i], 0x01010101u, s0);
                q0 = dp4a_u(w[i], w[i], q0);
                s1 = dp4a_u(w[i + 1], 0x01010101u, s1);
                q1 = dp4a_u(w[i + 1], w[i + 1], q1);
              }
              L.Sg[ix] = s0 + s1;
              L.Qg[ix] = q0 + q1;
              L.mm[ix] = (uint16_t)bin_extremes32(w);
            }
            L.fmask[(frow0 + t) * NBO + gi] |= fbm;  // (this lane alone resolves (t, gi))
          }
        }
      } else
      for (unsigned e = lane; e < n; e += 32) {
        const int pair = (int)wlist[e];
        const int t = pair >> 16, gi = pair & 0xFFFF;  // (column, bin) packed by the flag pass
        const bool lastbin = gi == NB - 1;
        const unsigned gsz = lastbin ? (unsigned)Gl : (unsigned)G;
        const unsigned bit = 1u << (t0 + t - t_item);
        if (rnd) {
          // Random replacement: the bin's flags of this iteration go to fcur
          // first, so each draw tests the flag of the value it would copy
          // (unflagged values are never written in this iteration).
          const unsigned s_old = L.Sg[t * NBP + gi], q_old = L.Qg[t * NBP + gi];
          const unsigned A = L.A[2 * t + (lastbin ? 1 : 0)];
          int lo, hi;
          if (fast32 && gsz == 32) {
            lo = s_old <= A ? 0 : (int)((s_old - A + 31) >> 5);
            const unsigned hv = (s_old + A) >> 5;
            hi = hv > 255 ? 255 : (int)hv;
          } else {
            keep_from(s_old, A, gsz, lastbin ? rcpL : rcpG, lo, hi);
          }
          const int c0 = gi * G;
          const BinView bv{L.tile, t, c0, (int)gsz, pitch};
          const unsigned tb = 1u << t;
          for (unsigned i = 0; i < gsz; i++) {
            const int x = bv.byte(i);
            if (x < lo || x > hi) {
              atomicOr(&L.fcur[c0 + i], tb);
              atomicOr(&L.fmask[c0 + i], bit);
            }
          }
          const unsigned long long key = draw_key(J.beam, t0 + t);
          unsigned s_new = s_old, q_new = q_old;
          for (unsigned i = 0; i < gsz; i++) {
            if (!(L.fcur[c0 + i] & tb)) continue;
            const unsigned x = bv.byte(i);
            unsigned y = x;
            for (int a = 0; a < DRAW_ATTEMPTS; a++) {
              const unsigned u = draw_pos(key, c0 + (int)i, 2, cut.it0 + it, a, gsz);
              if (!(L.fcur[c0 + u] & tb)) {
                y = bv.byte(u);
                break;
              }
            }
            if (y != x) {
              bv.byte(i) = (uint8_t)y;
              s_new += y - x;
              q_new += y * y - x * x;
            }
          }
          for (unsigned i = 0; i < gsz; i++)
            if (L.fcur[c0 + i] & tb) atomicAnd(&L.fcur[c0 + i], ~tb);
          if (s_new != s_old || q_new != q_old) {
            L.Sg[t * NBP + gi] = s_new;
            L.Qg[t * NBP + gi] = q_new;
          }
          continue;
        }
        if (fast32 && gsz == 32) {
          // the bin in registers: two 16-byte loads, half order staggered by lane
          uint32_t w[8];
          load_bin32(L.tile, t, gi, pitch, lane & 1, w);
          const unsigned s_old = L.Sg[t * NBP + gi], q_old = L.Qg[t * NBP + gi];
          const unsigned A = L.A[2 * t + (lastbin ? 1 : 0)];
          const int lo = s_old <= A ? 0 : (int)((s_old - A + 31) >> 5);
          const unsigned hv = (s_old + A) >> 5;
          const int hi = hv > 255 ? 255 : (int)hv;
          unsigned r;
          if (cut.replace == REP_MEDIAN) {
            unsigned m = L.med[t * NBP + gi];
            if (m == 0xFFFFu) {
              // the lower median lies within one standard deviation of the bin mean
              const float mu = (float)s_old * (1.0f / 32.0f);
              const float var = (float)q_old * (1.0f / 32.0f) - mu * mu;
              const float sd = sqrtf(var > 0.f ? var : 0.f);
              m = median32_regs(w, max(0, (int)floorf(mu - sd) - 1), min(255, (int)ceilf(mu + sd) + 1));
              L.med[t * NBP + gi] = (uint16_t)m;
            }
            r = m;
          } else {
            r = (s_old + 16) >> 5;  // floor((2 S + 32) / 64)
          }
          const ByteKeep kp = make_keep(lo, hi);
          const uint32_t r4 = splat4(r);
          uint32_t fbm = 0;  // flagged channels of the bin: bit j = channel 32 gi + j
#pragma unroll
          for (int i = 0; i < 8; i++) {
            const uint32_t f = outside_exact(w[i], kp);
            w[i] = sel8(w[i], r4, wide8(f));
            fbm |= (((f >> 7) * 0x01020408u) >> 24) << (4 * i);
          }
          if (fbm) {  // (the flag pass lists bins by a superset test: some have nothing to replace)
            store_bin32(L.tile, t, gi, pitch, w);
            if (it + 1 < cut.iterations) {  // later iterations start from the new bin sums
              unsigned s0 = 0, q0 = 0, s1 = 0, q1 = 0;
#pragma unroll
              for (int i = 0; i < 8; i += 2) {
                s0 = dp4a_u(w[i], 0x01010101u, s0);
                q0 = dp4a_u(w[i], w[i], q0);
                s1 = dp4a_u(w[i + 1], 0x01010101u, s1);
                q1 = dp4a_u(w[i + 1], w[i + 1], q1);
              }
              L.Sg[t * NBP + gi] = s0 + s1;
              L.Qg[t * NBP + gi] = q0 + q1;
              L.mm[t * NBP + gi] = (uint16_t)bin_extremes32(w);
            }
            L.fmask[(t0 - t_item + t) * NBO + gi] |= fbm;  // (this lane alone resolves (t, gi))
          }
          continue;
        }
        const unsigned S = L.Sg[t * NBP + gi];
        const BinView bv{L.tile, t, gi * G, (int)gsz, pitch};
        int lo, hi;
        keep_from(S, L.A[2 * t + (lastbin ? 1 : 0)], gsz, lastbin ? rcpL : rcpG, lo, hi);
        unsigned r;
        if (cut.replace == REP_MEDIAN) {
          unsigned m = L.med[t * NBP + gi];
          if (m == 0xFFFFu) {
            int wlo = 0, whi = 255;
            if (words) {
              const int nw = (gsz + 3) >> 2;
              unsigned q = 0;
              for (int i = 0; i < nw; i++) q = dp4a_u(bv.word(i), bv.word(i), q);  // bytes past the bin are 0
              const float mu = (float)S / (float)gsz;
              float var = (float)q / (float)gsz - mu * mu;
              const float sd = sqrtf(var > 0.f ? var : 0.f);
              wlo = max(0, (int)floorf(mu - sd) - 1);
              whi = min(255, (int)ceilf(mu + sd) + 1);
            }
            m = bin_median(bv, words, wlo, whi);
            L.med[t * NBP + gi] = (uint16_t)m;
          }
          r = m;
        } else {
          r = udiv_q(2 * S + gsz, 2 * gsz, 0.5f * (lastbin ? rcpL : rcpG));
        }
        unsigned s_old = 0, q_old = 0, s_new = 0, q_new = 0;
        if (words) {
          const ByteKeep kp = make_keep(lo, hi);
          const uint32_t r4 = splat4(r);
          const int nw = (gsz + 3) >> 2;
          for (int i = 0; i < nw; i++) {
            const uint32_t x = bv.word(i);
            uint32_t f = outside_exact(x, kp);
            if (i == nw - 1 && (gsz & 3)) f &= (1u << (8 * (gsz & 3))) - 1u;  // bytes past the bin
            s_old = dp4a_u(x, 0x01010101u, s_old);
            q_old = dp4a_u(x, x, q_old);
            const uint32_t y = sel_bytes(x, r4, f);
            s_new = dp4a_u(y, 0x01010101u, s_new);
            q_new = dp4a_u(y, y, q_new);
            if (f) {
              bv.word(i) = y;
              if (bin_bits) {  // (G = 32: word i holds bin channels 4 i .. 4 i + 3)
                L.fmask[(t0 - t_item + t) * NBO + gi] |= bits_of4(f) << (4 * i);
              } else {
                uint32_t ff = f;
                while (ff) {
                  const int byte = (__ffs(ff) - 1) >> 3;
                  ff &= ff - 1;
                  atomicOr(&L.fmask[gi * G + 4 * i + byte], bit);
                }
              }
            }
          }
        } else {
          for (unsigned i = 0; i < gsz; i++) {
            const unsigned x = bv.byte(i);
            s_old += x;
            q_old += x * x;
            unsigned y = x;
            if ((int)x < lo || (int)x > hi) {
              y = r;
              bv.byte(i) = (uint8_t)r;
              atomicOr(&L.fmask[gi * G + i], bit);
            }
            s_new += y;
            q_new += y * y;
          }
        }
        if (s_new != s_old || q_new != q_old) {
          L.Sg[t * NBP + gi] = s_new;
          L.Qg[t * NBP + gi] = q_new;
        }
      }
      __syncwarp();
    }
    __syncthreads();

    // ---- store: transpose back to [c][t], lanes along time; in place, only the
    //      flagged bytes of this sub-slab (a warp per tile row, a lane per bin)
    if (sparse_store) {
      for (int t = warp; t < ws; t += NT / 32) {
        const unsigned* frow = L.fmask + (t0 - t_item + t) * NBO;
        uint8_t* drow = dst + t0 + t;
        for (int gi = lane; gi < NB; gi += 32) {
          unsigned f = frow[gi];
          while (f) {
            const int c = 32 * gi + __ffs(f) - 1;
            f &= f - 1;
            drow[(size_t)c * T] = L.tile[toff(t, c, pitch)];
          }
        }
      }
    } else if (full && out4) fd_store_full<true>(L.tile, dst, C, T, t0, pitch);
    else if (full) fd_store_full<false>(L.tile, dst, C, T, t0, pitch);
    else for (int u = threadIdx.x; u < nq * nt4; u += NT) {
      const int tq = u % nt4, cq = u / nt4;
      const int c = 4 * cq, tt = 4 * tq;
      const int nv = min(4, ws - tt);
      uint32_t a0 = *reinterpret_cast<const uint32_t*>(L.tile + toff(tt, c, pitch));
      uint32_t a1 = nv > 1 ? *reinterpret_cast<const uint32_t*>(L.tile + toff(tt + 1, c, pitch)) : 0u;
      uint32_t a2 = nv > 2 ? *reinterpret_cast<const uint32_t*>(L.tile + toff(tt + 2, c, pitch)) : 0u;
      uint32_t a3 = nv > 3 ? *reinterpret_cast<const uint32_t*>(L.tile + toff(tt + 3, c, pitch)) : 0u;
      transpose4x4(a0, a1, a2, a3);
      uint8_t* a = dst + (size_t)c * T + t0 + tt;
      if (nv == 4 && c + 3 < C && out4) {
        *reinterpret_cast<uint32_t*>(a) = a0;
        *reinterpret_cast<uint32_t*>(a + T) = a1;
        *reinterpret_cast<uint32_t*>(a + 2 * (size_t)T) = a2;
        *reinterpret_cast<uint32_t*>(a + 3 * (size_t)T) = a3;
      } else {
        store4_row(a, a0, nv);
        if (c + 1 < C) store4_row(a + T, a1, nv);
        if (c + 2 < C) store4_row(a + 2 * (size_t)T, a2, nv);
        if (c + 3 < C) store4_row(a + 3 * (size_t)T, a3, nv);
      }
    }
    __syncthreads();
  }

  // ---- flags
  if (bin_bits && P.mask_kind == MASK_BITS && J.mask) {
    // per-channel words from the [t][bin] words: a warp per bin, one transpose
    // each; lane j then holds the word of channel 32 gi + j
    const int nt = t_end - t_item, W32 = (T + 31) >> 5;
    const unsigned valid = nt >= 32 ? 0xFFFFFFFFu : ((1u << nt) - 1u);
    for (int gi = warp; gi < NB; gi += NT / 32) {
      const unsigned v = L.fmask[lane * NBO + gi];
      const bool any = __any_sync(0xffffffffu, v != 0u);  // (a bin with no flag in the item skips the transpose)
      if (!any && P.mask_or) continue;
      const unsigned f = any ? warp_transpose32(v) & valid : 0u;
      const int c = gi * 32 + lane;
      if (c < C) {
        unsigned* wp = static_cast<unsigned*>(J.mask) + (size_t)c * W32 + item;
        if (P.mask_or) {
          // the word holds this beam's TDSC flags (published before this item
          // started) and only this item writes its FDSC bits: a reduction that
          // returns nothing, so the item does not wait for the word
          if (f) atomicOr(wp, f);
        } else {
          *wp = f;
        }
      }
    }
  } else {
    fd_write_flags(P, J, L.fmask, item, t_end - t_item, NB, bin_bits);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// FDSC on columns wider than the tile: the CTA cleans the item's time samples
// one column at a time.  The column is gathered into shared memory (one byte
// per channel row, read through L2), cleaned there with the same exact integer
// decisions as the tile path, and scattered back; the flags are bits per
// channel.  A warp takes a bin for the sums and the medians, 32 channels for
// the flags and replacements.  Out of line: such beams are rare.
// ---------------------------------------------------------------------------
template <bool RND>
__device__ __noinline__ void fdsc_wide_u8(const Params& P, const Job& J, int item, unsigned char* smem,
                                          unsigned long long* scr) {
  const CutDev& cut = P.fd;
  const int C = J.C, T = J.T, G = cut.bin, NB = J.nb, Gl = J.last_g;
  const int W = (C + 31) >> 5, W32 = (T + 31) >> 5, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t_item = item * FD_ITEM_T, t_end = min(t_item + FD_ITEM_T, T);
  const uint8_t* src = static_cast<const uint8_t*>(P.fd_reads_out ? J.out : J.in);
  uint8_t* dst = static_cast<uint8_t*>(J.out);
  unsigned char* p = smem;
  uint8_t* x = p;  // the column
  p += align16i(C);
  unsigned* fcur = reinterpret_cast<unsigned*>(p);  // flags of this iteration, bit c % 32 of word c / 32
  p += align16i(W * 4);
  unsigned* facc = reinterpret_cast<unsigned*>(p);  // flags of every iteration so far
  p += align16i(W * 4);
  unsigned long long* Sb = reinterpret_cast<unsigned long long*>(p);  // per bin: sum
  p += align16i(NB * 8);
  unsigned long long* Qb = reinterpret_cast<unsigned long long*>(p);  // sum of squares
  p += align16i(NB * 8);
  unsigned* lh = reinterpret_cast<unsigned*>(p);  // keep interval, lo | hi << 16
  p += align16i(NB * 4);
  unsigned* rep = reinterpret_cast<unsigned*>(p);  // replacement value
  const bool rnd = RND && cut.replace == REP_RANDOM;
  const unsigned long long mf = J.m_full, ml = J.m_last;
  const unsigned long long multF = (unsigned long long)C * mf * mf, multL = (unsigned long long)C * ml * ml;
  const float rcpG = __frcp_rn((float)G), rcpL = __frcp_rn((float)Gl);  // (= 1.0f / G, 1.0f / Gl)
  // this item's mask words start from zero unless they hold the beam's TDSC flags
  if (J.mask && P.mask_kind == MASK_BITS && !P.mask_or)
    for (int c = threadIdx.x; c < C; c += NT) static_cast<unsigned*>(J.mask)[(size_t)c * W32 + item] = 0u;
  for (int t = t_item; t < t_end; t++) {
    for (int c = threadIdx.x; c < C; c += NT) x[c] = src[(size_t)c * T + t];
    for (int w = threadIdx.x; w < W; w += NT) facc[w] = 0u;
    __syncthreads();
    const unsigned long long key = draw_key(J.beam, t);
    for (int it = 0; it < cut.iterations; it++) {
      for (int g = warp; g < NB; g += NT / 32) {
        const int c0 = g * G, c1 = min(c0 + G, C);
        unsigned long long s = 0, q = 0;
        for (int c = c0 + lane; c < c1; c += 32) {
          const unsigned v = x[c];
          s += v;
          q += v * v;
        }
        s = warp_sum(s);
        q = warp_sum(q);
        if (lane == 0) {
          Sb[g] = s;
          Qb[g] = q;
        }
      }
      __syncthreads();
      // sum over the column of D^2 = sum over bins of m^2 G (G Q - S^2)
      unsigned long long v[1] = {0};
      for (int g = threadIdx.x; g < NB; g += NT) {
        const bool last = g == NB - 1;
        const unsigned long long gs = last ? (unsigned)Gl : (unsigned)G, m = last ? ml : mf;
        v[0] += m * m * gs * (gs * Qb[g] - Sb[g] * Sb[g]);
      }
      grp_sum<NT, 1>(v, scr);
      const unsigned long long F = thr_floor(v[0], cut.k2);
      const unsigned Af = max_keep_grp<32>(F, multF, 255u * (unsigned)G, __frcp_rn((float)multF));
      const unsigned Al = Gl == G ? Af : max_keep_grp<32>(F, multL, 255u * (unsigned)Gl, __frcp_rn((float)multL));
      for (int g = threadIdx.x; g < NB; g += NT) {
        const bool last = g == NB - 1;
        const unsigned gs = last ? (unsigned)Gl : (unsigned)G;
        int lo, hi;
        keep_from((unsigned)Sb[g], last ? Al : Af, gs, last ? rcpL : rcpG, lo, hi);
        lh[g] = (unsigned)lo | ((unsigned)hi << 16);
        rep[g] = udiv_q((unsigned)(2 * Sb[g] + gs), 2u * gs, 0.5f * (last ? rcpL : rcpG));  // the mean
      }
      __syncthreads();
      for (int w = warp; w < W; w += NT / 32) {
        const int c = 32 * w + lane;
        bool f = false;
        if (c < C) {
          const unsigned b = lh[c / G];
          const int xv = x[c];
          f = xv < (int)(b & 0xFFFFu) || xv > (int)(b >> 16);
        }
        const unsigned bits = __ballot_sync(0xffffffffu, f);
        if (lane == 0) fcur[w] = bits;
      }
      __syncthreads();
      if (cut.replace == REP_MEDIAN) {
        // lower median of each bin with a flag: bisection on counts
        for (int g = warp; g < NB; g += NT / 32) {
          const int c0 = g * G, c1 = min(c0 + G, C);
          bool any = false;
          for (int c = c0 + lane; c < c1; c += 32) any |= ((fcur[c >> 5] >> (c & 31)) & 1u) != 0u;
          if (!__any_sync(0xffffffffu, any)) continue;
          const int need = (c1 - c0 + 1) >> 1;
          int lo = 0, hi = 255;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            unsigned cnt = 0;
            for (int c = c0 + lane; c < c1; c += 32) cnt += x[c] <= mid ? 1u : 0u;
            cnt = __reduce_add_sync(0xffffffffu, cnt);
            if ((int)cnt >= need) hi = mid;
            else lo = mid + 1;
          }
          if (lane == 0) rep[g] = (unsigned)lo;
        }
        __syncthreads();
      }
      // replace; a draw copies an unflagged value, which no thread writes in this iteration
      for (int w = warp; w < W; w += NT / 32) {
        const int c = 32 * w + lane;
        const unsigned fw = fcur[w];
        if (c < C && ((fw >> lane) & 1u)) {
          const int g = c / G;
          unsigned y = x[c];
          if (rnd) {
            const int c0 = g * G;
            const unsigned gs = g == NB - 1 ? (unsigned)Gl : (unsigned)G;
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
          x[c] = (uint8_t)y;
        }
        if (lane == 0) facc[w] |= fw;
      }
      __syncthreads();
    }
    for (int c = threadIdx.x; c < C; c += NT) {
      dst[(size_t)c * T + t] = x[c];
      const bool f = ((facc[c >> 5] >> (c & 31)) & 1u) != 0u;
      if (!J.mask) continue;
      if (P.mask_kind == MASK_BITS) {
        if (f) atomicOr(static_cast<unsigned*>(J.mask) + (size_t)c * W32 + item, 1u << (t - t_item));
      } else if (P.mask_kind == MASK_BYTES) {
        uint8_t* bp = static_cast<uint8_t*>(J.mask) + (size_t)c * T + t;
        if (P.mask_or) {
          if (f) *bp = (uint8_t)(__ldcg(bp) | 2u);
        } else {
          *bp = (uint8_t)(f ? 2u : 0u);
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// persistent engine
// ---------------------------------------------------------------------------
__device__ bool wait_rows(const Params& P, int job, unsigned need, int* flag) {
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

__device__ __forceinline__ int seg_of(const Params& P, int item) {
  int lo = 0, hi = P.n_segs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P.segs[mid].start <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// TDSC of one row longer than the shared-memory stage (the whole CTA, rows read
// from global memory in every pass); out of line, as such rows are rare.
__device__ __noinline__ void tdsc_row_u8_long(const Params& P, const Job& J, int row, uint4* st,
                                              unsigned long long* scr) {
  unsigned no_par = 0;  // (nothing is staged)
  tdsc_row_u8<NT, false, true>(P, J, row, st, scr, threadIdx.x, nullptr, no_par, 0);
}

// TDSC with random replacement on a row longer than the random-replacement
// stage (the whole CTA).  Nothing is staged.  Iteration 0 reads the input row
// and writes every sample of the output row; later iterations read the output
// row and rewrite its flagged samples.  The flags live in shared memory as
// bitmaps over the sample index (fcur: this iteration's, facc: the OR over the
// iterations), so a draw tests the flag of the very sample it would copy, and
// an iteration writes only samples that no draw of it may read.  A warp takes
// one 32-sample word at a time, lane i sample 32 w + i.  Out of line, as such
// rows are rare.
__device__ __noinline__ void tdsc_row_u8_long_rnd(const Params& P, const Job& J, int row, unsigned* bm,
                                                  unsigned long long* scr) {
  const CutDev& cut = P.td;
  const int T = J.T, lane = threadIdx.x & 31;
  const uint8_t* beam_in = static_cast<const uint8_t*>(J.in);
  const uint8_t* rin = beam_in + (size_t)row * T;
  uint8_t* rout = static_cast<uint8_t*>(J.out) + (size_t)row * T;
  const int NW = (T + 31) >> 5;
  unsigned* fcur = bm;
  unsigned* facc = bm + NW;
  for (int w = threadIdx.x; w < NW; w += NT) facc[w] = 0;
  // sums of the input row
  unsigned long long sq[2] = {0, 0};
  for (int i = threadIdx.x; i < T; i += NT) {
    const unsigned x = ld1_na(rin + i);
    sq[0] += x;
    sq[1] += x * x;
  }
  grp_sum<NT, 2>(sq, scr);
  unsigned long long S = sq[0], Q = sq[1];
  if (J.stats && threadIdx.x == 0) {
    J.stats[2 * (size_t)row] = (double)S;
    J.stats[2 * (size_t)row + 1] = (double)Q;
  }
  const unsigned long long key = draw_key(J.beam, row);
  const float rcpT = 1.0f / (float)T;
  for (int it = 0; it < cut.iterations; it++) {
    const uint8_t* src = it == 0 ? rin : rout;  // the current values
    int lo, hi;
    tdsc_keep_warp<NT>(S, Q, T, rcpT, cut.k2, lo, hi);
    for (int w = threadIdx.x >> 5; w < NW; w += NT / 32) {
      const int i = 32 * w + lane;
      bool f = false;
      if (i < T) {
        const int x = ld1_na(src + i);
        f = x < lo || x > hi;
      }
      const unsigned bits = __ballot_sync(0xffffffffu, f);
      if (lane == 0) fcur[w] = bits;
    }
    __syncthreads();
    long long dS = 0, dQ = 0;
    for (int w = threadIdx.x >> 5; w < NW; w += NT / 32) {
      const int i = 32 * w + lane;
      const unsigned fw = fcur[w];
      if (i < T) {
        if ((fw >> lane) & 1u) {
          const unsigned x = ld1_na(src + i);
          unsigned nv = x;
          for (int a = 0; a < DRAW_ATTEMPTS; a++) {
            const unsigned u = draw_pos(key, i, 1, cut.it0 + it, a, (unsigned)T);
            if (!((fcur[u >> 5] >> (u & 31)) & 1u)) {
              nv = ld1_na(src + u);
              break;
            }
          }
          rout[i] = (uint8_t)nv;
          dS += (long long)nv - (long long)x;
          dQ += (long long)(nv * nv) - (long long)(x * x);
        } else if (it == 0 && rout != rin) {
          rout[i] = ld1_na(rin + i);
        }
      }
      if (lane == 0) facc[w] |= fw;
    }
    unsigned long long d[2] = {(unsigned long long)dS, (unsigned long long)dQ};
    grp_sum<NT, 2>(d, scr);  // (its barriers also publish this iteration's writes of the output row)
    S += d[0];
    Q += d[1];
  }
  __syncthreads();
  // the mask: facc holds the row's bits word for word
  if (P.mask_kind == MASK_BITS && J.mask) {
    unsigned* mrow = static_cast<unsigned*>(J.mask) + (size_t)row * NW;
    for (int w = threadIdx.x; w < NW; w += NT) mrow[w] = P.td_mask_or ? (mrow[w] | facc[w]) : facc[w];
  } else if (P.mask_kind == MASK_BYTES && J.mask) {
    uint8_t* mb = static_cast<uint8_t*>(J.mask) + (size_t)row * T;
    for (int i = threadIdx.x; i < T; i += NT) {
      const uint8_t f = (uint8_t)((facc[i >> 5] >> (i & 31)) & 1u);
      mb[i] = P.td_mask_or ? (uint8_t)(mb[i] | f) : f;
    }
  }
  __syncthreads();
}

// MINB = CTAs per SM the register allocation targets (the TDSC row stage is
// 102 KB, so two CTAs share an SM).  RND: random replacement is compiled in
// (a separate build, so that the mean and median paths carry none of it).
template <int MINB, bool RND>
__global__ void __launch_bounds__(NT, MINB) k_engine_u8(const __grid_constant__ Params P) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long scr[GRP_SUM_MAX * (NT / 32)];
  __shared__ int s_item, s_seg, s_flag;
  // TDSC staging mbarriers, one per staging group so that a barrier's phases
  // are always tracked by the same threads: [0, 8) warps, [8, 40) quarter
  // warps, 40 the CTA.  mpar bits: 0 this warp's, 1 this octet's, 2 the CTA's.
  __shared__ __align__(8) unsigned long long s_mbar[TD_MBARS];
  if (threadIdx.x < TD_MBARS) mbar_init(&s_mbar[threadIdx.x], 1);
  mbar_init_fence();
  __syncthreads();
  unsigned mpar = 0;
  for (;;) {
    if (threadIdx.x == 0) {
      const int it = (int)atomicAdd(P.counters, 1u);
      s_item = it;
      s_seg = it < P.n_items ? seg_of(P, it) : 0;  // (one thread searches the segment table)
    }
    __syncthreads();
    const int item = s_item, seg = s_seg;
    __syncthreads();
    if (item >= P.n_items) return;
    const Seg sg = P.segs[seg];
    const int idx = item - sg.start;
    const Job& J = P.jobs[sg.job];
    if (sg.kind == 0) {
      unsigned done;
      if (J.td_mode == 3) {
        // four rows per warp: lane octet q cleans row 4 warp + q in a quarter of the warp's stage
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = lane >> 3;
        const int row = idx * 4 * TD_ROWS_PER_ITEM + 4 * warp + q;
        if (row < J.rows)
          tdsc_row_u8<8, RND>(P, J, row,
                              reinterpret_cast<uint4*>(smem + warp * TD_WARP_STAGE + q * (TD_WARP_STAGE / 4)), scr,
                              lane & 7, &s_mbar[8 + 4 * warp + q], mpar, 1);
        const int left = J.rows - idx * 4 * TD_ROWS_PER_ITEM;
        done = (unsigned)(left < 4 * TD_ROWS_PER_ITEM ? left : 4 * TD_ROWS_PER_ITEM);
      } else if (J.td_mode == 0) {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int row = idx * TD_ROWS_PER_ITEM + warp;
        if (row < J.rows)
          tdsc_row_u8<32, RND>(P, J, row, reinterpret_cast<uint4*>(smem + warp * TD_WARP_STAGE), scr, lane,
                               &s_mbar[warp], mpar, 0);
        const int left = J.rows - idx * TD_ROWS_PER_ITEM;
        done = (unsigned)(left < TD_ROWS_PER_ITEM ? left : TD_ROWS_PER_ITEM);
      } else if (J.td_mode == 1) {
        tdsc_row_u8<NT, RND>(P, J, idx, reinterpret_cast<uint4*>(smem), scr, threadIdx.x, &s_mbar[40], mpar, 2);
        done = 1;
      } else {
        if constexpr (RND) {
          if (P.td.replace == REP_RANDOM) tdsc_row_u8_long_rnd(P, J, idx, reinterpret_cast<unsigned*>(smem), scr);
          else tdsc_row_u8_long(P, J, idx, reinterpret_cast<uint4*>(smem), scr);
        } else {
          tdsc_row_u8_long(P, J, idx, reinterpret_cast<uint4*>(smem), scr);
        }
        done = 1;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        if (sg.job != P.withhold_job) atomicAdd(P.counters + 1 + sg.job, done);
      }
    } else {
      if (P.wait_tdsc && !wait_rows(P, sg.job, (unsigned)J.rows, &s_flag)) continue;
      if (J.fd_wide) fdsc_wide_u8<RND>(P, J, idx, smem, scr);
      else fdsc_item_u8<RND>(P, J, idx, smem);
    }
  }
}

}  // namespace
}  // namespace rfim
