// engine_u8.cu -- uint8 TDSC / FDSC kernels and the persistent work-queue engine.
//
// Work items (one queue, dequeued in order by every CTA of a persistent grid):
//   TDSC row   : one (beam, channel) row of T samples, held in registers by a
//                CTA of 256 threads (16-byte chunks, NCH per thread).  All
//                iterations run on chip; the row's output and TDSC flags are
//                written once.  Completion is published per beam.
//   FDSC item  : 32 time samples x all C channels of one beam.  The slab is
//                loaded (transposed to [t][c]) into shared memory, all FDSC
//                iterations run on chip, output and flags are written once.
//                In the fused schedule the item first waits (bounded) until
//                its beam's TDSC rows are done and reads their output, which
//                the queue order keeps resident in L2.
// Layout: BCT (x[b][c][t], time fastest).
#include <cstdint>
#include <cstdio>

#include "engine.h"

namespace rfim {

// ---------------------------------------------------------------------------
// loads / stores with alignment and bounds handling
// ---------------------------------------------------------------------------

// 16 bytes at a 16-aligned address a, bytes outside [lo, hi) read as 0.
__device__ __forceinline__ uint4 load16_guarded(const uint8_t* a, const uint8_t* lo, const uint8_t* hi) {
  if (a >= lo && a + 16 <= hi) return __ldcs(reinterpret_cast<const uint4*>(a));
  uint32_t w[4] = {0, 0, 0, 0};
  for (int b = 0; b < 16; b++) {
    const uint8_t* p = a + b;
    if (p >= lo && p < hi) w[b >> 2] |= (uint32_t)__ldcs(p) << (8 * (b & 3));
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

// 4 bytes of a row at global address a: bytes [0, n) valid (n <= 4), the rest 0.
// Reads only inside [lo, hi).  `cg` loads bypass L1 (data written by other CTAs).
__device__ __forceinline__ uint32_t load4_any(const uint8_t* a, int n, const uint8_t* lo, const uint8_t* hi) {
  const uintptr_t ia = (uintptr_t)a;
  const int off = (int)(ia & 3);
  const uint8_t* al = a - off;
  if (n == 4 && off == 0 && a >= lo && a + 4 <= hi) return __ldcg(reinterpret_cast<const unsigned*>(a));
  if (n == 4 && al >= lo && al + 8 <= hi) {
    const uint32_t w0 = __ldcg(reinterpret_cast<const unsigned*>(al));
    const uint32_t w1 = __ldcg(reinterpret_cast<const unsigned*>(al + 4));
    return __funnelshift_r(w0, w1, 8 * off);
  }
  uint32_t w = 0;
  for (int b = 0; b < n; b++) {
    const uint8_t* p = a + b;
    if (p >= lo && p < hi) w |= (uint32_t)__ldcg(p) << (8 * b);
  }
  return w;
}

__device__ __forceinline__ void store4_any(uint8_t* a, uint32_t w, int n) {
  if (n == 4 && (((uintptr_t)a) & 3) == 0) {
    *reinterpret_cast<uint32_t*>(a) = w;
    return;
  }
  for (int b = 0; b < n; b++) a[b] = (uint8_t)(w >> (8 * b));
}

// ---------------------------------------------------------------------------
// exact thresholds
// ---------------------------------------------------------------------------

// TDSC keep interval of a row: |T x - S| <= A  <=>  lo <= x <= hi.
__device__ __forceinline__ void tdsc_keep(unsigned long long S, unsigned long long Q, int T, const ExactK2& k2,
                                          int& lo, int& hi) {
  const unsigned long long Tl = (unsigned long long)T;
  const unsigned long long R = Tl * Q - S * S;
  const unsigned long long A = max_keep(R, 1ull, 255u * (unsigned)T, k2);
  const long long lo_num = (long long)S - (long long)A;
  lo = lo_num <= 0 ? 0 : (int)((lo_num + (long long)Tl - 1) / (long long)Tl);
  const unsigned long long hv = (S + A) / Tl;
  hi = hv > 255 ? 255 : (int)hv;
}

// ---------------------------------------------------------------------------
// TDSC on one row, row resident in registers
// ---------------------------------------------------------------------------
struct RowGeom {
  const uint8_t* cb;  // 16-aligned base of the chunk grid of the input row
  int head;           // offset of the row start inside chunk 0
  int nch;            // chunks covering the row
  int tail;           // valid bytes in the last chunk (1..16)
};

__device__ __forceinline__ int chunk_lo(const RowGeom& g, int k) { return k == 0 ? g.head : 0; }
__device__ __forceinline__ int chunk_hi(const RowGeom& g, int k) { return k == g.nch - 1 ? g.tail : 16; }

template <int NCH>
__device__ __forceinline__ unsigned row_median(const uint4 (&v)[NCH], const RowGeom& g, int T, unsigned long long S,
                                               unsigned long long Q, unsigned* red) {
  // Lower median m = min{p : #(x <= p) >= need}, need = floor((T+1)/2).
  // With f(p) = sum |x - p|, #(x <= p) = (T + f(p+1) - f(p)) / 2 for p <= 254.
  // The median lies within one standard deviation of the mean.
  const int need = (T + 1) >> 1;
  const float mu = (float)S / (float)T;
  float var = (float)Q / (float)T - mu * mu;
  var = var > 0.f ? var : 0.f;
  const float sd = sqrtf(var);
  int lo = (int)floorf(mu - sd) - 1, hi = (int)ceilf(mu + sd) + 1;
  lo = lo < 0 ? 0 : lo;
  hi = hi > 255 ? 255 : hi;
  const unsigned npad = 16u * (unsigned)g.nch - (unsigned)T;  // zero bytes inside the chunk grid
  int q0 = (int)floorf(mu);
  bool first = true;
  while (lo < hi) {
    int pts[4];
    if (first) {
      int c = q0 - 1;
      if (c < lo) c = lo;
      if (c > hi - 2) c = hi - 2;
      if (c < 0) c = 0;
      pts[0] = c;
      pts[1] = c + 1;
      pts[2] = c + 2;
      pts[3] = c + 3;
    } else {
      const int a = lo + (hi - lo) / 3, b = lo + 2 * (hi - lo) / 3;
      pts[0] = a;
      pts[1] = a + 1;
      pts[2] = b > a ? b : a + 1;
      pts[3] = pts[2] + 1;
    }
    unsigned f[4] = {0, 0, 0, 0};
    uint32_t p4[4];
#pragma unroll
    for (int i = 0; i < 4; i++) p4[i] = (uint32_t)(pts[i] > 255 ? 255 : pts[i]) * 0x01010101u;
#pragma unroll
    for (int j = 0; j < NCH; j++) {
      const int k = threadIdx.x + j * NT;
      if (k < g.nch) {
#pragma unroll
        for (int i = 0; i < 4; i++) {
          f[i] = sad4(v[j].x, p4[i], f[i]);
          f[i] = sad4(v[j].y, p4[i], f[i]);
          f[i] = sad4(v[j].z, p4[i], f[i]);
          f[i] = sad4(v[j].w, p4[i], f[i]);
        }
      }
    }
    block_sum<unsigned, 4>(f, red);
#pragma unroll
    for (int i = 0; i < 4; i++) f[i] -= npad * (unsigned)(pts[i] > 255 ? 255 : pts[i]);
    auto count_at = [&](int i) -> int {  // #(x <= pts[i]) from f[i], f[i+1]
      if (pts[i] >= 255) return T;
      return (int)(((long long)T + (long long)f[i + 1] - (long long)f[i]) / 2);
    };
    if (first) {
      // counts at c, c+1, c+2
      for (int i = 0; i < 3; i++) {
        const int p = pts[i];
        if (p < lo || p > hi) continue;
        if (count_at(i) >= need) {
          hi = p;
          break;
        }
        lo = p + 1;
      }
      first = false;
    } else {
      const int cA = count_at(0);
      if (cA >= need) {
        hi = pts[0];
      } else {
        lo = pts[0] + 1;
        if (pts[2] <= hi) {
          const int cB = count_at(2);
          if (cB >= need) hi = pts[2];
          else lo = pts[2] + 1;
        }
      }
    }
  }
  return (unsigned)lo;
}

template <int NCH>
__device__ void tdsc_row_u8(const Params& P, const Job& J, int row, unsigned char* smem, unsigned long long* red64,
                            unsigned* red32, int* bc) {
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

  uint4 v[NCH];
  uint32_t fl[NCH];
  unsigned long long sq[2] = {0, 0};
  {
    uint32_t s = 0, q = 0;
#pragma unroll
    for (int j = 0; j < NCH; j++) {
      const int k = threadIdx.x + j * NT;
      uint4 w = make_uint4(0, 0, 0, 0);
      if (k < g.nch) {
        w = load16_guarded(g.cb + 16 * k, blo, bhi);
        const int lo = chunk_lo(g, k), hi = chunk_hi(g, k);
        if (lo != 0 || hi != 16) {
          const uint4 m = chunk_keep_mask(lo, hi);
          w.x &= m.x;
          w.y &= m.y;
          w.z &= m.z;
          w.w &= m.w;
        }
        s = dp4a_u(w.x, 0x01010101u, s);
        s = dp4a_u(w.y, 0x01010101u, s);
        s = dp4a_u(w.z, 0x01010101u, s);
        s = dp4a_u(w.w, 0x01010101u, s);
        q = dp4a_u(w.x, w.x, q);
        q = dp4a_u(w.y, w.y, q);
        q = dp4a_u(w.z, w.z, q);
        q = dp4a_u(w.w, w.w, q);
      }
      v[j] = w;
      fl[j] = 0;
    }
    sq[0] = s;
    sq[1] = q;
  }
  block_sum<unsigned long long, 2>(sq, red64);
  unsigned long long S = sq[0], Q = sq[1];

  unsigned med = 0;
  if (cut.replace == REP_MEDIAN) med = row_median<NCH>(v, g, T, S, Q, red32);

  for (int it = 0; it < cut.iterations; it++) {
    const bool last = (it == cut.iterations - 1);
    if (threadIdx.x == 0) {
      int lo, hi;
      tdsc_keep(S, Q, T, cut.k2, lo, hi);
      bc[0] = lo;
      bc[1] = hi;
      bc[2] = cut.replace == REP_MEDIAN ? (int)med : (int)((2 * S + (unsigned long long)T) / (2ull * T));
    }
    __syncthreads();
    const int lo = bc[0], hi = bc[1], r = bc[2];
    __syncthreads();
    const ByteKeep kp = make_keep(lo, hi);
    const uint32_t r4 = (uint32_t)r * 0x01010101u;
    int ds = 0, dq = 0;
#pragma unroll
    for (int j = 0; j < NCH; j++) {
      const int k = threadIdx.x + j * NT;
      if (k < g.nch) {
        uint4 msk = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
        const int clo = chunk_lo(g, k), chi = chunk_hi(g, k);
        if (clo != 0 || chi != 16) msk = chunk_keep_mask(clo, chi);
        uint32_t* w = reinterpret_cast<uint32_t*>(&v[j]);
        const uint32_t* mw = reinterpret_cast<const uint32_t*>(&msk);
#pragma unroll
        for (int i = 0; i < 4; i++) {
          const uint32_t x = w[i];
          const uint32_t f = outside_exact(x, kp) & mw[i];
          if (f) {
            const uint32_t F = widen80(f);
            if (!last) {
              const uint32_t xm = x & F;
              const int n = __popc(f);
              ds += n * r - (int)dp4a_u(xm, 0x01010101u, 0u);
              dq += n * r * r - (int)dp4a_u(xm, xm, 0u);
            }
            w[i] = (x & ~F) | (r4 & F);
            fl[j] |= bits4(f) << (4 * i);
          }
        }
      }
    }
    if (!last) {
      long long d[2] = {ds, dq};
      block_sum<long long, 2>(d, reinterpret_cast<long long*>(red64));
      S = (unsigned long long)((long long)S + d[0]);
      Q = (unsigned long long)((long long)Q + d[1]);
    }
  }

  // ---- write the row
  const bool same_align = (((uintptr_t)rout) & 15) == (uintptr_t)g.head;
  uint8_t* ob = rout - g.head;  // chunk grid of the output (16-aligned if same_align)
#pragma unroll
  for (int j = 0; j < NCH; j++) {
    const int k = threadIdx.x + j * NT;
    if (k < g.nch) {
      const int clo = chunk_lo(g, k), chi = chunk_hi(g, k);
      if (same_align && clo == 0 && chi == 16)
        *reinterpret_cast<uint4*>(ob + 16 * k) = v[j];
      else
        store16_partial(ob + 16 * k, v[j], clo, chi);
    }
  }
  if (P.mask_kind == MASK_BITS && J.mask) {
    uint16_t* f16 = reinterpret_cast<uint16_t*>(smem);
#pragma unroll
    for (int j = 0; j < NCH; j++) {
      const int k = threadIdx.x + j * NT;
      if (k < g.nch) f16[k] = (uint16_t)fl[j];
    }
    __syncthreads();
    const int W32 = (T + 31) >> 5;
    uint32_t* mrow = static_cast<uint32_t*>(J.mask) + (size_t)row * W32;
    for (int w = threadIdx.x; w < W32; w += NT) {
      const int o = g.head + 32 * w;
      const int k0 = o >> 4, sh = o & 15;
      unsigned long long bits = f16[k0];
      if (k0 + 1 < g.nch) bits |= (unsigned long long)f16[k0 + 1] << 16;
      if (k0 + 2 < g.nch) bits |= (unsigned long long)f16[k0 + 2] << 32;
      uint32_t word = (uint32_t)(bits >> sh);
      const int valid = T - 32 * w;
      if (valid < 32) word &= (1u << valid) - 1u;
      mrow[w] = word;
    }
    __syncthreads();
  } else if (P.mask_kind == MASK_BYTES && J.mask) {
    uint8_t* mrowb = static_cast<uint8_t*>(J.mask) + (size_t)row * T;
    const bool ma = (((uintptr_t)mrowb) & 15) == (uintptr_t)g.head;
    uint8_t* mb = mrowb - g.head;
#pragma unroll
    for (int j = 0; j < NCH; j++) {
      const int k = threadIdx.x + j * NT;
      if (k < g.nch) {
        const uint32_t f = fl[j];
        const uint4 fb = make_uint4(bytes_from_bits4(f), bytes_from_bits4(f >> 4), bytes_from_bits4(f >> 8),
                                    bytes_from_bits4(f >> 12));
        const int clo = chunk_lo(g, k), chi = chunk_hi(g, k);
        if (ma && clo == 0 && chi == 16)
          *reinterpret_cast<uint4*>(mb + 16 * k) = fb;
        else
          store16_partial(mb + 16 * k, fb, clo, chi);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// FDSC on one item: 32 time samples x C channels, tile [t][c] in shared memory
// ---------------------------------------------------------------------------
struct FdLayout {
  uint8_t* tile;          // ws rows x pitch bytes
  unsigned* Sg;           // ws x nb bin sums
  uint16_t* med;          // ws x nb cached bin medians (0xFFFF unknown)
  unsigned long long* V;  // ws: sum of D^2 per column
  unsigned* A;            // ws x 2: keep half-widths per bin-size class
  unsigned* fmask;        // C: FDSC flag bits of the item (bit = t - t_item)
  unsigned* list;         // ws x nb flagged pairs
  unsigned* cnt;
};


__device__ __forceinline__ FdLayout fd_layout(unsigned char* smem, int ws, int pitch, int nb, int C) {
  FdLayout L;
  unsigned char* p = smem;
  L.tile = p;
  p += ws * pitch;
  L.Sg = reinterpret_cast<unsigned*>(p);
  p += align16i(ws * nb * 4);
  L.med = reinterpret_cast<uint16_t*>(p);
  p += align16i(ws * nb * 2);
  L.V = reinterpret_cast<unsigned long long*>(p);
  p += align16i(ws * 8);
  L.A = reinterpret_cast<unsigned*>(p);
  p += align16i(ws * 8);
  L.fmask = reinterpret_cast<unsigned*>(p);
  p += align16i(C * 4);
  L.list = reinterpret_cast<unsigned*>(p);
  p += align16i(ws * nb * 4);
  L.cnt = reinterpret_cast<unsigned*>(p);
  return L;
}

// S and Q of one bin row: channels [c0, c0 + n) of tile row `row`.
__device__ __forceinline__ void bin_sums(const uint8_t* row, int c0, int n, bool words, unsigned& S, unsigned& Q) {
  unsigned s = 0, q = 0;
  if (words) {  // c0 % 4 == 0; bytes past C in the last word are 0
    const uint32_t* w = reinterpret_cast<const uint32_t*>(row + c0);
    const int nw = (n + 3) >> 2;
    for (int i = 0; i < nw; i++) {
      const uint32_t x = w[i];
      s = dp4a_u(x, 0x01010101u, s);
      q = dp4a_u(x, x, q);
    }
  } else {
    for (int i = 0; i < n; i++) {
      const unsigned x = row[c0 + i];
      s += x;
      q += x * x;
    }
  }
  S = s;
  Q = q;
}

// Lower median of bytes [c0, c0+n) of a tile row (n <= 255*...): counting search.
__device__ unsigned bin_median(const uint8_t* row, int c0, int n, bool words) {
  const int need = (n + 1) >> 1;
  int lo = 0, hi = 255;
  if (words) {
    const uint32_t* w = reinterpret_cast<const uint32_t*>(row + c0);
    const int nw = (n + 3) >> 2;
    const unsigned npad = 4u * nw - n;  // zero bytes (channels >= C)
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      const uint32_t pa = (uint32_t)mid * 0x01010101u, pb = (uint32_t)(mid + 1) * 0x01010101u;
      unsigned fa = 0, fb = 0;
      for (int i = 0; i < nw; i++) {
        fa = sad4(w[i], pa, fa);
        fb = sad4(w[i], pb, fb);
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
      for (int i = 0; i < n; i++) cnt += row[c0 + i] <= mid;
      if (cnt >= need) hi = mid;
      else lo = mid + 1;
    }
  }
  return (unsigned)lo;
}

__device__ __forceinline__ unsigned long long fd_contrib(unsigned long long m, unsigned gsz, unsigned S, unsigned Q) {
  // sum over the bin of D^2 = m^2 * G * (G Q - S^2)
  return m * m * (unsigned long long)gsz * ((unsigned long long)gsz * Q - (unsigned long long)S * S);
}

__device__ __forceinline__ void fd_keep(unsigned S, unsigned A, unsigned gsz, int& lo, int& hi) {
  const long long ln = (long long)S - (long long)A;
  lo = ln <= 0 ? 0 : (int)((ln + gsz - 1) / gsz);
  const unsigned hv = (S + A) / gsz;
  hi = hv > 255 ? 255 : (int)hv;
}

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
  const bool words = (G & 3) == 0;
  const unsigned long long mf = J.m_full, ml = J.m_last;
  FdLayout L = fd_layout(smem, Ws, pitch, NB, C);

  for (int c = threadIdx.x; c < C; c += NT) L.fmask[c] = 0;

  for (int t0 = t_item; t0 < t_end; t0 += Ws) {
    const int ws = min(Ws, t_end - t0);
    const int nt4 = (ws + 3) >> 2, nq = (C + 3) >> 2;
    // ---- load (transposed into [t][c])
    for (int u = threadIdx.x; u < nq * nt4; u += NT) {
      const int tq = u % nt4, cq = u / nt4;
      const int tt = 4 * tq;
      const int nv = min(4, ws - tt);
      uint32_t w0 = 0, w1 = 0, w2 = 0, w3 = 0;
      const int c = 4 * cq;
      const uint8_t* a = src + (size_t)c * T + t0 + tt;
      if (c + 0 < C) w0 = load4_any(a, nv, blo, bhi);
      if (c + 1 < C) w1 = load4_any(a + T, nv, blo, bhi);
      if (c + 2 < C) w2 = load4_any(a + 2 * (size_t)T, nv, blo, bhi);
      if (c + 3 < C) w3 = load4_any(a + 3 * (size_t)T, nv, blo, bhi);
      transpose4x4(w0, w1, w2, w3);
      uint8_t* trow = L.tile + (size_t)tt * pitch + c;
      *reinterpret_cast<uint32_t*>(trow) = w0;
      if (nv > 1) *reinterpret_cast<uint32_t*>(trow + pitch) = w1;
      if (nv > 2) *reinterpret_cast<uint32_t*>(trow + 2 * pitch) = w2;
      if (nv > 3) *reinterpret_cast<uint32_t*>(trow + 3 * pitch) = w3;
    }
    for (int t = threadIdx.x; t < Ws; t += NT) L.V[t] = 0;
    for (int i = threadIdx.x; i < Ws * NB; i += NT) L.med[i] = 0xFFFFu;
    if (threadIdx.x == 0) *L.cnt = 0;
    __syncthreads();

    // ---- pass A: bin sums
    const int npairs = ws * NB;
    for (int p = threadIdx.x; p < npairs; p += NT) {
      const int t = p % ws, gi = p / ws;
      const unsigned gsz = gi == NB - 1 ? (unsigned)Gl : (unsigned)G;
      unsigned S, Q;
      bin_sums(L.tile + (size_t)t * pitch, gi * G, gsz, words, S, Q);
      L.Sg[t * NB + gi] = S;
      atomicAdd(&L.V[t], fd_contrib(gi == NB - 1 ? ml : mf, gsz, S, Q));
    }
    __syncthreads();

    for (int it = 0; it < cut.iterations; it++) {
      // ---- per-column keep half-widths
      for (int t = threadIdx.x; t < ws; t += NT) {
        const unsigned long long Vt = L.V[t];
        L.A[2 * t] = max_keep(Vt, (unsigned long long)C * mf * mf, 255u * (unsigned)G, cut.k2);
        L.A[2 * t + 1] = (Gl == G) ? L.A[2 * t]
                                   : max_keep(Vt, (unsigned long long)C * ml * ml, 255u * (unsigned)Gl, cut.k2);
      }
      __syncthreads();
      // ---- pass B: find bins with a byte outside their keep interval
      for (int p = threadIdx.x; p < npairs; p += NT) {
        const int t = p % ws, gi = p / ws;
        const bool lastbin = gi == NB - 1;
        const unsigned gsz = lastbin ? (unsigned)Gl : (unsigned)G;
        int lo, hi;
        fd_keep(L.Sg[t * NB + gi], L.A[2 * t + (lastbin ? 1 : 0)], gsz, lo, hi);
        bool any;
        if (lo == 0 && hi == 255) {
          any = false;
        } else if (words) {
          const ByteKeep kp = make_keep(lo, hi);
          const uint32_t* w = reinterpret_cast<const uint32_t*>(L.tile + (size_t)t * pitch + gi * G);
          const int nw = (gsz + 3) >> 2;
          uint32_t acc = 0;
          for (int i = 0; i < nw; i++) acc |= outside_fast(w[i], kp);
          any = (acc & 0x80808080u) != 0;
        } else {
          any = false;
          const uint8_t* rr = L.tile + (size_t)t * pitch + gi * G;
          for (unsigned i = 0; i < gsz; i++) any |= (rr[i] < lo) | (rr[i] > hi);
        }
        if (any) L.list[atomicAdd(L.cnt, 1u)] = (unsigned)p;
      }
      __syncthreads();
      const unsigned n = *L.cnt;
      // ---- flagged bins: exact flags, replacement, statistics update
      for (unsigned e = threadIdx.x; e < n; e += NT) {
        const int p = (int)L.list[e];
        const int t = p % ws, gi = p / ws;
        const bool lastbin = gi == NB - 1;
        const unsigned gsz = lastbin ? (unsigned)Gl : (unsigned)G;
        const unsigned S = L.Sg[t * NB + gi];
        int lo, hi;
        fd_keep(S, L.A[2 * t + (lastbin ? 1 : 0)], gsz, lo, hi);
        uint8_t* rr = L.tile + (size_t)t * pitch + gi * G;
        unsigned r;
        if (cut.replace == REP_MEDIAN) {
          unsigned m = L.med[t * NB + gi];
          if (m == 0xFFFFu) {
            m = bin_median(L.tile + (size_t)t * pitch, gi * G, gsz, words);
            L.med[t * NB + gi] = (uint16_t)m;
          }
          r = m;
        } else {
          r = (2 * S + gsz) / (2 * gsz);
        }
        unsigned s_old = 0, q_old = 0, s_new = 0, q_new = 0;
        const unsigned bit = 1u << (t0 + t - t_item);
        for (unsigned i = 0; i < gsz; i++) {
          const unsigned x = rr[i];
          s_old += x;
          q_old += x * x;
          unsigned y = x;
          if ((int)x < lo || (int)x > hi) {
            y = r;
            rr[i] = (uint8_t)r;
            atomicOr(&L.fmask[gi * G + i], bit);
          }
          s_new += y;
          q_new += y * y;
        }
        if (s_new != s_old || q_new != q_old) {
          const unsigned long long m = lastbin ? ml : mf;
          L.Sg[t * NB + gi] = s_new;
          atomicAdd(&L.V[t], fd_contrib(m, gsz, s_new, q_new) - fd_contrib(m, gsz, s_old, q_old));
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) *L.cnt = 0;
      // the next iteration's first __syncthreads orders this reset before pass B
    }
    __syncthreads();

    // ---- store the slab (transpose back to [c][t])
    for (int u = threadIdx.x; u < nq * nt4; u += NT) {
      const int tq = u % nt4, cq = u / nt4;
      const int tt = 4 * tq;
      const int nv = min(4, ws - tt);
      const uint8_t* trow = L.tile + (size_t)tt * pitch + 4 * cq;
      uint32_t w0 = *reinterpret_cast<const uint32_t*>(trow);
      uint32_t w1 = nv > 1 ? *reinterpret_cast<const uint32_t*>(trow + pitch) : 0u;
      uint32_t w2 = nv > 2 ? *reinterpret_cast<const uint32_t*>(trow + 2 * pitch) : 0u;
      uint32_t w3 = nv > 3 ? *reinterpret_cast<const uint32_t*>(trow + 3 * pitch) : 0u;
      transpose4x4(w0, w1, w2, w3);
      const int c = 4 * cq;
      uint8_t* a = dst + (size_t)c * T + t0 + tt;
      if (c + 0 < C) store4_any(a, w0, nv);
      if (c + 1 < C) store4_any(a + T, w1, nv);
      if (c + 2 < C) store4_any(a + 2 * (size_t)T, w2, nv);
      if (c + 3 < C) store4_any(a + 3 * (size_t)T, w3, nv);
    }
    __syncthreads();
  }

  // ---- flags
  const int nt = t_end - t_item;
  const unsigned valid = nt >= 32 ? 0xFFFFFFFFu : ((1u << nt) - 1u);
  if (P.mask_kind == MASK_BITS && J.mask) {
    const int W32 = (T + 31) >> 5;
    unsigned* mb = static_cast<unsigned*>(J.mask) + item;
    for (int c = threadIdx.x; c < C; c += NT) {
      const unsigned f = L.fmask[c] & valid;
      unsigned* wp = mb + (size_t)c * W32;
      if (P.mask_or) {
        if (f) *wp = __ldcg(wp) | f;
      } else {
        *wp = f;
      }
    }
  } else if (P.mask_kind == MASK_BYTES && J.mask) {
    uint8_t* mb = static_cast<uint8_t*>(J.mask);
    for (int u = threadIdx.x; u < C * nt; u += NT) {
      const int c = u / nt, t = u % nt;
      const unsigned f = (L.fmask[c] >> t) & 1u;
      uint8_t* bp = mb + (size_t)c * T + t_item + t;
      if (P.mask_or) {
        if (f) *bp = (uint8_t)(__ldcg(bp) | 2u);
      } else {
        *bp = (uint8_t)(f ? 2u : 0u);
      }
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// persistent engine
// ---------------------------------------------------------------------------
__device__ bool wait_rows(const Params& P, int job, unsigned need, int* bc) {
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
    bc[3] = good;
  }
  __syncthreads();
  const bool ok = bc[3] != 0;
  __syncthreads();
  return ok;
}

template <int NCH>
__global__ void __launch_bounds__(NT) k_engine_u8(const __grid_constant__ Params P) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long red64[2 * (NT / 32)];
  __shared__ unsigned red32[4 * (NT / 32)];
  __shared__ int bc[4];
  __shared__ int s_item;
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
      tdsc_row_u8<NCH>(P, J, idx, smem, red64, red32, bc);
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        if (sg.job != P.withhold_job) atomicAdd(P.counters + 1 + sg.job, 1u);
      }
    } else {
      if (P.wait_tdsc && !wait_rows(P, sg.job, (unsigned)J.rows, bc)) continue;
      fdsc_item_u8(P, J, idx, smem);
    }
  }
}

// ---------------------------------------------------------------------------
// host-side helpers for this translation unit
// ---------------------------------------------------------------------------
int engine_nch_for(int max_T) {
  const int nch = (max_T + 30) / 16 + 1;  // worst-case head offset of 15
  const int per = (nch + NT - 1) / NT;
  if (per <= 1) return 1;
  if (per <= 2) return 2;
  if (per <= 4) return 4;
  if (per <= 8) return 8;
  if (per <= 16) return 16;
  return -1;
}

int engine_smem_u8(const Params& p, int nch) {
  int s = nch * NT * 2 + 16;  // TDSC: per-chunk flag bits
  for (int j = 0; j < p.n_jobs; j++) {
    const Job& J = p.jobs[j];
    if (p.fd.iterations > 0) s = s > fd_smem_bytes(J.ws, J.pitch, J.nb, J.C) ? s : fd_smem_bytes(J.ws, J.pitch, J.nb, J.C);
  }
  return align16i(s);
}

void* engine_kernel_u8(int nch) {
  switch (nch) {
    case 1: return (void*)k_engine_u8<1>;
    case 2: return (void*)k_engine_u8<2>;
    case 4: return (void*)k_engine_u8<4>;
    case 8: return (void*)k_engine_u8<8>;
    case 16: return (void*)k_engine_u8<16>;
  }
  return nullptr;
}

int launch_engine_u8(const Params& p, const LaunchCfg& cfg, void* stream) {
  void* fn = engine_kernel_u8(cfg.nch);
  if (!fn) return (int)cudaErrorInvalidValue;
  void* args[] = {const_cast<Params*>(&p)};
  return (int)cudaLaunchKernel(fn, dim3(cfg.grid), dim3(NT), args, (size_t)cfg.smem, (cudaStream_t)stream);
}

}  // namespace rfim
