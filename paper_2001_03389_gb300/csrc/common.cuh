// common.cuh -- device helpers shared by the sigma-cut kernels (sm_103a).
//
// Exact uint8 decisions.  The library decides a uint8 flag as
//     (double)lhs > fl(k2 * (double)R)
// with lhs, R exact integers below 2^53 and k2 = fl(k*k) a double (TDSC:
// lhs = (T x - S)^2, R = T Q - S^2; FDSC: lhs = C D^2, R = sum D^2).  The right
// side is evaluated as written, one IEEE double multiply per row or column and
// iteration, and turned into the integer floor(fl(k2 R)): for integers lhs,
// lhs > fl(k2 R) iff lhs > floor(fl(k2 R)), so every per-candidate test is a
// 64-bit integer comparison.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace rfim {

constexpr int NT = 256;  // threads per CTA in every kernel of the engine

// The squared threshold of a cut.  Built on the host.
struct ExactK2 {
  double k2;  // fl(k * k)
  float k2f;  // k2 rounded to float, for first guesses only
};

// floor(fl(k2 * R)) for an integer R < 2^53, saturated at 2^62 (beyond every
// left side, which stays below 2^53).
__device__ __forceinline__ unsigned long long thr_floor(unsigned long long R, const ExactK2& k) {
  const double t = __dmul_rn(k.k2, __ull2double_rn(R));
  return t < 4.0e18 ? __double2ull_rz(t) : (1ull << 62);
}

// ---------------------------------------------------------------------------
// SIMD-within-a-word helpers on 4 packed bytes.
// ---------------------------------------------------------------------------

// per-byte |a - b| (PTX vabsdiff4, a native instruction on sm_103a)
__device__ __forceinline__ uint32_t absdiff4(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("vabsdiff4.u32.u32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(0u));
  return d;
}

// acc + sum over bytes |a_i - b_i|
__device__ __forceinline__ uint32_t sad4(uint32_t a, uint32_t b, uint32_t acc) {
  uint32_t d;
  asm("vabsdiff4.u32.u32.u32.add %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(acc));
  return d;
}

__device__ __forceinline__ uint32_t dp4a_u(uint32_t a, uint32_t b, uint32_t c) {
  return (uint32_t)__dp4a(a, b, c);  // unsigned bytes: __dp4a(unsigned, unsigned, unsigned)
}

// Keep-interval test on bytes.  A byte x is kept iff lo <= x <= hi.
//   m = lo + floor((hi - lo) / 2), h = floor((hi - lo) / 2) (h <= 127):
//   |x - m| > h  covers x < lo and x > hi, and also x == hi when hi - lo is odd,
//   so the exact test additionally clears bytes equal to hi in that case.
struct ByteKeep {
  uint32_t m4;   // m in every byte
  uint32_t k4;   // (127 - h) in every byte
  uint32_t hi4;  // hi in every byte
  uint32_t all;  // 0x80808080 when the keep interval is empty (everything flagged)
  bool odd;      // hi - lo odd
};

// byte 0 of v replicated into all four bytes
__device__ __forceinline__ uint32_t splat4(uint32_t v) { return __byte_perm(v, 0u, 0u); }

__device__ __forceinline__ ByteKeep make_keep(int lo, int hi) {
  ByteKeep k;
  if (lo > hi) {
    k.m4 = 0;
    k.k4 = 0;
    k.hi4 = 0;
    k.all = 0x80808080u;
    k.odd = false;
    return k;
  }
  const int h = (hi - lo) >> 1;
  k.m4 = splat4((uint32_t)(lo + h));
  k.k4 = splat4((uint32_t)(127 - h));
  k.hi4 = splat4((uint32_t)hi);
  k.all = 0;
  k.odd = ((hi - lo) & 1) != 0;
  return k;
}

// floor(n / d) for d >= 1 and quotients below 2^20 (every quotient here is a
// byte value or a few hundred): a float-reciprocal estimate, corrected exactly.
__device__ __forceinline__ unsigned udiv_q(unsigned n, unsigned d, float rcp) {
  unsigned q = __float2uint_rz(__uint2float_rz(n) * rcp);
  while (q * d > n) q--;
  while ((q + 1) * d <= n) q++;
  return q;
}

// bit 7 of each byte set iff that byte is outside [lo, hi] (exact)
__device__ __forceinline__ uint32_t outside_exact(uint32_t x, const ByteKeep& k) {
  const uint32_t d = absdiff4(x, k.m4);
  uint32_t g = ((d & 0x7F7F7F7Fu) + k.k4) | d;  // bit 7: d > h, per byte exactly
  if (k.odd) {
    const uint32_t e = x ^ k.hi4;
    g &= ((e & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | e;  // bit 7: x != hi
  }
  return (g & 0x80808080u) | k.all;
}

// superset test: bit 7 set for every byte outside [lo, hi], possibly also for x == hi
__device__ __forceinline__ uint32_t outside_fast(uint32_t x, const ByteKeep& k) {
  const uint32_t d = absdiff4(x, k.m4);
  return (((d & 0x7F7F7F7Fu) + k.k4) | d | k.all);
}

// 0x80 per byte -> 0xFF per byte
__device__ __forceinline__ uint32_t widen80(uint32_t f) { return f | (f - (f >> 7)); }

// 4 low bits -> 0x01 per selected byte
__device__ __forceinline__ uint32_t bytes_from_bits4(uint32_t n) { return ((n & 0xFu) * 0x00204081u) & 0x01010101u; }

// Byte-mask words of a 16-byte chunk keeping bytes with index in [lo, hi)
__device__ __forceinline__ uint4 chunk_keep_mask(int lo, int hi) {
  const uint32_t vb = (hi >= 16 ? 0xFFFFu : ((1u << hi) - 1u)) & ~((1u << lo) - 1u);
  uint4 m;
  m.x = bytes_from_bits4(vb) * 0xFFu;
  m.y = bytes_from_bits4(vb >> 4) * 0xFFu;
  m.z = bytes_from_bits4(vb >> 8) * 0xFFu;
  m.w = bytes_from_bits4(vb >> 12) * 0xFFu;
  return m;
}

// 4x4 byte transpose: rows r0..r3 (byte j of r_i is element (i, j)) -> columns.
__device__ __forceinline__ void transpose4x4(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  const uint32_t t0 = __byte_perm(r0, r1, 0x5140);
  const uint32_t t1 = __byte_perm(r0, r1, 0x7362);
  const uint32_t t2 = __byte_perm(r2, r3, 0x5140);
  const uint32_t t3 = __byte_perm(r2, r3, 0x7362);
  r0 = __byte_perm(t0, t2, 0x5410);
  r1 = __byte_perm(t0, t2, 0x7632);
  r2 = __byte_perm(t1, t3, 0x5410);
  r3 = __byte_perm(t1, t3, 0x7632);
}

// ---------------------------------------------------------------------------
// Reductions over the CTA (NT threads).  `scratch` holds NT/32 * N words.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------------------
// Random replacement draws: the SplitMix64 output function (Steele, Lea,
// Flood, "Fast splittable pseudorandom number generators", 2014) of a key
// built from (beam, line, index, method, iteration, attempt).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// key of a (beam, line): mix64(mix64(beam) ^ line)
__device__ __forceinline__ unsigned long long draw_key(int beam, int line) {
  return mix64(mix64((unsigned long long)beam) ^ (unsigned long long)line);
}

// position in [0, n) of attempt a (method 1 = TDSC, 2 = FDSC)
__device__ __forceinline__ unsigned draw_pos(unsigned long long key, int index, int method, int it, int a,
                                             unsigned n) {
  const unsigned long long h = mix64(mix64(key ^ (unsigned long long)index) ^
                                     ((unsigned long long)method << 8 | (unsigned long long)it << 16 |
                                      (unsigned long long)a << 24));
  return (unsigned)(((h >> 32) * (unsigned long long)n) >> 32);
}

constexpr int DRAW_ATTEMPTS = 32;

// ---------------------------------------------------------------------------
// TMA 1-D bulk copies (global -> shared) completing on an mbarrier
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// makes initialised mbarriers visible to the asynchronous (TMA) proxy
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// orders this thread's earlier shared-memory accesses before later TMA writes
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// the single arrival of a phase, announcing `bytes` of copies to complete on it
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// bytes (a multiple of 16; both addresses 16-byte aligned) from global src to shared dst
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Wait for the phase of `parity` to complete, giving up after limit_ns (false).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity,
                                                  unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  while (!mbar_try_wait(bar, parity))
    if (globaltimer_ns() - t0 > limit_ns) return false;
  return true;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

}  // namespace rfim
