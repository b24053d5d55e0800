// api.cu -- the C ABI of librfim.so: context, validation, work-queue planning,
// launches, CUDA-graph batching and host-buffer cleaning.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/rfim.h"
#include "engine.h"
#include "runtime.h"

using namespace rfim;

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
namespace {

constexpr int COUNTER_BLOCKS = 256;
constexpr int COUNTER_STRIDE = 2 + MAX_JOBS;  // head + per-job done counters (+ pad)

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  std::vector<unsigned char> key;
};

}  // namespace

struct rfim_ctx {
  int device = 0;
  int sms = 0;
  size_t hbm_budget = 0;
  std::string tune_cache;
  std::string last_error;
  unsigned* d_counters = nullptr;  // COUNTER_BLOCKS x COUNTER_STRIDE
  unsigned* d_status = nullptr;
  unsigned seq = 0;
  // options
  long long spin_limit_us = 2000000;
  int schedule = 0;
  int tile_samples = 0;
  int ctas_per_sm = 0;
  int withhold = 0;
  int smem_target = 113 * 1024;
  int fused_lag = 1;
  int order = 0;  // 0 = blocked (all TDSC iterations, then FDSC), 1 = interleaved rounds
  int f32_records = 0;  // float32 fused launches: TDSC records its cuts and FDSC replays them
  long long stage_group_bytes = 32ll << 20;  // rfim_clean_host: bytes per staged group
  // test hook: allocations left before every later one fails (-1 = off)
  long long fail_alloc_after = -1;
  int stage_streams = 3;                     // rfim_clean_host: streams in the staging ring
  // graphs for rfim_clean_batch (each with its own counter blocks)
  std::map<std::vector<unsigned char>, std::pair<cudaGraphExec_t, unsigned*>> graphs;
  unsigned* capture_counters = nullptr;  // while capturing: counter blocks of the graph
  int capture_used = 0;
  cudaStream_t capture_stream = nullptr;
  // BTC blocks: BCT scratch copies of the data and the mask
  void* btc_buf = nullptr;
  size_t btc_cap = 0;
  void* btc_mask = nullptr;
  size_t btc_mask_cap = 0;
  // host staging (rfim_clean_host)
  HostStager* stager = nullptr;
  // streaming service
  StreamService* stream = nullptr;
  // autotuner
  Tuner* tuner = nullptr;
  // float32 fused launches: per-row TDSC cuts that FDSC items replay (grow-only;
  // outgrown buffers stay allocated until destroy, as captured graphs hold them)
  float* prog = nullptr;
  size_t prog_cap = 0;
  std::vector<float*> prog_retired;
  std::mutex mu;
};

namespace {

rfim_status fail(rfim_ctx* ctx, rfim_status s, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ctx->last_error = buf;
  }
  return s;
}

// A failed runtime call (a launch with a bad configuration, say) also leaves
// its error as the thread's last CUDA error, which the caller's next CUDA
// call would report; errors that do not corrupt the context are cleared here
// and returned as a status only.
rfim_status clear_cuda_error() {
  (void)cudaGetLastError();
  return RFIM_ERR_CUDA;
}

rfim_status cuda_fail(rfim_ctx* ctx, cudaError_t e, const char* what) {
  clear_cuda_error();
  return fail(ctx, RFIM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

ExactK2 make_k2(double k) {
  ExactK2 r;
  r.k2 = k * k;  // fl(k * k): one IEEE rounding
  r.k2f = (float)r.k2;
  return r;
}

long long gcdll(long long a, long long b) {
  while (b) {
    long long t = a % b;
    a = b;
    b = t;
  }
  return a;
}

size_t dtype_size(rfim_dtype d) { return d == RFIM_F32 ? 4 : 1; }

struct CutNorm {
  bool on = false;
  double k = 0;
  int it = 0;
  int rep = 0;
  int bin = 0;
};

rfim_status check_cut(rfim_ctx* ctx, const rfim_cut* c, int C, bool fdsc, CutNorm& out) {
  out = CutNorm();
  if (!c) return RFIM_OK;
  if (!std::isfinite(c->k) || !(c->k > 0.0)) return fail(ctx, RFIM_ERR_ARG, "k must be finite and > 0, got %g", c->k);
  if (c->iterations < 1 || c->iterations > 16)
    return fail(ctx, RFIM_ERR_ARG, "iterations must be in 1..16, got %d", c->iterations);
  if (c->replace != RFIM_REPLACE_MEAN && c->replace != RFIM_REPLACE_MEDIAN && c->replace != RFIM_REPLACE_RANDOM)
    return fail(ctx, RFIM_ERR_ARG, "unknown replacement strategy %d", (int)c->replace);
  int bin = c->fdsc_bin;
  if (fdsc) {
    if (bin == 0) bin = std::min(32, C);
    if (bin < 1 || bin > C) return fail(ctx, RFIM_ERR_ARG, "fdsc_bin must be in 1..channels (%d), got %d", C, bin);
  }
  out.on = true;
  out.k = c->k;
  out.it = c->iterations;
  out.rep = (int)c->replace;
  out.bin = bin;
  return RFIM_OK;
}

bool ranges_overlap(const void* a, size_t na, const void* b, size_t nb) {
  const char* pa = (const char*)a;
  const char* pb = (const char*)b;
  return pa < pb + nb && pb < pa + na;
}

const long long LIM53 = (1LL << 53) / 65025;  // (255 n)^2 style bounds: n^2 <= LIM53

rfim_status check_block(rfim_ctx* ctx, const rfim_block* b, const CutNorm& td, const CutNorm& fd) {
  if (!b) return fail(ctx, RFIM_ERR_ARG, "null block");
  if (!b->in || !b->out) return fail(ctx, RFIM_ERR_ARG, "null in/out pointer");
  if (b->beams < 1 || b->channels < 1 || b->samples < 1)
    return fail(ctx, RFIM_ERR_ARG, "beams, channels, samples must be >= 1 (%d, %d, %d)", b->beams, b->channels,
                b->samples);
  if (b->dtype != RFIM_U8 && b->dtype != RFIM_F32) return fail(ctx, RFIM_ERR_ARG, "unknown dtype %d", (int)b->dtype);
  if (b->layout != RFIM_LAYOUT_BCT && b->layout != RFIM_LAYOUT_BTC)
    return fail(ctx, RFIM_ERR_ARG, "unknown layout %d", (int)b->layout);
  if (b->mask_fmt != RFIM_MASK_NONE && b->mask_fmt != RFIM_MASK_BITS && b->mask_fmt != RFIM_MASK_BYTES)
    return fail(ctx, RFIM_ERR_ARG, "unknown mask format %d", (int)b->mask_fmt);
  if (b->mask_fmt != RFIM_MASK_NONE && !b->mask) return fail(ctx, RFIM_ERR_ARG, "mask format set but mask is null");
  if (b->mask_fmt == RFIM_MASK_BITS && ((uintptr_t)b->mask & 3))
    return fail(ctx, RFIM_ERR_ARG, "bit mask pointer must be 4-byte aligned");
  if (b->dtype == RFIM_F32 && (((uintptr_t)b->in & 3) || ((uintptr_t)b->out & 3)))
    return fail(ctx, RFIM_ERR_ARG, "float32 buffers must be 4-byte aligned");
  const size_t N = (size_t)b->beams * b->channels * b->samples;
  const size_t bytes = N * dtype_size(b->dtype);
  if (b->out != b->in && ranges_overlap(b->in, bytes, b->out, bytes))
    return fail(ctx, RFIM_ERR_ARG, "out overlaps in without being equal to it");
  if (b->mask_fmt != RFIM_MASK_NONE) {
    const size_t slow = b->layout == RFIM_LAYOUT_BCT ? (size_t)b->beams * b->channels : (size_t)b->beams * b->samples;
    const size_t fast = b->layout == RFIM_LAYOUT_BCT ? (size_t)b->samples : (size_t)b->channels;
    const size_t mbytes = b->mask_fmt == RFIM_MASK_BITS ? slow * ((fast + 31) / 32) * 4 : N;
    if (ranges_overlap(b->mask, mbytes, b->in, bytes) || ranges_overlap(b->mask, mbytes, b->out, bytes))
      return fail(ctx, RFIM_ERR_ARG, "mask overlaps the data");
  }
  if (b->dtype == RFIM_U8) {
    if (td.on && (long long)b->samples * b->samples > LIM53)
      return fail(ctx, RFIM_ERR_RANGE, "TDSC uint8: (255*T)^2 must stay below 2^53 (T <= 372181), T = %d", b->samples);
    if (fd.on) {
      const int C = b->channels, G = fd.bin;
      const int nb = (C + G - 1) / G, gl = C - (nb - 1) * G;
      const long long L = (long long)G / gcdll(G, gl) * gl;
      if (L > 372181 || L * L > LIM53 / C)
        return fail(ctx, RFIM_ERR_RANGE, "FDSC uint8: C * (255 * lcm(bin sizes))^2 must stay below 2^53");
    }
  }
  return RFIM_OK;
}

// Engine limits (shapes the kernels do not take).
rfim_status check_impl(rfim_ctx* ctx, const rfim_block* b, const CutNorm& td, const CutNorm& fd) {
  if (b->layout != RFIM_LAYOUT_BCT)
    return fail(ctx, RFIM_ERR_ARG, "BTC blocks are cleaned through a context's BCT scratch (not here)");
  if (b->dtype == RFIM_F32) {
    if (td.on && td.rep == RFIM_REPLACE_RANDOM && b->samples > TD32_MAX_T &&
        td32_rnd_long_bytes(b->samples) > MAX_SMEM_PER_CTA)
      return fail(ctx, RFIM_ERR_ARG, "float32 TDSC with random replacement: rows longer than %d samples are not "
                  "supported", (MAX_SMEM_PER_CTA / 8) * 32);
    if (fd.on) {
      // the tile of one sample, else the column-at-a-time layout, must fit a CTA's shared memory
      const int C = b->channels, nb = (C + fd.bin - 1) / fd.bin;
      if (fd32_smem_bytes(1, C, nb, fd.rep == RFIM_REPLACE_RANDOM) > MAX_SMEM_PER_CTA &&
          fd_wide_smem_f32(C, nb) > MAX_SMEM_PER_CTA)
        return fail(ctx, RFIM_ERR_RANGE, "FDSC: a column of %d float32 channels does not fit shared memory", C);
    }
    return RFIM_OK;
  }
  if (td.on && td_row_mode(b->samples) < 0)
    return fail(ctx, RFIM_ERR_RANGE, "TDSC rows longer than %lld samples are not available", TD_MAX_T);
  if (td.on && td.rep == RFIM_REPLACE_RANDOM && td_random_row_mode(b->samples) < 0)
    return fail(ctx, RFIM_ERR_ARG, "uint8 TDSC with random replacement: the row's flag bitmaps do not fit");
  if (fd.on) {
    // the smallest FDSC tile (8 samples x all channels), else the column-at-a-time
    // layout, must fit one CTA's shared memory
    const int C = b->channels, nb = (C + fd.bin - 1) / fd.bin;
    if (fd_smem_bytes(8, fd_pitch(C), nb, C, fd.rep == RFIM_REPLACE_RANDOM, fd.bin) > MAX_SMEM_PER_CTA &&
        fd_wide_smem_u8(C, nb) > MAX_SMEM_PER_CTA)
      return fail(ctx, RFIM_ERR_RANGE, "FDSC: a column of %d channels does not fit shared memory", C);
  }
  return RFIM_OK;
}

struct Plan {
  std::vector<Job> jobs;
  CutNorm td, fd;
  int mask_kind = 0;
  int max_T = 1;
  rfim_dtype dtype = RFIM_U8;
  bool prog = false;  // the jobs carry TDSC cut records (float32; used by fused launches only)
};

int pick_ws_opt(int tile_samples, int C, int nb, int pitch, int budget, bool rnd, int bin) {
  if (tile_samples > 0) return tile_samples < 8 ? 8 : tile_samples;  // uint8 tiles are 8, 16 or 32 wide
  for (int ws : {32, 16, 8})
    if (fd_smem_bytes(ws, pitch, nb, C, rnd, bin) <= budget) return ws;
  return 8;
}

// Work-queue description of beam j of block b.
Job make_job(const rfim_block* b, int j, const CutNorm& fd, int tile_samples, int smem_target) {
  const int C = b->channels, T = b->samples;
  const size_t es = dtype_size(b->dtype);
  const size_t beam = (size_t)C * T;
  const int W32 = (T + 31) / 32;
  Job J;
  memset(&J, 0, sizeof J);
  J.in = (const char*)b->in + j * beam * es;
  J.out = (char*)b->out + j * beam * es;
  if (b->mask_fmt == RFIM_MASK_BITS)
    J.mask = (unsigned*)b->mask + (size_t)j * C * W32;
  else if (b->mask_fmt == RFIM_MASK_BYTES)
    J.mask = (unsigned char*)b->mask + j * beam;
  else
    J.mask = nullptr;
  J.src_lo = J.in;
  J.src_hi = (const char*)J.in + beam * es;
  J.beam = j;
  J.C = C;
  J.T = T;
  J.rows = C;
  const int G = fd.on ? fd.bin : std::min(32, C);
  J.nb = (C + G - 1) / G;
  J.last_g = C - (J.nb - 1) * G;
  const long long L = (long long)G / gcdll(G, J.last_g) * J.last_g;
  J.m_full = (unsigned long long)(L / G);
  J.m_last = (unsigned long long)(L / J.last_g);
  J.pitch = fd_pitch(C * (int)es);
  J.ws = pick_ws_opt(tile_samples, C, J.nb, J.pitch, smem_target, fd.on && fd.rep == RFIM_REPLACE_RANDOM, G);
  J.fd_items = (T + FD_ITEM_T - 1) / FD_ITEM_T;
  const int tm = td_row_mode(T);  // (-1 only with TDSC off: no TDSC items then)
  J.td_mode = tm < 0 ? 1 : tm;
  J.td_items = J.td_mode == 0   ? (C + TD_ROWS_PER_ITEM - 1) / TD_ROWS_PER_ITEM
               : J.td_mode == 3 ? (C + 4 * TD_ROWS_PER_ITEM - 1) / (4 * TD_ROWS_PER_ITEM)
                                : C;
  if (b->dtype == RFIM_F32) {
    // float32: one CTA per TDSC row; FDSC sub-slab of 8, 4, 2 or 1 samples
    // TDSC: two rows per item (a half CTA each) when both stages fit, else one
    J.td_mode = 2 * td32_smem_bytes(T) <= MAX_SMEM_PER_CTA ? 0 : T <= TD32_MAX_T ? 1 : 2;
    J.td_items = J.td_mode == 0 ? (C + 1) / 2 : C;
    J.ws = 1;
    for (int ws : {8, 4, 2})
      if ((tile_samples == 0 || ws <= tile_samples) && fd32_smem_bytes(ws, C, J.nb, fd.on && fd.rep == RFIM_REPLACE_RANDOM) <= smem_target) {
        J.ws = ws;
        break;
      }
    J.fd_items = (T + J.ws - 1) / J.ws;
    if (fd.on && fd32_smem_bytes(1, C, J.nb, fd.rep == RFIM_REPLACE_RANDOM) > MAX_SMEM_PER_CTA) {
      J.fd_wide = 1;  // columns one at a time, 32 samples per item
      J.fd_items = (T + FD_ITEM_T - 1) / FD_ITEM_T;
    }
  } else if (fd.on && fd_smem_bytes(8, J.pitch, J.nb, C, fd.rep == RFIM_REPLACE_RANDOM, G) > MAX_SMEM_PER_CTA) {
    J.fd_wide = 1;  // columns one at a time
  }
  return J;
}

// uint8 TDSC with random replacement: warp or CTA rows by the stage the flags need
void random_row_mode(Job& J, const rfim_block* b, const CutNorm& td) {
  if (b->dtype != RFIM_U8 || !td.on || td.rep != RFIM_REPLACE_RANDOM) return;
  const int m = td_random_row_mode(b->samples);
  J.td_mode = m < 0 ? 0 : m;  // (-1 is refused by check_impl)
  J.td_items = J.td_mode == 0 ? (b->channels + TD_ROWS_PER_ITEM - 1) / TD_ROWS_PER_ITEM : b->channels;
}

void add_block_jobs(rfim_ctx* ctx, Plan& pl, const rfim_block* b) {
  for (int j = 0; j < b->beams; j++) {
    pl.jobs.push_back(make_job(b, j, pl.fd, ctx->tile_samples, ctx->smem_target));
    random_row_mode(pl.jobs.back(), b, pl.td);
    pl.max_T = std::max(pl.max_T, b->samples);
  }
}

// The k the kernels use: clamped to [K_MIN_U8 (uint8 only), K_MAX], which
// changes no decision.
//  - Above: |x - mu| <= sigma sqrt(n - 1) for every sample of n values, so no
//    cut with k > sqrt(n - 1) flags anything; n < 2^31 gives sqrt(n) < 46341,
//    and k = 1e6 flags nothing too.  (The clamp keeps k^2 and the float-float
//    split of k finite.)
//  - Below, uint8: the threshold fl(k2 R) has R < 2^53 (validated), so for
//    k <= 1e-9 it is below 1 and, the left side being an integer, every such
//    k flags exactly the samples with a nonzero left side.
// float32 takes k unclamped below: there the threshold is k sigma itself.
constexpr double K_MAX = 1e6, K_MIN_U8 = 1e-9;

CutDev cut_dev(const CutNorm& c, rfim_dtype dt) {
  CutDev d;
  memset(&d, 0, sizeof d);
  if (c.on) {
    double k = std::min(c.k, K_MAX);
    if (dt == RFIM_U8) k = std::max(k, K_MIN_U8);
    d.k2 = make_k2(k);
    d.k = k;
    d.k_hi = (float)k;
    d.k_lo = (float)(k - (double)d.k_hi);
    d.iterations = c.it;
    d.replace = c.rep;
    d.bin = c.bin;
  }
  return d;
}

// Queue segments of p's jobs.  mode: 0 = TDSC only, 1/3 = FDSC only, 2 = fused
// (TDSC rows of beam j + lag queued before the FDSC items of beam j).
void fill_segments(Params& p, int mode, int lag) {
  int n = 0, s = 0;
  auto push = [&](int job, int kind, int count) {
    if (count <= 0) return;
    p.segs[s].start = n;
    p.segs[s].job = job;
    p.segs[s].kind = kind;
    s++;
    n += count;
  };
  const int nj = p.n_jobs;
  if (mode == 0) {
    for (int j = 0; j < nj; j++) push(j, 0, p.jobs[j].td_items);
  } else if (mode == 1 || mode == 3) {
    for (int j = 0; j < nj; j++) push(j, 1, p.jobs[j].fd_items);
  } else {
    lag = std::max(0, lag);
    for (int j = 0; j < nj + lag; j++) {
      if (j < nj) push(j, 0, p.jobs[j].td_items);
      const int f = j - lag;
      if (f >= 0) push(f, 1, p.jobs[f].fd_items);
    }
  }
  p.n_segs = s;
  p.n_items = n;
}

struct OccKey {
  void* fn;
  int smem;
  bool operator<(const OccKey& o) const { return fn < o.fn || (fn == o.fn && smem < o.smem); }
};

int occupancy(void* fn, int smem) {
  static std::mutex m;
  static std::map<OccKey, int> cache;
  std::lock_guard<std::mutex> g(m);
  OccKey k{fn, smem};
  auto it = cache.find(k);
  if (it != cache.end()) return it->second;
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_SMEM_PER_CTA);
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, NT, smem) != cudaSuccess) n = 1;
  if (n < 1) n = 1;
  cache[k] = n;
  return n;
}

// Build the Params of one launch over jobs [j0, j1) with the given item kinds.
// mode: 0 = TDSC only, 1 = FDSC only (reads `in`), 2 = fused TDSC->FDSC, 3 = FDSC reading `out`,
// 5 = TDSC on `out` in place, OR-ing its flags into the mask (interleaved rounds).
// The automatic schedule: one fused launch, except when every TDSC row of the
// launch takes a quarter warp (rows of at most TD_QUAD_CHUNKS chunks, as in
// streaming chunks).  There two launches, TDSC then FDSC, measured 6 % faster
// (1536 x 1250 uint8 chunks); on longer rows the fused launch is faster.
bool separate_by_default(const Job* jobs, int n, int dtype) {
  if (dtype != RFIM_U8 || n < 1) return false;
  for (int j = 0; j < n; j++)
    if (jobs[j].td_mode != 3) return false;
  return true;
}

void fill_params(rfim_ctx* ctx, const Plan& pl, int j0, int j1, int mode, Params& p, unsigned* counters) {
  memset(&p, 0, sizeof p);
  p.n_jobs = j1 - j0;
  for (int j = j0; j < j1; j++) p.jobs[j - j0] = pl.jobs[j];
  p.td = cut_dev(pl.td, pl.dtype);
  p.fd = cut_dev(pl.fd, pl.dtype);
  if (mode == 1 || mode == 3) p.td.iterations = 0;
  if (mode == 0 || mode == 5) p.fd.iterations = 0;
  if (mode == 5) {
    for (int j = 0; j < p.n_jobs; j++) {
      Job& J = p.jobs[j];
      const size_t beam = (size_t)J.C * J.T * (pl.dtype == RFIM_F32 ? 4 : 1);
      J.in = J.out;
      J.src_lo = J.out;
      J.src_hi = (const char*)J.out + beam;
    }
    p.td_mask_or = 1;
  }
  if (!(pl.prog && mode == 2))
    for (int j = 0; j < p.n_jobs; j++) p.jobs[j].prog = nullptr;
  p.mask_kind = pl.mask_kind;
  // fused float32 with cut records: FDSC reads the input and replays TDSC's cuts
  p.fd_reads_out = (mode == 2 && !(pl.prog && p.n_jobs > 0)) || mode == 3 ? 1 : 0;
  p.wait_tdsc = mode == 2 ? 1 : 0;
  p.mask_or = (mode == 2 || mode == 3) ? 1 : 0;
  p.withhold_job = (ctx->withhold && mode == 2) ? 0 : -1;
  p.spin_limit_ns = (unsigned long long)ctx->spin_limit_us * 1000ull;
  p.counters = counters;
  p.status = ctx->d_status;
  p.dtype = pl.dtype == RFIM_F32 ? 1 : 0;
  fill_segments(p, mode == 5 ? 0 : mode, ctx->fused_lag);
}

// float32 FDSC items OR their bits into the mask words they share: a launch
// whose TDSC part did not write the mask first starts from zeroed bit masks.
cudaError_t clear_f32_fdsc_masks(const Params& p, cudaStream_t st) {
  if (p.dtype != 1 || p.fd.iterations == 0 || p.mask_or || p.mask_kind != MASK_BITS) return cudaSuccess;
  for (int j = 0; j < p.n_jobs; j++) {
    const Job& J = p.jobs[j];
    if (!J.mask) continue;
    const size_t bytes = (size_t)J.C * ((J.T + 31) / 32) * 4;
    cudaError_t e = cudaMemsetAsync(J.mask, 0, bytes, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

rfim_status launch_one(rfim_ctx* ctx, Params& p, int max_T, cudaStream_t st) {
  (void)max_T;
  LaunchCfg cfg;
  cfg.smem = engine_smem(p);
  if (cfg.smem > MAX_SMEM_PER_CTA) return fail(ctx, RFIM_ERR_ARG, "tile does not fit in shared memory (%d bytes)", cfg.smem);
  void* fn = engine_kernel(p);
  int per_sm = occupancy(fn, cfg.smem);
  if (ctx->ctas_per_sm > 0) per_sm = std::min(per_sm, ctx->ctas_per_sm);
  cfg.grid = std::max(1, std::min(p.n_items, ctx->sms * per_sm));
  cudaError_t e = cudaMemsetAsync(p.counters, 0, sizeof(unsigned) * (1 + p.n_jobs), st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemsetAsync");
  if ((e = clear_f32_fdsc_masks(p, st)) != cudaSuccess) return cuda_fail(ctx, e, "cudaMemsetAsync");
  e = (cudaError_t)launch_engine(p, cfg, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "engine launch");
  return RFIM_OK;
}

unsigned* next_counters(rfim_ctx* ctx) {
  if (ctx->capture_counters) return ctx->capture_counters + (size_t)(ctx->capture_used++) * COUNTER_STRIDE;
  const unsigned b = ctx->seq++ % COUNTER_BLOCKS;
  return ctx->d_counters + (size_t)b * COUNTER_STRIDE;
}

// Run a plan: mode as in fill_params; fused may fall back to two launches.
rfim_status run_plan(rfim_ctx* ctx, const Plan& pl, cudaStream_t st) {
  const int nj = (int)pl.jobs.size();
  static thread_local Params p;  // ~20 KB: keep off the stack
  for (int j0 = 0; j0 < nj; j0 += MAX_JOBS) {
    const int j1 = std::min(nj, j0 + MAX_JOBS);
    rfim_status s;
    if (pl.td.on && pl.fd.on && ctx->order == 1) {
      // interleaved: round r = TDSC iteration r on every row, then FDSC iteration r on every column
      const int rounds = std::max(pl.td.it, pl.fd.it);
      for (int r = 0; r < rounds; r++) {
        if (r < pl.td.it) {
          fill_params(ctx, pl, j0, j1, r == 0 ? 0 : 5, p, next_counters(ctx));
          p.td.iterations = 1;
          p.td.it0 = r;  // round r is iteration r: its random draws are keyed by r
          if ((s = launch_one(ctx, p, pl.max_T, st)) != RFIM_OK) return s;
        }
        if (r < pl.fd.it) {
          fill_params(ctx, pl, j0, j1, 3, p, next_counters(ctx));
          p.fd.iterations = 1;
          p.fd.it0 = r;
          if ((s = launch_one(ctx, p, pl.max_T, st)) != RFIM_OK) return s;
        }
      }
    } else if (pl.td.on && pl.fd.on) {
      const bool fused = ctx->schedule == 1 ||
                         (ctx->schedule == 0 && !separate_by_default(pl.jobs.data() + j0, j1 - j0, pl.dtype));
      if (fused) {
        fill_params(ctx, pl, j0, j1, 2, p, next_counters(ctx));
        if ((s = launch_one(ctx, p, pl.max_T, st)) != RFIM_OK) return s;
      } else {
        fill_params(ctx, pl, j0, j1, 0, p, next_counters(ctx));
        if ((s = launch_one(ctx, p, pl.max_T, st)) != RFIM_OK) return s;
        fill_params(ctx, pl, j0, j1, 3, p, next_counters(ctx));
        if ((s = launch_one(ctx, p, pl.max_T, st)) != RFIM_OK) return s;
      }
    } else if (pl.td.on) {
      fill_params(ctx, pl, j0, j1, 0, p, next_counters(ctx));
      if ((s = launch_one(ctx, p, pl.max_T, st)) != RFIM_OK) return s;
    } else if (pl.fd.on) {
      fill_params(ctx, pl, j0, j1, 1, p, next_counters(ctx));
      if ((s = launch_one(ctx, p, pl.max_T, st)) != RFIM_OK) return s;
    }
  }
  return RFIM_OK;
}

rfim_status make_plan(rfim_ctx* ctx, const rfim_block* blocks, int n, const rfim_cut* tdsc, const rfim_cut* fdsc,
                      Plan& pl) {
  if (n < 1) return fail(ctx, RFIM_ERR_ARG, "empty batch");
  if (!blocks) return fail(ctx, RFIM_ERR_ARG, "null block array");
  for (int i = 0; i < n; i++) {
    const rfim_block* b = &blocks[i];
    if (!b) return fail(ctx, RFIM_ERR_ARG, "null block");
    CutNorm td, fd;
    rfim_status s;
    if ((s = check_cut(ctx, tdsc, b->channels, false, td)) != RFIM_OK) return s;
    if ((s = check_cut(ctx, fdsc, b->channels, true, fd)) != RFIM_OK) return s;
    if ((s = check_block(ctx, b, td, fd)) != RFIM_OK) return s;
    if ((s = check_impl(ctx, b, td, fd)) != RFIM_OK) return s;
    if (i == 0) {
      pl.td = td;
      pl.fd = fd;
      pl.mask_kind = (int)b->mask_fmt;
      pl.dtype = b->dtype;
    } else {
      if (b->dtype != blocks[0].dtype || b->layout != blocks[0].layout)
        return fail(ctx, RFIM_ERR_ARG, "all blocks of a batch must share dtype and layout");
      if ((int)b->mask_fmt != pl.mask_kind) return fail(ctx, RFIM_ERR_ARG, "all blocks of a batch must share mask format");
      if (fd.on && fd.bin != pl.fd.bin)
        return fail(ctx, RFIM_ERR_ARG, "fdsc_bin resolves differently across blocks; pass an explicit bin");
    }
  }
  for (int i = 0; i < n; i++) add_block_jobs(ctx, pl, &blocks[i]);
  // float32 with both methods, non-random TDSC and a bit mask: record TDSC's
  // cuts per row (the fused launch then writes each value once, from FDSC)
  bool records = ctx->f32_records && pl.dtype == RFIM_F32 && pl.td.on && pl.fd.on &&
                 pl.td.rep != RFIM_REPLACE_RANDOM && pl.mask_kind == RFIM_MASK_BITS;
  // the FDSC tile then also holds one mask word per channel: the widest sub-slab that still fits
  auto records_ws = [&](const Job& J) {
    const bool rnd = pl.fd.rep == RFIM_REPLACE_RANDOM;
    const int budget = std::min(MAX_SMEM_PER_CTA, std::max(ctx->smem_target, fd32_smem_bytes(1, J.C, J.nb, rnd, true)));
    for (int cand : {8, 4, 2, 1})
      if ((ctx->tile_samples == 0 || cand <= ctx->tile_samples) && fd32_smem_bytes(cand, J.C, J.nb, rnd, true) <= budget)
        return cand;
    return 0;
  };
  for (const Job& J : pl.jobs)
    if (records && records_ws(J) == 0) records = false;
  if (records) {
    for (Job& J : pl.jobs) {
      J.ws = records_ws(J);
      J.fd_items = (J.T + J.ws - 1) / J.ws;
    }
    size_t rows = 0;
    for (const Job& J : pl.jobs) rows += (size_t)J.C;
    const size_t bytes = rows * (size_t)pl.td.it * PROG_FLOATS * sizeof(float);
    if (bytes > ctx->prog_cap) {
      float* p = nullptr;
      const size_t cap = std::max(bytes, 2 * ctx->prog_cap);
      cudaError_t e = ctx_malloc(ctx, reinterpret_cast<void**>(&p), cap);
      if (e != cudaSuccess) return fail(ctx, RFIM_ERR_OOM, "TDSC cut records: %s", cudaGetErrorString(e));
      if (ctx->prog) ctx->prog_retired.push_back(ctx->prog);
      ctx->prog = p;
      ctx->prog_cap = cap;
    }
    size_t off = 0;
    for (Job& J : pl.jobs) {
      J.prog = ctx->prog + off;
      off += (size_t)J.C * pl.td.it * PROG_FLOATS;
    }
    pl.prog = true;
  }
  return RFIM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

rfim_status rfim_create(rfim_ctx** out, int device, size_t hbm_budget_bytes, const char* tune_cache) {
  if (!out) return RFIM_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return RFIM_ERR_ARG;
  rfim_ctx* ctx = new (std::nothrow) rfim_ctx();
  if (!ctx) return RFIM_ERR_OOM;
  ctx->device = device;
  ctx->hbm_budget = hbm_budget_bytes;
  if (tune_cache) ctx->tune_cache = tune_cache;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_counters, sizeof(unsigned) * COUNTER_BLOCKS * COUNTER_STRIDE);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status, sizeof(unsigned) * 4);
  if (e == cudaSuccess) e = cudaMemset(ctx->d_counters, 0, sizeof(unsigned) * COUNTER_BLOCKS * COUNTER_STRIDE);
  if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(unsigned) * 4);
  if (e != cudaSuccess) {
    cudaFree(ctx->d_counters);
    cudaFree(ctx->d_status);
    delete ctx;
    return e == cudaErrorMemoryAllocation ? RFIM_ERR_OOM : RFIM_ERR_CUDA;
  }
  ctx->tuner = tuner_create(ctx->tune_cache);
  *out = ctx;
  return RFIM_OK;
}

rfim_status rfim_destroy(rfim_ctx* ctx) {
  if (!ctx) return RFIM_OK;
  cudaSetDevice(ctx->device);
  if (ctx->stream) {
    stream_service_destroy(ctx->stream);
    ctx->stream = nullptr;
  }
  cudaDeviceSynchronize();
  for (auto& kv : ctx->graphs) {
    cudaGraphExecDestroy(kv.second.first);
    cudaFree(kv.second.second);
  }
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  cudaFree(ctx->btc_buf);
  cudaFree(ctx->btc_mask);
  cudaFree(ctx->prog);
  for (float* p : ctx->prog_retired) cudaFree(p);
  if (ctx->stager) stager_destroy(ctx->stager);
  if (ctx->tuner) tuner_destroy(ctx->tuner);
  cudaFree(ctx->d_counters);
  cudaFree(ctx->d_status);
  delete ctx;
  return RFIM_OK;
}

rfim_status rfim_set_option(rfim_ctx* ctx, const char* key, long long value) {
  if (!ctx || !key) return RFIM_ERR_ARG;
  const std::string k = key;
  if (k == "spin_limit_us") {
    if (value < 1) return fail(ctx, RFIM_ERR_ARG, "spin_limit_us must be >= 1");
    ctx->spin_limit_us = value;
  } else if (k == "schedule") {
    if (value < 0 || value > 2) return fail(ctx, RFIM_ERR_ARG, "schedule must be 0, 1 or 2");
    ctx->schedule = (int)value;
  } else if (k == "tile_samples") {
    if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8 && value != 16 && value != 32)
      return fail(ctx, RFIM_ERR_ARG, "tile_samples must be 0, 1, 2, 4, 8, 16 or 32");
    ctx->tile_samples = (int)value;
  } else if (k == "stage_group_bytes") {
    if (value < (1ll << 20) || value > (1ll << 34)) return fail(ctx, RFIM_ERR_ARG, "stage_group_bytes must be in 1 MB..16 GB");
    ctx->stage_group_bytes = value;
  } else if (k == "stage_streams") {
    if (value < 1 || value > 4) return fail(ctx, RFIM_ERR_ARG, "stage_streams must be 1..4");
    ctx->stage_streams = (int)value;
  } else if (k == "f32_records") {
    if (value != 0 && value != 1) return fail(ctx, RFIM_ERR_ARG, "f32_records must be 0 or 1");
    ctx->f32_records = (int)value;
  } else if (k == "order") {
    if (value != 0 && value != 1) return fail(ctx, RFIM_ERR_ARG, "order must be 0 (blocked) or 1 (interleaved)");
    ctx->order = (int)value;
  } else if (k == "ctas_per_sm") {
    if (value < 0 || value > 32) return fail(ctx, RFIM_ERR_ARG, "ctas_per_sm must be in 0..32");
    ctx->ctas_per_sm = (int)value;
  } else if (k == "withhold_tdsc_done") {
    ctx->withhold = value ? 1 : 0;
  } else if (k == "smem_target") {
    if (value < 16384 || value > MAX_SMEM_PER_CTA) return fail(ctx, RFIM_ERR_ARG, "smem_target out of range");
    ctx->smem_target = (int)value;
  } else if (k == "fail_alloc_after") {
    ctx->fail_alloc_after = value < 0 ? -1 : value;
  } else if (k == "fused_lag") {
    if (value < 0 || value > 8) return fail(ctx, RFIM_ERR_ARG, "fused_lag must be in 0..8");
    ctx->fused_lag = (int)value;
  } else {
    return fail(ctx, RFIM_ERR_ARG, "unknown option '%s'", key);
  }
  return RFIM_OK;
}

// BTC blocks (channel fastest): each block is transposed into a BCT scratch
// copy, cleaned there in place with the BCT engine, and transposed back; the
// mask is produced in BCT form and transposed into the caller's BTC mask.
static rfim_status run_btc(rfim_ctx* ctx, const rfim_block* blocks, int n, const rfim_cut* tdsc,
                           const rfim_cut* fdsc, cudaStream_t st) {
  for (int i = 0; i < n; i++) {
    const rfim_block* b = &blocks[i];
    if (!b) return fail(ctx, RFIM_ERR_ARG, "null block");
    CutNorm td, fd;
    rfim_status s;
    if ((s = check_cut(ctx, tdsc, b->channels, false, td)) != RFIM_OK) return s;
    if ((s = check_cut(ctx, fdsc, b->channels, true, fd)) != RFIM_OK) return s;
    if ((s = check_block(ctx, b, td, fd)) != RFIM_OK) return s;
    if (b->layout != RFIM_LAYOUT_BTC || b->dtype != blocks[0].dtype || b->mask_fmt != blocks[0].mask_fmt)
      return fail(ctx, RFIM_ERR_ARG, "all blocks of a batch must share dtype, layout and mask format");
    const size_t es = dtype_size(b->dtype);
    const size_t N = (size_t)b->beams * b->channels * b->samples;
    const size_t mbytes = b->mask_fmt == RFIM_MASK_BITS
                              ? (size_t)b->beams * b->channels * ((b->samples + 31) / 32) * 4
                              : (b->mask_fmt == RFIM_MASK_BYTES ? N : 0);
    if (ctx->btc_cap < N * es) {
      cudaFree(ctx->btc_buf);
      ctx->btc_buf = nullptr;
      ctx->btc_cap = 0;
      if (ctx_malloc(ctx, &ctx->btc_buf, N * es) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, RFIM_ERR_OOM, "BTC scratch of %zu bytes", N * es);
      }
      ctx->btc_cap = N * es;
    }
    if (mbytes && ctx->btc_mask_cap < mbytes) {
      cudaFree(ctx->btc_mask);
      ctx->btc_mask = nullptr;
      ctx->btc_mask_cap = 0;
      if (ctx_malloc(ctx, &ctx->btc_mask, mbytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, RFIM_ERR_OOM, "BTC mask scratch of %zu bytes", mbytes);
      }
      ctx->btc_mask_cap = mbytes;
    }
    int e = launch_transpose(b->in, ctx->btc_buf, b->beams, b->samples, b->channels, (int)es, st);
    if (e != 0) return cuda_fail(ctx, (cudaError_t)e, "BTC transpose");
    rfim_block d = *b;
    d.in = ctx->btc_buf;
    d.out = ctx->btc_buf;
    d.mask = mbytes ? ctx->btc_mask : nullptr;
    d.layout = RFIM_LAYOUT_BCT;
    Plan pl;
    if ((s = make_plan(ctx, &d, 1, tdsc, fdsc, pl)) != RFIM_OK) return s;
    if ((s = run_plan(ctx, pl, st)) != RFIM_OK) return s;
    e = launch_transpose(ctx->btc_buf, b->out, b->beams, b->channels, b->samples, (int)es, st);
    if (e == 0 && b->mask_fmt == RFIM_MASK_BITS)
      e = launch_transpose_bits(ctx->btc_mask, b->mask, b->beams, b->channels, b->samples, st);
    else if (e == 0 && b->mask_fmt == RFIM_MASK_BYTES)
      e = launch_transpose(ctx->btc_mask, b->mask, b->beams, b->channels, b->samples, 1, st);
    if (e != 0) return cuda_fail(ctx, (cudaError_t)e, "BTC transpose back");
  }
  return RFIM_OK;
}

static rfim_status clean_common(rfim_ctx* ctx, const rfim_block* blk, const rfim_cut* tdsc, const rfim_cut* fdsc,
                                void* stream) {
  if (!ctx) return RFIM_ERR_ARG;
  if (!tdsc && !fdsc) return fail(ctx, RFIM_ERR_ARG, "no cut given");
  cudaSetDevice(ctx->device);
  if (blk && blk->layout == RFIM_LAYOUT_BTC) return run_btc(ctx, blk, 1, tdsc, fdsc, (cudaStream_t)stream);
  Plan pl;
  rfim_status s = make_plan(ctx, blk, 1, tdsc, fdsc, pl);
  if (s != RFIM_OK) return s;
  return run_plan(ctx, pl, (cudaStream_t)stream);
}

rfim_status rfim_tdsc(rfim_ctx* ctx, const rfim_block* blk, const rfim_cut* cut, void* stream) {
  if (ctx && !cut) return fail(ctx, RFIM_ERR_ARG, "null cut");
  return clean_common(ctx, blk, cut, nullptr, stream);
}

rfim_status rfim_fdsc(rfim_ctx* ctx, const rfim_block* blk, const rfim_cut* cut, void* stream) {
  if (ctx && !cut) return fail(ctx, RFIM_ERR_ARG, "null cut");
  return clean_common(ctx, blk, nullptr, cut, stream);
}

rfim_status rfim_clean(rfim_ctx* ctx, const rfim_block* blk, const rfim_cut* tdsc, const rfim_cut* fdsc,
                       void* stream) {
  return clean_common(ctx, blk, tdsc, fdsc, stream);
}

rfim_status rfim_clean_batch(rfim_ctx* ctx, const rfim_block* blocks, int n, const rfim_cut* tdsc,
                             const rfim_cut* fdsc, unsigned flags, void* stream) {
  if (!ctx) return RFIM_ERR_ARG;
  if (!tdsc && !fdsc) return fail(ctx, RFIM_ERR_ARG, "no cut given");
  if (flags & ~(RFIM_BATCH_GRAPH | RFIM_BATCH_AUTOTUNE)) return fail(ctx, RFIM_ERR_ARG, "unknown batch flags");
  cudaSetDevice(ctx->device);
  if (n >= 1 && blocks && blocks[0].layout == RFIM_LAYOUT_BTC)
    return run_btc(ctx, blocks, n, tdsc, fdsc, (cudaStream_t)stream);  // block by block, no capture
  Plan pl;
  rfim_status s = make_plan(ctx, blocks, n, tdsc, fdsc, pl);
  if (s != RFIM_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  if (flags & RFIM_BATCH_AUTOTUNE) {
    s = tuner_apply(ctx->tuner, ctx, blocks, n, tdsc, fdsc);
    if (s != RFIM_OK) return s;
    pl = Plan();
    if ((s = make_plan(ctx, blocks, n, tdsc, fdsc, pl)) != RFIM_OK) return s;
  }
  if (!(flags & RFIM_BATCH_GRAPH)) return run_plan(ctx, pl, st);
  // key: the plan's jobs, cuts and the options that shape the launch
  std::vector<unsigned char> key(sizeof(Job) * pl.jobs.size() + 256);
  memcpy(key.data(), pl.jobs.data(), sizeof(Job) * pl.jobs.size());
  unsigned char* kp = key.data() + sizeof(Job) * pl.jobs.size();
  memcpy(kp, &pl.td, sizeof(CutNorm));
  memcpy(kp + 64, &pl.fd, sizeof(CutNorm));
  int opts[10] = {pl.mask_kind, ctx->schedule, ctx->ctas_per_sm, ctx->fused_lag, ctx->withhold,
                  (int)ctx->spin_limit_us, ctx->tile_samples, ctx->smem_target, ctx->order, ctx->f32_records};
  memcpy(kp + 128, opts, sizeof opts);
  auto it = ctx->graphs.find(key);
  if (it == ctx->graphs.end()) {
    if (!ctx->capture_stream) {
      cudaError_t e = cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamCreate");
    }
    // A replayed graph reuses its counter blocks: give it its own, outside the ring.
    const int rounds = ctx->order == 1 ? std::max(1, std::max(pl.td.it, pl.fd.it)) : 1;
    const int launches = 2 * rounds * (((int)pl.jobs.size() + MAX_JOBS - 1) / MAX_JOBS);
    unsigned* gc = nullptr;
    cudaError_t e = ctx_malloc(ctx, reinterpret_cast<void**>(&gc), sizeof(unsigned) * COUNTER_STRIDE * launches);
    if (e != cudaSuccess) return fail(ctx, RFIM_ERR_OOM, "graph counters: %s", cudaGetErrorString(e));
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      cudaFree(gc);
      return cuda_fail(ctx, e, "cudaStreamBeginCapture");
    }
    ctx->capture_counters = gc;
    ctx->capture_used = 0;
    s = run_plan(ctx, pl, ctx->capture_stream);
    ctx->capture_counters = nullptr;
    e = cudaStreamEndCapture(ctx->capture_stream, &g);
    if (s != RFIM_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaFree(gc);
      return s != RFIM_OK ? s : cuda_fail(ctx, e, "cudaStreamEndCapture");
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      cudaFree(gc);
      return cuda_fail(ctx, e, "cudaGraphInstantiate");
    }
    if (ctx->graphs.size() > 64) {
      cudaDeviceSynchronize();
      for (auto& kv : ctx->graphs) {
        cudaGraphExecDestroy(kv.second.first);
        cudaFree(kv.second.second);
      }
      ctx->graphs.clear();
    }
    it = ctx->graphs.emplace(key, std::make_pair(ex, gc)).first;
  }
  cudaError_t e = cudaGraphLaunch(it->second.first, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphLaunch");
  return RFIM_OK;
}

rfim_status rfim_clean_host(rfim_ctx* ctx, const rfim_block* host_blk, const rfim_cut* tdsc, const rfim_cut* fdsc) {
  if (!ctx) return RFIM_ERR_ARG;
  if (!tdsc && !fdsc) return fail(ctx, RFIM_ERR_ARG, "no cut given");
  cudaSetDevice(ctx->device);
  if (!ctx->stager) {
    ctx->stager = stager_create(ctx);
    if (!ctx->stager) return fail(ctx, RFIM_ERR_OOM, "could not create host staging");
  }
  return stager_run(ctx->stager, ctx, host_blk, tdsc, fdsc);
}

rfim_status rfim_device_status(rfim_ctx* ctx, void* stream) {
  if (!ctx) return RFIM_ERR_ARG;
  cudaSetDevice(ctx->device);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
  unsigned st = 0;
  e = cudaMemcpy(&st, ctx->d_status, sizeof st, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "status read");
  if (st) {
    cudaMemset(ctx->d_status, 0, sizeof(unsigned));
    // counters of a launch that timed out are left mid-way; the ring resets them per launch
    return fail(ctx, RFIM_ERR_TIMEOUT, "a device-side wait gave up (status %u)", st);
  }
  // the streaming service's batches report through their own status words
  if (ctx->stream) {
    const unsigned long long n = stream_service_take_timeouts(ctx->stream);
    if (n) return fail(ctx, RFIM_ERR_TIMEOUT, "%llu streaming batch(es) had a device-side wait give up", n);
  }
  return RFIM_OK;
}

const char* rfim_status_str(rfim_status s) {
  switch (s) {
    case RFIM_OK: return "ok";
    case RFIM_ERR_ARG: return "invalid argument";
    case RFIM_ERR_RANGE: return "shape outside the exact-integer range";
    case RFIM_ERR_OOM: return "out of memory";
    case RFIM_ERR_CUDA: return "CUDA error";
    case RFIM_ERR_TIMEOUT: return "device-side wait timed out";
    case RFIM_ERR_BUSY: return "busy";
    case RFIM_ERR_STATE: return "invalid state";
  }
  return "unknown status";
}

const char* rfim_last_error(rfim_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

const char* rfim_version(void) { return "rfim-gb300 0.1 sm_103a"; }

}  // extern "C"

// ---------------------------------------------------------------------------
// entry points used by the runtime (stream service, stager, tuner)
// ---------------------------------------------------------------------------
namespace rfim {

rfim_status ctx_clean_async(rfim_ctx* ctx, const rfim_block* blocks, int n, const rfim_cut* tdsc,
                            const rfim_cut* fdsc, cudaStream_t st) {
  if (n >= 1 && blocks && blocks[0].layout == RFIM_LAYOUT_BTC) return run_btc(ctx, blocks, n, tdsc, fdsc, st);
  Plan pl;
  rfim_status s = make_plan(ctx, blocks, n, tdsc, fdsc, pl);
  if (s != RFIM_OK) return s;
  return run_plan(ctx, pl, st);
}

int ctx_device(rfim_ctx* ctx) { return ctx->device; }
size_t ctx_hbm_budget(rfim_ctx* ctx) { return ctx->hbm_budget; }
void ctx_set_error(rfim_ctx* ctx, const char* msg) { ctx->last_error = msg; }

// Every device (and pinned host) allocation a context makes after rfim_create
// goes through here, so that the "fail_alloc_after" test hook can refuse it
// exactly as a full device would (cudaErrorMemoryAllocation, nothing allocated).
cudaError_t ctx_malloc(rfim_ctx* ctx, void** p, size_t bytes, bool pinned_host) {
  *p = nullptr;
  if (ctx && ctx->fail_alloc_after >= 0) {
    if (ctx->fail_alloc_after == 0) return cudaErrorMemoryAllocation;
    ctx->fail_alloc_after--;
  }
  return pinned_host ? cudaMallocHost(p, bytes) : cudaMalloc(p, bytes);
}
StreamService*& ctx_stream_service(rfim_ctx* ctx) { return ctx->stream; }
void ctx_stage_options(rfim_ctx* ctx, size_t& group_bytes, int& streams) {
  group_bytes = (size_t)ctx->stage_group_bytes;
  streams = ctx->stage_streams;
}
void ctx_get_tunables(rfim_ctx* ctx, Tunables& t) {
  t.schedule = ctx->schedule;
  t.ctas_per_sm = ctx->ctas_per_sm;
  t.smem_target = ctx->smem_target;
  t.fused_lag = ctx->fused_lag;
}
void ctx_set_tunables(rfim_ctx* ctx, const Tunables& t) {
  ctx->schedule = t.schedule;
  ctx->ctas_per_sm = t.ctas_per_sm;
  ctx->smem_target = t.smem_target;
  ctx->fused_lag = t.fused_lag;
}

// Plan and launch one block with caller-provided counters: no heap or device
// allocation, default tuning (fused schedule with one beam of lag).
rfim_status noalloc_clean(const rfim_block* b, const rfim_cut* tdsc, const rfim_cut* fdsc, unsigned* counters,
                          unsigned* status, cudaStream_t st) {
  return launch_blocks_fixed(b, 1, tdsc, fdsc, counters, status, st);
}

rfim_status ctx_validate(rfim_ctx* ctx, const rfim_block* b, const rfim_cut* tdsc, const rfim_cut* fdsc) {
  CutNorm td, fd;
  rfim_status s;
  if ((s = check_cut(ctx, tdsc, b->channels, false, td)) != RFIM_OK) return s;
  if ((s = check_cut(ctx, fdsc, b->channels, true, fd)) != RFIM_OK) return s;
  if ((s = check_block(ctx, b, td, fd)) != RFIM_OK) return s;
  return check_impl(ctx, b, td, fd);
}

void ctx_wait_options(rfim_ctx* ctx, unsigned long long& spin_limit_ns, int& withhold_job) {
  spin_limit_ns = (unsigned long long)ctx->spin_limit_us * 1000ull;
  withhold_job = ctx->withhold ? 0 : -1;
}

rfim_status launch_blocks_fixed(const rfim_block* blocks, int n, const rfim_cut* tdsc, const rfim_cut* fdsc,
                                unsigned* counters, unsigned* status, cudaStream_t st, double* const* stats,
                                unsigned long long spin_limit_ns, int withhold_job) {
  if (!tdsc && !fdsc) return RFIM_ERR_ARG;
  if (!blocks || n < 1) return RFIM_ERR_ARG;
  CutNorm td, fd;
  rfim_status s;
  int beams = 0;
  for (int i = 0; i < n; i++) {
    const rfim_block* b = &blocks[i];
    if ((s = check_cut(nullptr, tdsc, b->channels, false, td)) != RFIM_OK) return s;
    if ((s = check_cut(nullptr, fdsc, b->channels, true, fd)) != RFIM_OK) return s;
    if ((s = check_block(nullptr, b, td, fd)) != RFIM_OK) return s;
    if ((s = check_impl(nullptr, b, td, fd)) != RFIM_OK) return s;
    if (b->dtype != blocks[0].dtype || b->layout != blocks[0].layout || b->mask_fmt != blocks[0].mask_fmt)
      return RFIM_ERR_ARG;
    if (fd.on && fdsc->fdsc_bin == 0 && b->channels != blocks[0].channels) return RFIM_ERR_ARG;
    beams += b->beams;
  }
  if (beams > MAX_JOBS) return RFIM_ERR_RANGE;
  Params p;  // on the stack: no allocation
  memset(&p, 0, sizeof p);
  p.n_jobs = beams;
  for (int i = 0, j0 = 0; i < n; j0 += blocks[i].beams, i++)
    for (int j = 0; j < blocks[i].beams; j++) {
      p.jobs[j0 + j] = make_job(&blocks[i], j, fd, 0, 113 * 1024);
      random_row_mode(p.jobs[j0 + j], &blocks[i], td);
      if (stats && stats[i]) p.jobs[j0 + j].stats = stats[i] + 2 * (size_t)j * blocks[i].channels;
    }
  const rfim_block* b = &blocks[0];
  const bool both = td.on && fd.on;
  const bool separate = both && separate_by_default(p.jobs, beams, b->dtype);
  // the status word keeps the previous call's value: clear it once
  if (cudaMemsetAsync(status, 0, sizeof(unsigned), st) != cudaSuccess) return clear_cuda_error();
  // one fused launch (mode 2), or TDSC (mode 0) then FDSC on its output (mode 3)
  const int modes[2] = {separate ? 0 : (both ? 2 : (td.on ? 0 : 1)), separate ? 3 : -1};
  for (const int mode : modes) {
    if (mode < 0) break;
    p.td = cut_dev(td, b->dtype);
    p.fd = cut_dev(fd, b->dtype);
    if (mode == 1 || mode == 3) p.td.iterations = 0;
    if (mode == 0) p.fd.iterations = 0;
    p.mask_kind = (int)b->mask_fmt;
    p.fd_reads_out = (mode == 2 || mode == 3) ? 1 : 0;
    p.wait_tdsc = mode == 2 ? 1 : 0;
    p.mask_or = (mode == 2 || mode == 3) ? 1 : 0;
    p.withhold_job = mode == 2 ? withhold_job : -1;
    p.spin_limit_ns = spin_limit_ns;
    p.counters = counters;
    p.status = status;
    p.dtype = b->dtype == RFIM_F32 ? 1 : 0;
    fill_segments(p, mode, 1);
    LaunchCfg cfg;
    cfg.smem = engine_smem(p);
    if (cfg.smem > MAX_SMEM_PER_CTA) return RFIM_ERR_ARG;
    void* fn = engine_kernel(p);
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return clear_cuda_error();
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_SMEM_PER_CTA) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NT, cfg.smem) != cudaSuccess)
      return clear_cuda_error();
    cfg.grid = std::max(1, std::min(p.n_items, sms * std::max(1, per_sm)));
    // the shared counters keep the previous launch's values: clear them
    if (cudaMemsetAsync(counters, 0, sizeof(unsigned) * (1 + p.n_jobs), st) != cudaSuccess ||
        clear_f32_fdsc_masks(p, st) != cudaSuccess)
      return clear_cuda_error();
    if (launch_engine(p, cfg, st) != (int)cudaSuccess) return clear_cuda_error();
  }
  return RFIM_OK;
}

}  // namespace rfim
