// runtime.cu -- host-buffer staging (rfim_clean_host) and the autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "runtime.h"

namespace rfim {

namespace {
size_t esize(rfim_dtype d) { return d == RFIM_F32 ? 4 : 1; }

size_t mask_beam_bytes(const rfim_block* b) {
  if (b->mask_fmt == RFIM_MASK_NONE || !b->mask) return 0;
  const size_t slow = b->layout == RFIM_LAYOUT_BCT ? (size_t)b->channels : (size_t)b->samples;
  const size_t fast = b->layout == RFIM_LAYOUT_BCT ? (size_t)b->samples : (size_t)b->channels;
  if (b->mask_fmt == RFIM_MASK_BITS) return slow * ((fast + 31) / 32) * 4;
  return slow * fast;
}
}  // namespace

// ---------------------------------------------------------------------------
// Host staging: beams are cleaned in groups on up to four CUDA streams (a
// ring), so that the host-to-device copy of one group, the cleaning of another
// and the copy back of a third overlap.  Device buffers are owned by the context and grow on
// demand; each group is cleaned in place in its staging buffer.
// ---------------------------------------------------------------------------
constexpr int STAGE_MAX_STREAMS = 4;

struct HostStager {
  int dev = 0;
  cudaStream_t st[STAGE_MAX_STREAMS] = {};
  void* dbuf[STAGE_MAX_STREAMS] = {};
  void* dmask[STAGE_MAX_STREAMS] = {};
  size_t cap_buf = 0, cap_mask = 0;
};

HostStager* stager_create(rfim_ctx* ctx) {
  HostStager* s = new HostStager();
  s->dev = ctx_device(ctx);
  for (int i = 0; i < STAGE_MAX_STREAMS; i++) {
    if (cudaStreamCreateWithFlags(&s->st[i], cudaStreamNonBlocking) != cudaSuccess) {
      stager_destroy(s);
      return nullptr;
    }
  }
  return s;
}

void stager_destroy(HostStager* s) {
  if (!s) return;
  for (int i = 0; i < STAGE_MAX_STREAMS; i++) {
    if (s->st[i]) cudaStreamSynchronize(s->st[i]);
    cudaFree(s->dbuf[i]);
    cudaFree(s->dmask[i]);
    if (s->st[i]) cudaStreamDestroy(s->st[i]);
  }
  delete s;
}

rfim_status stager_run(HostStager* s, rfim_ctx* ctx, const rfim_block* hb, const rfim_cut* tdsc,
                       const rfim_cut* fdsc) {
  if (!hb || !hb->in || !hb->out || hb->beams < 1 || hb->channels < 1 || hb->samples < 1) {
    ctx_set_error(ctx, "invalid host block");
    return RFIM_ERR_ARG;
  }
  const size_t beam = (size_t)hb->channels * hb->samples * esize(hb->dtype);
  const size_t mbeam = mask_beam_bytes(hb);
  size_t group_bytes;
  int ns;
  ctx_stage_options(ctx, group_bytes, ns);
  ns = std::max(1, std::min(ns, STAGE_MAX_STREAMS));
  const int group = (int)std::max<size_t>(1, std::min<size_t>((size_t)hb->beams, group_bytes / std::max<size_t>(beam, 1)));
  const size_t need = beam * group, needm = mbeam * group;
  for (int i = 0; i < STAGE_MAX_STREAMS; i++) {
    if (s->cap_buf < need || (needm && s->cap_mask < needm)) cudaStreamSynchronize(s->st[i]);
  }
  if (s->cap_buf < need) {
    for (int i = 0; i < STAGE_MAX_STREAMS; i++) {
      cudaFree(s->dbuf[i]);
      s->dbuf[i] = nullptr;
      if (ctx_malloc(ctx, &s->dbuf[i], need) != cudaSuccess) {
        s->cap_buf = 0;
        ctx_set_error(ctx, "staging allocation failed");
        return RFIM_ERR_OOM;
      }
    }
    s->cap_buf = need;
  }
  if (needm && s->cap_mask < needm) {
    for (int i = 0; i < STAGE_MAX_STREAMS; i++) {
      cudaFree(s->dmask[i]);
      s->dmask[i] = nullptr;
      if (ctx_malloc(ctx, &s->dmask[i], needm) != cudaSuccess) {
        s->cap_mask = 0;
        ctx_set_error(ctx, "staging allocation failed");
        return RFIM_ERR_OOM;
      }
    }
    s->cap_mask = needm;
  }
  const char* hin = (const char*)hb->in;
  char* hout = (char*)hb->out;
  char* hmask = (char*)hb->mask;
  rfim_status st = RFIM_OK;
  int gi = 0;
  for (int b0 = 0; b0 < hb->beams; b0 += group, gi++) {
    const int i = gi % ns;
    const int nb = std::min(group, hb->beams - b0);
    cudaStream_t str = s->st[i];
    cudaError_t e = cudaMemcpyAsync(s->dbuf[i], hin + (size_t)b0 * beam, (size_t)nb * beam, cudaMemcpyHostToDevice, str);
    if (e != cudaSuccess) {
      ctx_set_error(ctx, cudaGetErrorString(e));
      (void)cudaGetLastError();  // reported here: not left for the caller's next call
      st = RFIM_ERR_CUDA;
      break;
    }
    rfim_block d = *hb;
    d.in = s->dbuf[i];
    d.out = s->dbuf[i];
    d.mask = mbeam ? s->dmask[i] : nullptr;
    d.beams = nb;
    if (!mbeam) d.mask_fmt = RFIM_MASK_NONE;
    st = ctx_clean_async(ctx, &d, 1, tdsc, fdsc, str);
    if (st != RFIM_OK) break;
    e = cudaMemcpyAsync(hout + (size_t)b0 * beam, s->dbuf[i], (size_t)nb * beam, cudaMemcpyDeviceToHost, str);
    if (e == cudaSuccess && mbeam)
      e = cudaMemcpyAsync(hmask + (size_t)b0 * mbeam, s->dmask[i], (size_t)nb * mbeam, cudaMemcpyDeviceToHost, str);
    if (e != cudaSuccess) {
      ctx_set_error(ctx, cudaGetErrorString(e));
      (void)cudaGetLastError();  // reported here: not left for the caller's next call
      st = RFIM_ERR_CUDA;
      break;
    }
  }
  for (int i = 0; i < ns; i++) {
    cudaError_t e = cudaStreamSynchronize(s->st[i]);
    if (e != cudaSuccess && st == RFIM_OK) {
      ctx_set_error(ctx, cudaGetErrorString(e));
      (void)cudaGetLastError();  // reported here: not left for the caller's next call
      st = RFIM_ERR_CUDA;
    }
  }
  return st;
}

// ---------------------------------------------------------------------------
// Autotuner: for a batch signature (dtype, layout, shapes, cuts, device) it
// times candidate schedules -- fused persistent launch with TDSC queued one or
// two beams ahead, or separate TDSC and FDSC launches -- and FDSC tile budgets
// (which set the time width of the shared-memory tile and the CTAs per SM),
// on scratch outputs, keeps the fastest and stores it in a JSON cache.
// ---------------------------------------------------------------------------
struct Tuner {
  std::string path;
  std::map<std::string, Tunables> cache;
  std::mutex mu;
};

static void tuner_load(Tuner* t) {
  if (t->path.empty()) return;
  std::ifstream f(t->path);
  if (!f) return;
  std::string line;
  // one entry per line: "<key>": {"schedule": a, "ctas_per_sm": b, "smem_target": c, "fused_lag": d},
  while (std::getline(f, line)) {
    const size_t q0 = line.find('"');
    if (q0 == std::string::npos) continue;
    const size_t q1 = line.find('"', q0 + 1);
    if (q1 == std::string::npos) continue;
    const std::string key = line.substr(q0 + 1, q1 - q0 - 1);
    Tunables v{0, 0, 0, 1};
    if (sscanf(line.c_str() + q1 + 1, ": {\"schedule\": %d, \"ctas_per_sm\": %d, \"smem_target\": %d, \"fused_lag\": %d",
               &v.schedule, &v.ctas_per_sm, &v.smem_target, &v.fused_lag) == 4)
      t->cache[key] = v;
  }
}

static void tuner_save(Tuner* t) {
  if (t->path.empty()) return;
  const std::string tmp = t->path + ".tmp";
  {
    std::ofstream f(tmp);
    if (!f) return;
    f << "{\n";
    size_t i = 0;
    for (auto& kv : t->cache) {
      f << "  \"" << kv.first << "\": {\"schedule\": " << kv.second.schedule << ", \"ctas_per_sm\": " << kv.second.ctas_per_sm
        << ", \"smem_target\": " << kv.second.smem_target << ", \"fused_lag\": " << kv.second.fused_lag << "}"
        << (++i < t->cache.size() ? "," : "") << "\n";
    }
    f << "}\n";
  }
  std::rename(tmp.c_str(), t->path.c_str());
}

Tuner* tuner_create(const std::string& cache_path) {
  Tuner* t = new Tuner();
  t->path = cache_path;
  tuner_load(t);
  return t;
}

void tuner_destroy(Tuner* t) { delete t; }

static std::string batch_key(rfim_ctx* ctx, const rfim_block* b, int n, const rfim_cut* tdsc, const rfim_cut* fdsc) {
  std::map<std::pair<int, int>, int> shapes;
  for (int i = 0; i < n; i++) shapes[{b[i].channels, b[i].samples}] += b[i].beams;
  std::ostringstream k;
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, ctx_device(ctx));
  k << prop.name << "|d" << b[0].dtype << "l" << b[0].layout << "m" << b[0].mask_fmt;
  for (auto& s : shapes) k << "|" << s.second << "x" << s.first.first << "x" << s.first.second;
  auto cut = [&](const char* nm, const rfim_cut* c) {
    if (!c) return;
    k << "|" << nm << c->k << "," << c->iterations << "," << c->replace << "," << c->fdsc_bin;
  };
  cut("t", tdsc);
  cut("f", fdsc);
  std::string s = k.str();
  for (auto& ch : s)
    if (ch == '"' || ch == '\\' || ch == '\n') ch = '_';
  return s;
}

rfim_status tuner_apply(Tuner* t, rfim_ctx* ctx, const rfim_block* blocks, int n, const rfim_cut* tdsc,
                        const rfim_cut* fdsc) {
  std::lock_guard<std::mutex> g(t->mu);
  const std::string key = batch_key(ctx, blocks, n, tdsc, fdsc);
  auto it = t->cache.find(key);
  if (it != t->cache.end()) {
    ctx_set_tunables(ctx, it->second);
    return RFIM_OK;
  }
  // scratch copies: outputs (and inputs for in-place blocks) never touch user memory
  std::vector<rfim_block> tb(blocks, blocks + n);
  std::vector<void*> allocs;
  auto cleanup = [&]() {
    for (void* p : allocs) cudaFree(p);
  };
  for (auto& b : tb) {
    const size_t bytes = (size_t)b.beams * b.channels * b.samples * esize(b.dtype);
    void* o = nullptr;
    if (ctx_malloc(ctx, &o, bytes) != cudaSuccess) {
      cleanup();
      ctx_set_error(ctx, "autotune scratch allocation failed");
      return RFIM_ERR_OOM;
    }
    allocs.push_back(o);
    if (b.in == b.out) {
      void* i2 = nullptr;
      if (ctx_malloc(ctx, &i2, bytes) != cudaSuccess) {
        cleanup();
        ctx_set_error(ctx, "autotune scratch allocation failed");
        return RFIM_ERR_OOM;
      }
      allocs.push_back(i2);
      cudaMemcpy(i2, b.in, bytes, cudaMemcpyDeviceToDevice);
      b.in = i2;
    }
    b.out = o;
    const size_t mb = mask_beam_bytes(&b) * b.beams;
    if (mb) {
      void* m = nullptr;
      if (ctx_malloc(ctx, &m, mb) != cudaSuccess) {
        cleanup();
        ctx_set_error(ctx, "autotune scratch allocation failed");
        return RFIM_ERR_OOM;
      }
      allocs.push_back(m);
      b.mask = m;
    }
  }
  Tunables orig;
  ctx_get_tunables(ctx, orig);
  std::vector<Tunables> cands;
  const bool both = tdsc && fdsc;
  for (int smem : {76 * 1024, 113 * 1024, 220 * 1024}) {
    if (both) {
      cands.push_back({1, 0, smem, 1});
      cands.push_back({1, 0, smem, 2});
      cands.push_back({2, 0, smem, 1});
    } else {
      cands.push_back({0, 0, smem, 1});
    }
  }
  cudaStream_t st;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  Tunables bestv = orig;
  for (const Tunables& c : cands) {
    ctx_set_tunables(ctx, c);
    if (ctx_clean_async(ctx, tb.data(), n, tdsc, fdsc, st) != RFIM_OK) continue;
    cudaEventRecord(e0, st);
    const int reps = 3;
    bool ok = true;
    for (int r = 0; r < reps && ok; r++) ok = ctx_clean_async(ctx, tb.data(), n, tdsc, fdsc, st) == RFIM_OK;
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || !ok) continue;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= reps;
    if (ms < best) {
      best = ms;
      bestv = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  cleanup();
  ctx_set_tunables(ctx, bestv);
  t->cache[key] = bestv;
  tuner_save(t);
  return RFIM_OK;
}

}  // namespace rfim
