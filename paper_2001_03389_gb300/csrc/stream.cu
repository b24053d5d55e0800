// stream.cu -- streaming service: continuous batching of beam chunks.
//
// Each chunk is one batch in the sense of Sec. IV (statistics from the chunk
// alone), so chunks are independent and can be grouped freely.  Chunks wait
// in a FIFO after admission; a dispatcher thread launches everything waiting
// (up to 160 chunks) as one micro-batch on an idle CUDA stream, so that
// batches overlap on the device, and a host function enqueued behind each
// batch marks its chunks done.  Device-pointer chunks are read in place (the
// kernels clean them into the slot), host chunks are copied into the slot.
//
// Per-beam state on the device: every slot also holds its chunk's per-channel
// input statistics (sum and sum of squares, written by the first TDSC pass),
// and each beam keeps the slot of its latest completed chunk -- cleaned data,
// mask and statistics -- resident until a newer chunk of the beam completes.
// The statistics are records for the caller; no decision reads them.
//
// Each stream's launches report their device status word (a bounded wait
// that gave up) through pinned host memory; a batch that timed out completes
// its chunks with RFIM_ERR_TIMEOUT.
#include <cuda_runtime.h>
#include <time.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "engine.h"
#include "runtime.h"

namespace rfim {

namespace {

double now_mono() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

constexpr int N_STREAMS = 4;
constexpr int MAX_BATCH = MAX_JOBS;  // chunks per micro-batch (one launch)
constexpr int CTR_WORDS = 2 + MAX_JOBS;

enum TicketState { T_WAITING = 0, T_INFLIGHT = 1, T_DONE = 2 };

struct Ticket {
  int slot;
  int beam;
  int state;
  rfim_status status;      // result once done: RFIM_OK, or why the chunk's batch failed
  unsigned long long seq;  // index of the chunk among its beam's pushes
  const void* src;  // device chunk read in place, or the slot itself (host chunks)
  double arrival;
  double done;
};

}  // namespace

struct StreamService {
  rfim_ctx* ctx = nullptr;
  int device = 0;
  int n_beams = 0, C = 0, T = 0;
  rfim_dtype dtype = RFIM_U8;
  rfim_cut td{}, fd{};
  bool has_td = false, has_fd = false;
  size_t chunk_bytes = 0, mask_bytes = 0;  // slot strides (256-byte multiples)
  size_t in_bytes = 0;                      // input bytes of one chunk
  int n_slots = 0;
  unsigned char* d_slots = nullptr;
  unsigned char* d_masks = nullptr;
  double* d_stats = nullptr;  // per slot: 2 doubles per channel (input sum, sum of squares)
  unsigned* d_ctr = nullptr;  // N_STREAMS counter blocks + status words
  unsigned* h_status = nullptr;  // pinned: each stream's status word after its last batch
  unsigned long long spin_limit_ns = 2000000000ull;
  int withhold = -1;
  std::vector<int> free_slots;
  std::vector<int> slot_refs;  // holders of a slot: its ticket until released, its beam's state
  std::vector<int> beam_slot;  // slot of each beam's latest completed chunk (-1: none yet)
  std::vector<unsigned long long> beam_seq;  // that chunk's index among the beam's pushes
  int state_slots = 0;                       // slots held as beam states
  std::unordered_map<unsigned long long, Ticket> tickets;
  unsigned long long next_ticket = 1;
  std::deque<unsigned long long> waiting;
  cudaStream_t streams[N_STREAMS] = {};
  cudaStream_t copy_stream = nullptr;
  std::mutex copy_mu;
  struct Batch {
    StreamService* svc;
    int lane;
    std::vector<unsigned long long> ids;
  };
  Batch batches[N_STREAMS];
  bool busy[N_STREAMS] = {};
  // statistics
  std::vector<double> lat;
  double bytes_done = 0.0, first_arrival = 0.0, last_done = 0.0;
  std::vector<unsigned long long> beam_chunks;
  std::vector<double> beam_last_latency;
  unsigned long long timeouts = 0;  // batches whose device-side wait gave up, not yet reported
  // threads
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread dispatcher;
  bool stop = false;
  bool disp_waiting = false;  // the dispatcher sleeps on cv_work (pushes wake it only then)
  rfim_status fault = RFIM_OK;
};

namespace {

// one holder of slot i fewer; a slot nobody holds returns to the pool (under s->mu)
void slot_unref(StreamService* s, int i) {
  if (--s->slot_refs[i] == 0) s->free_slots.push_back(i);
}

// Host function behind a batch: its chunks are done (runs on a CUDA thread,
// makes no CUDA call; the stream's status word was copied to h_status first).
void CUDART_CB batch_done(void* arg) {
  auto* b = static_cast<StreamService::Batch*>(arg);
  StreamService* s = b->svc;
  const double t = now_mono();
  const rfim_status st = s->h_status[b->lane] ? RFIM_ERR_TIMEOUT : RFIM_OK;
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (st != RFIM_OK) {
      s->fault = st;
      s->timeouts++;
    }
    for (unsigned long long id : b->ids) {
      auto it = s->tickets.find(id);
      if (it == s->tickets.end()) continue;
      Ticket& k = it->second;
      k.state = T_DONE;
      k.status = st;
      k.done = t;
      const int old = s->beam_slot[k.beam];
      // the beam's newest result: its slot becomes the beam's state (a beam
      // without one takes a slot only while states hold under half of them)
      if (st == RFIM_OK && (old < 0 ? 2 * s->state_slots < s->n_slots : k.seq > s->beam_seq[k.beam])) {
        if (old < 0) s->state_slots++;
        s->beam_slot[k.beam] = k.slot;
        s->beam_seq[k.beam] = k.seq;
        s->slot_refs[k.slot]++;
        if (old >= 0) slot_unref(s, old);
      }
      const double l = t - k.arrival;
      s->lat.push_back(l);
      if (s->lat.size() == 1 || k.arrival < s->first_arrival) s->first_arrival = k.arrival;
      s->last_done = std::max(s->last_done, t);
      s->bytes_done += (double)s->in_bytes;
      s->beam_last_latency[k.beam] = l;
    }
    b->ids.clear();
    s->busy[b->lane] = false;
  }
  s->cv_done.notify_all();
  s->cv_work.notify_all();
}

void dispatch_loop(StreamService* s) {
  cudaSetDevice(s->device);
  std::vector<rfim_block> blocks;
  std::vector<double*> stats;
  blocks.reserve(MAX_BATCH);
  stats.reserve(MAX_BATCH);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    int lane = -1;
    s->disp_waiting = true;
    s->cv_work.wait(lk, [&] {
      if (s->stop) return true;
      if (s->waiting.empty()) return false;
      for (int i = 0; i < N_STREAMS; i++)
        if (!s->busy[i]) {
          lane = i;
          return true;
        }
      return false;
    });
    s->disp_waiting = false;
    if (s->stop) break;
    // close a micro-batch: everything waiting, up to MAX_BATCH chunks
    StreamService::Batch& b = s->batches[lane];
    b.ids.clear();
    blocks.clear();
    stats.clear();
    while (!s->waiting.empty() && (int)b.ids.size() < MAX_BATCH) {
      const unsigned long long id = s->waiting.front();
      s->waiting.pop_front();
      Ticket& k = s->tickets[id];
      k.state = T_INFLIGHT;
      b.ids.push_back(id);
      rfim_block blk;
      blk.in = k.src;
      blk.out = s->d_slots + (size_t)k.slot * s->chunk_bytes;
      blk.mask = s->d_masks + (size_t)k.slot * s->mask_bytes;
      blk.beams = 1;
      blk.channels = s->C;
      blk.samples = s->T;
      blk.dtype = s->dtype;
      blk.layout = RFIM_LAYOUT_BCT;
      blk.mask_fmt = RFIM_MASK_BITS;
      blocks.push_back(blk);
      stats.push_back(s->d_stats + (size_t)k.slot * 2 * s->C);
    }
    s->busy[lane] = true;
    lk.unlock();
    unsigned* ctr = s->d_ctr + (size_t)lane * CTR_WORDS;
    rfim_status st = launch_blocks_fixed(blocks.data(), (int)blocks.size(), s->has_td ? &s->td : nullptr,
                                         s->has_fd ? &s->fd : nullptr, ctr, ctr + 1 + MAX_JOBS, s->streams[lane],
                                         stats.data(), s->spin_limit_ns, s->withhold);
    cudaError_t e = cudaSuccess;
    // the batch's status word (cleared by the launch) to the host, then the completion
    if (st == RFIM_OK)
      e = cudaMemcpyAsync(s->h_status + lane, ctr + 1 + MAX_JOBS, sizeof(unsigned), cudaMemcpyDeviceToHost,
                          s->streams[lane]);
    if (st == RFIM_OK && e == cudaSuccess) e = cudaLaunchHostFunc(s->streams[lane], batch_done, &b);
    if (e != cudaSuccess) (void)cudaGetLastError();
    lk.lock();
    if (st != RFIM_OK || e != cudaSuccess) {
      // the batch never ran: report the fault and complete its chunks as failed
      s->fault = st != RFIM_OK ? st : RFIM_ERR_CUDA;
      for (unsigned long long id : b.ids) {
        auto it = s->tickets.find(id);
        if (it != s->tickets.end()) {
          it->second.state = T_DONE;
          it->second.status = s->fault;
          it->second.done = now_mono();
        }
      }
      b.ids.clear();
      s->busy[lane] = false;
      s->cv_done.notify_all();
    }
  }
}

void svc_free(StreamService* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->dispatcher.joinable()) s->dispatcher.join();
  cudaSetDevice(s->device);
  for (int i = 0; i < N_STREAMS; i++)
    if (s->streams[i]) {
      cudaStreamSynchronize(s->streams[i]);
      cudaStreamDestroy(s->streams[i]);
    }
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  cudaFree(s->d_slots);
  cudaFree(s->d_masks);
  cudaFree(s->d_stats);
  cudaFree(s->d_ctr);
  cudaFreeHost(s->h_status);
  delete s;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

StreamService* svc_of(rfim_ctx* ctx) { return ctx ? ctx_stream_service(ctx) : nullptr; }

rfim_status svc_push(StreamService* s, int beam, const void* chunk, bool on_device, double arrival_time_s,
                     unsigned long long* ticket);

}  // namespace

void stream_service_destroy(StreamService* s) { svc_free(s); }

// Batches whose device-side wait gave up since the last call (then cleared).
unsigned long long stream_service_take_timeouts(StreamService* s) {
  std::lock_guard<std::mutex> g(s->mu);
  const unsigned long long n = s->timeouts;
  s->timeouts = 0;
  return n;
}

}  // namespace rfim

using namespace rfim;

extern "C" {

rfim_status rfim_stream_open(rfim_ctx* ctx, int n_beams, int channels, int chunk_samples, rfim_dtype dtype,
                             const rfim_cut* tdsc, const rfim_cut* fdsc) {
  if (!ctx) return RFIM_ERR_ARG;
  if (ctx_stream_service(ctx)) {
    ctx_set_error(ctx, "streaming service already open");
    return RFIM_ERR_STATE;
  }
  if (n_beams < 1 || channels < 1 || chunk_samples < 1 || (dtype != RFIM_U8 && dtype != RFIM_F32)) {
    ctx_set_error(ctx, "invalid streaming shape");
    return RFIM_ERR_ARG;
  }
  if (!tdsc && !fdsc) {
    ctx_set_error(ctx, "no cut given");
    return RFIM_ERR_ARG;
  }
  const int dev = ctx_device(ctx);
  cudaSetDevice(dev);
  auto* s = new StreamService();
  s->ctx = ctx;
  s->device = dev;
  s->n_beams = n_beams;
  s->C = channels;
  s->T = chunk_samples;
  s->dtype = dtype;
  if (tdsc) {
    s->td = *tdsc;
    s->has_td = true;
  }
  if (fdsc) {
    s->fd = *fdsc;
    s->has_fd = true;
  }
  s->in_bytes = (size_t)channels * chunk_samples * (dtype == RFIM_F32 ? 4 : 1);
  s->chunk_bytes = s->in_bytes;
  s->mask_bytes = (size_t)channels * ((chunk_samples + 31) / 32) * 4;
  s->chunk_bytes = (s->chunk_bytes + 255) & ~(size_t)255;  // slots on 256-byte boundaries
  s->mask_bytes = (s->mask_bytes + 255) & ~(size_t)255;
  // validate the shape and cuts with a dry plan (no launch): a zero-beam check
  {
    rfim_block b{};
    b.in = (const void*)256;
    b.out = (void*)(256 + s->chunk_bytes);
    b.mask = (void*)(256 + 2 * s->chunk_bytes);
    b.beams = 1;
    b.channels = channels;
    b.samples = chunk_samples;
    b.dtype = dtype;
    b.layout = RFIM_LAYOUT_BCT;
    b.mask_fmt = RFIM_MASK_BITS;
    rfim_status st = ctx_validate(ctx, &b, tdsc, fdsc);
    if (st != RFIM_OK) {
      delete s;
      return st;
    }
  }
  size_t budget = ctx_hbm_budget(ctx);
  if (budget == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    budget = fr / 4;
  }
  const size_t per = s->chunk_bytes + s->mask_bytes;
  const size_t want = (size_t)n_beams * 4;
  s->n_slots = (int)std::min<size_t>(want, budget / per);
  if (s->n_slots < 1) {
    delete s;
    ctx_set_error(ctx, "HBM budget holds no streaming slot");
    return RFIM_ERR_OOM;
  }
  if (ctx_malloc(ctx, reinterpret_cast<void**>(&s->d_slots), s->chunk_bytes * s->n_slots) != cudaSuccess ||
      ctx_malloc(ctx, reinterpret_cast<void**>(&s->d_masks), s->mask_bytes * s->n_slots) != cudaSuccess ||
      ctx_malloc(ctx, reinterpret_cast<void**>(&s->d_stats), sizeof(double) * 2 * channels * s->n_slots) !=
          cudaSuccess ||
      ctx_malloc(ctx, reinterpret_cast<void**>(&s->d_ctr), sizeof(unsigned) * CTR_WORDS * N_STREAMS) != cudaSuccess ||
      ctx_malloc(ctx, reinterpret_cast<void**>(&s->h_status), sizeof(unsigned) * N_STREAMS, true) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(s->d_slots);
    cudaFree(s->d_masks);
    cudaFree(s->d_stats);
    cudaFree(s->d_ctr);
    delete s;
    ctx_set_error(ctx, "streaming slot allocation failed");
    return RFIM_ERR_OOM;
  }
  cudaMemset(s->d_ctr, 0, sizeof(unsigned) * CTR_WORDS * N_STREAMS);
  cudaMemset(s->d_stats, 0, sizeof(double) * 2 * channels * s->n_slots);
  memset(s->h_status, 0, sizeof(unsigned) * N_STREAMS);
  ctx_wait_options(ctx, s->spin_limit_ns, s->withhold);
  for (int i = 0; i < N_STREAMS; i++) {
    cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking);
    s->batches[i].svc = s;
    s->batches[i].lane = i;
  }
  cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking);
  s->free_slots.reserve(s->n_slots);
  for (int i = s->n_slots - 1; i >= 0; i--) s->free_slots.push_back(i);
  s->slot_refs.assign(s->n_slots, 0);
  s->beam_slot.assign(n_beams, -1);
  s->beam_seq.assign(n_beams, 0);
  s->beam_chunks.assign(n_beams, 0);
  s->beam_last_latency.assign(n_beams, 0.0);
  s->dispatcher = std::thread(dispatch_loop, s);
  ctx_stream_service(ctx) = s;
  return RFIM_OK;
}

rfim_status rfim_stream_push(rfim_ctx* ctx, int beam, const void* chunk, double arrival_time_s,
                             unsigned long long* ticket) {
  StreamService* s = svc_of(ctx);
  if (!ctx) return RFIM_ERR_ARG;
  if (!s) return RFIM_ERR_STATE;
  if (beam < 0 || beam >= s->n_beams || !chunk || !ticket) return RFIM_ERR_ARG;
  return svc_push(s, beam, chunk, is_device_ptr(chunk), arrival_time_s, ticket);
}

}  // extern "C"

namespace rfim {
namespace {
rfim_status svc_push(StreamService* s, int beam, const void* chunk, bool on_device, double arrival_time_s,
                     unsigned long long* ticket) {
  int slot;
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->free_slots.empty()) return RFIM_ERR_BUSY;
    slot = s->free_slots.back();
    s->free_slots.pop_back();
    s->slot_refs[slot] = 1;  // held by its ticket
  }
  const void* src = chunk;
  if (!on_device) {
    // host chunk: copy it into the slot, cleaned in place there
    unsigned char* dst = s->d_slots + (size_t)slot * s->chunk_bytes;
    const size_t n = s->in_bytes;
    cudaError_t e;
    {
      std::lock_guard<std::mutex> g(s->copy_mu);
      e = cudaMemcpyAsync(dst, chunk, n, cudaMemcpyHostToDevice, s->copy_stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s->copy_stream);
    }
    if (e != cudaSuccess) {
      (void)cudaGetLastError();  // reported by the status: not left for the caller's next call
      std::lock_guard<std::mutex> g(s->mu);
      slot_unref(s, slot);
      return RFIM_ERR_CUDA;
    }
    src = dst;
  }
  unsigned long long id;
  bool wake;
  {
    std::lock_guard<std::mutex> g(s->mu);
    id = s->next_ticket++;
    Ticket k;
    k.slot = slot;
    k.beam = beam;
    k.state = T_WAITING;
    k.status = RFIM_OK;
    k.seq = s->beam_chunks[beam];
    k.src = src;
    k.arrival = arrival_time_s;
    k.done = 0.0;
    s->tickets.emplace(id, k);
    s->waiting.push_back(id);
    s->beam_chunks[beam]++;
    wake = s->disp_waiting;
  }
  if (wake) s->cv_work.notify_one();
  *ticket = id;
  return RFIM_OK;
}
}  // namespace
}  // namespace rfim

extern "C" {

rfim_status rfim_stream_poll(rfim_ctx* ctx, unsigned long long ticket, void** out_dev, void** mask_dev,
                             int wait_us) {
  StreamService* s = svc_of(ctx);
  if (!ctx) return RFIM_ERR_ARG;
  if (!s) return RFIM_ERR_STATE;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return RFIM_ERR_ARG;
  if (it->second.state != T_DONE && wait_us > 0) {
    s->cv_done.wait_for(lk, std::chrono::microseconds(wait_us), [&] {
      auto j = s->tickets.find(ticket);
      return j == s->tickets.end() || j->second.state == T_DONE;
    });
    it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return RFIM_ERR_ARG;
  }
  if (it->second.state != T_DONE) return RFIM_ERR_BUSY;
  if (it->second.status != RFIM_OK) return it->second.status;
  if (out_dev) *out_dev = s->d_slots + (size_t)it->second.slot * s->chunk_bytes;
  if (mask_dev) *mask_dev = s->d_masks + (size_t)it->second.slot * s->mask_bytes;
  return RFIM_OK;
}

rfim_status rfim_stream_release(rfim_ctx* ctx, unsigned long long ticket) {
  StreamService* s = svc_of(ctx);
  if (!ctx) return RFIM_ERR_ARG;
  if (!s) return RFIM_ERR_STATE;
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return RFIM_ERR_ARG;
  if (it->second.state != T_DONE) return RFIM_ERR_BUSY;
  slot_unref(s, it->second.slot);
  s->tickets.erase(it);
  return RFIM_OK;
}

rfim_status rfim_stream_beam_state(rfim_ctx* ctx, int beam, unsigned long long* chunk_index, double* stats,
                                   const void** out_dev, const void** mask_dev) {
  StreamService* s = svc_of(ctx);
  if (!ctx) return RFIM_ERR_ARG;
  if (!s) return RFIM_ERR_STATE;
  if (beam < 0 || beam >= s->n_beams) return RFIM_ERR_ARG;
  int slot;
  {
    std::lock_guard<std::mutex> g(s->mu);
    slot = s->beam_slot[beam];
    if (slot < 0) return RFIM_ERR_BUSY;
    if (chunk_index) *chunk_index = s->beam_seq[beam];
    if (out_dev) *out_dev = s->d_slots + (size_t)slot * s->chunk_bytes;
    if (mask_dev) *mask_dev = s->d_masks + (size_t)slot * s->mask_bytes;
    s->slot_refs[slot]++;  // held while its statistics are copied out
  }
  rfim_status st = RFIM_OK;
  if (stats) {
    cudaError_t e;
    {
      std::lock_guard<std::mutex> g(s->copy_mu);
      e = cudaMemcpyAsync(stats, s->d_stats + (size_t)slot * 2 * s->C, sizeof(double) * 2 * s->C,
                          cudaMemcpyDeviceToHost, s->copy_stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s->copy_stream);
    }
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      st = RFIM_ERR_CUDA;
    }
  }
  std::lock_guard<std::mutex> g(s->mu);
  slot_unref(s, slot);
  return st;
}

rfim_status rfim_stream_replay(rfim_ctx* ctx, int n, const int* beams, const void* const* chunks,
                               const double* arrival_s) {
  StreamService* s = svc_of(ctx);
  if (!ctx) return RFIM_ERR_ARG;
  if (!s) return RFIM_ERR_STATE;
  if (n < 0 || (n > 0 && (!beams || !chunks || !arrival_s))) return RFIM_ERR_ARG;
  std::deque<unsigned long long> out;
  std::unordered_map<const void*, bool> kind;  // pointer -> device memory (classified once)
  for (int i = 0; i < n; i++)
    if (beams[i] < 0 || beams[i] >= s->n_beams || !chunks[i]) return RFIM_ERR_ARG;
  auto reap = [&](bool block) -> rfim_status {
    while (!out.empty()) {
      rfim_status st = rfim_stream_poll(ctx, out.front(), nullptr, nullptr, block ? 1000000 : 0);
      if (st == RFIM_ERR_BUSY) {
        if (block) continue;
        return RFIM_OK;
      }
      if (st != RFIM_OK) return st;
      rfim_stream_release(ctx, out.front());
      out.pop_front();
    }
    return RFIM_OK;
  };
  for (int i = 0; i < n; i++) {
    // wait for the scheduled arrival, reaping completions meanwhile
    for (;;) {
      const double dt = arrival_s[i] - now_mono();
      if (dt <= 0) break;
      rfim_status st = reap(false);
      if (st != RFIM_OK) return st;
      if (dt > 200e-6) std::this_thread::sleep_for(std::chrono::microseconds((long)(dt * 0.5e6)));
    }
    unsigned long long id;
    auto kt = kind.find(chunks[i]);
    if (kt == kind.end()) kt = kind.emplace(chunks[i], is_device_ptr(chunks[i])).first;
    for (;;) {
      rfim_status st = svc_push(s, beams[i], chunks[i], kt->second, arrival_s[i], &id);
      if (st == RFIM_OK) break;
      if (st != RFIM_ERR_BUSY) return st;
      // no slot free: wait for the oldest outstanding chunk
      if (out.empty()) return RFIM_ERR_STATE;
      rfim_status r = rfim_stream_poll(ctx, out.front(), nullptr, nullptr, 1000000);
      if (r == RFIM_OK) {
        rfim_stream_release(ctx, out.front());
        out.pop_front();
      } else if (r != RFIM_ERR_BUSY) {
        return r;
      }
    }
    out.push_back(id);
    if ((i & 31) == 31) {
      rfim_status st = reap(false);
      if (st != RFIM_OK) return st;
    }
  }
  return reap(true);
}

rfim_status rfim_stream_stats(rfim_ctx* ctx, double* p50, double* p99, double* p999, double* gbps,
                              unsigned long long* chunks, int reset) {
  StreamService* s = svc_of(ctx);
  if (!ctx) return RFIM_ERR_ARG;
  if (!s) return RFIM_ERR_STATE;
  std::vector<double> v;
  double bytes, t0, t1;
  {
    std::lock_guard<std::mutex> g(s->mu);
    v = s->lat;
    bytes = s->bytes_done;
    t0 = s->first_arrival;
    t1 = s->last_done;
    if (reset) {
      s->lat.clear();
      s->bytes_done = 0.0;
      s->first_arrival = 0.0;
      s->last_done = 0.0;
    }
  }
  auto pct = [&](double q) -> double {
    if (v.empty()) return 0.0;
    const size_t k = std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5));
    std::nth_element(v.begin(), v.begin() + k, v.end());
    return v[k];
  };
  if (p50) *p50 = pct(0.50);
  if (p99) *p99 = pct(0.99);
  if (p999) *p999 = pct(0.999);
  if (gbps) *gbps = (t1 > t0 && !v.empty()) ? bytes / (t1 - t0) / 1e9 : 0.0;
  if (chunks) *chunks = (unsigned long long)v.size();
  return RFIM_OK;
}

rfim_status rfim_stream_close(rfim_ctx* ctx) {
  if (!ctx) return RFIM_ERR_ARG;
  StreamService*& s = ctx_stream_service(ctx);
  if (!s) return RFIM_ERR_STATE;
  svc_free(s);
  s = nullptr;
  return RFIM_OK;
}

}  // extern "C"
