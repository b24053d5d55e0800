// runtime.h -- host runtime pieces around the kernels: host-buffer staging,
// autotuner and the streaming (continuous-batching) service.
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "../../include/rfim.h"

namespace rfim {

struct HostStager;
struct StreamService;
struct Tuner;

// Options of the context that the tuner chooses.
struct Tunables {
  int schedule;     // 0 auto, 1 fused, 2 separate launches
  int ctas_per_sm;  // 0 = occupancy maximum
  int smem_target;  // bytes of shared memory an FDSC tile may use
  int fused_lag;    // beams of TDSC queued ahead of a beam's FDSC items
};

// context accessors (api.cu)
rfim_status ctx_clean_async(rfim_ctx* ctx, const rfim_block* blocks, int n, const rfim_cut* tdsc,
                            const rfim_cut* fdsc, cudaStream_t st);
int ctx_device(rfim_ctx* ctx);
size_t ctx_hbm_budget(rfim_ctx* ctx);
void ctx_set_error(rfim_ctx* ctx, const char* msg);
// a device (or, with pinned_host, page-locked host) allocation on behalf of the
// context; fails without allocating while the "fail_alloc_after" hook says so
cudaError_t ctx_malloc(rfim_ctx* ctx, void** p, size_t bytes, bool pinned_host = false);
StreamService*& ctx_stream_service(rfim_ctx* ctx);
void ctx_get_tunables(rfim_ctx* ctx, Tunables& t);
// host staging: bytes per group and streams in the ring
void ctx_stage_options(rfim_ctx* ctx, size_t& group_bytes, int& streams);
// validation of one block and its cuts as a launch would do it (no launch)
rfim_status ctx_validate(rfim_ctx* ctx, const rfim_block* b, const rfim_cut* tdsc, const rfim_cut* fdsc);
void ctx_set_tunables(rfim_ctx* ctx, const Tunables& t);

// host staging (runtime.cu)
HostStager* stager_create(rfim_ctx* ctx);
void stager_destroy(HostStager* s);
rfim_status stager_run(HostStager* s, rfim_ctx* ctx, const rfim_block* host_blk, const rfim_cut* tdsc,
                       const rfim_cut* fdsc);

// autotuner (runtime.cu)
Tuner* tuner_create(const std::string& cache_path);
void tuner_destroy(Tuner* t);
rfim_status tuner_apply(Tuner* t, rfim_ctx* ctx, const rfim_block* blocks, int n, const rfim_cut* tdsc,
                        const rfim_cut* fdsc);

// planning and launch with caller-provided counters, no allocation (api.cu):
// one launch over the blocks (at most 160 beams in all, same dtype, layout and
// mask format), default tuning; `counters` holds 1 + 160 words, `status` one.
rfim_status noalloc_clean(const rfim_block* b, const rfim_cut* tdsc, const rfim_cut* fdsc, unsigned* counters,
                          unsigned* status, cudaStream_t st);
// stats (nullable): per block, a device array of 2 doubles per (beam, channel)
// row that the first TDSC iteration fills with the input row's sum and sum of
// squares; spin_limit_ns bounds every device-side wait; withhold_job (-1 =
// none) is the test hook of rfim_set_option("withhold_tdsc_done").
rfim_status launch_blocks_fixed(const rfim_block* blocks, int n, const rfim_cut* tdsc, const rfim_cut* fdsc,
                                unsigned* counters, unsigned* status, cudaStream_t st, double* const* stats = nullptr,
                                unsigned long long spin_limit_ns = 2000000000ull, int withhold_job = -1);
// the context's spin limit (ns) and withhold test hook (-1 = off), as the next launch would use them
void ctx_wait_options(rfim_ctx* ctx, unsigned long long& spin_limit_ns, int& withhold_job);

// streaming service (stream.cu)
void stream_service_destroy(StreamService* s);
// batches of the service whose device-side wait gave up since the last call (clears the count)
unsigned long long stream_service_take_timeouts(StreamService* s);

}  // namespace rfim
