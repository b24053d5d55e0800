// noalloc.cu -- rfim_clean_noalloc: the cleaner for callers that cannot allocate.
//
// The engine needs a little device scratch: the work-queue head, one completion
// counter per beam and a status word.  rfim_clean takes it from its context,
// which allocates it with cudaMalloc.  This entry point instead uses a
// file-scope __device__ array, which every GPU that loads the library holds
// until the process exits, so a call allocates nothing, on the device or the host.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/rfim.h"
#include "engine.h"
#include "runtime.h"

namespace rfim {
namespace {

constexpr int NOALLOC_MAX_DEVICES = 64;
constexpr int NOALLOC_WORDS = 1 + MAX_JOBS + 1;  // queue head, per-beam counters, status word
static_assert(MAX_JOBS == RFIM_NOALLOC_MAX_BEAMS, "beam limit of the no-allocation entry point");

// The shared scratch of every rfim_clean_noalloc call on a device.
static __device__ __align__(256) unsigned g_noalloc_scratch[NOALLOC_WORDS];

std::mutex g_mu;
// Device address of g_noalloc_scratch per device.  In host code the array's name
// is only a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress, once per device, with that device current.
unsigned* g_scratch[NOALLOC_MAX_DEVICES];

}  // namespace
}  // namespace rfim

using namespace rfim;

namespace rfim {
namespace {
// The scratch array's device address on the current device (looked up once per device).
rfim_status noalloc_scratch(unsigned** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RFIM_ERR_CUDA;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return RFIM_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return RFIM_ERR_CUDA;
    g_scratch[dev] = static_cast<unsigned*>(p);
  }
  *out = g_scratch[dev];
  return RFIM_OK;
}
}  // namespace
}  // namespace rfim

extern "C" rfim_status rfim_clean_noalloc(const rfim_block* blk, const rfim_cut* tdsc, const rfim_cut* fdsc,
                                          void* stream) {
  unsigned* scratch = nullptr;
  const rfim_status s = noalloc_scratch(&scratch);
  if (s != RFIM_OK) return s;
  return noalloc_clean(blk, tdsc, fdsc, scratch, scratch + 1 + MAX_JOBS, (cudaStream_t)stream);
}

// The status word is the last of the shared array: read it after `stream`'s
// work, then clear it, with plain synchronous copies to and from a host
// variable (no allocation).
extern "C" rfim_status rfim_noalloc_status(void* stream) {
  unsigned* scratch = nullptr;
  rfim_status s = noalloc_scratch(&scratch);
  if (s != RFIM_OK) return s;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
    (void)cudaGetLastError();
    return RFIM_ERR_CUDA;
  }
  unsigned word = 0;
  const unsigned zero = 0;
  if (cudaMemcpy(&word, scratch + 1 + MAX_JOBS, sizeof word, cudaMemcpyDeviceToHost) != cudaSuccess ||
      (word && cudaMemcpy(scratch + 1 + MAX_JOBS, &zero, sizeof zero, cudaMemcpyHostToDevice) != cudaSuccess)) {
    (void)cudaGetLastError();
    return RFIM_ERR_CUDA;
  }
  return word ? RFIM_ERR_TIMEOUT : RFIM_OK;
}
