// engine_u8.cu -- the mean/median build of the uint8 engine (kernel
// k_engine_u8<2, false>) and its host-side helpers.  The device code is in
// engine_u8_impl.cuh; the build with random replacement is engine_u8_rnd.cu.
#include <cstdint>
#include <cstdio>

#include "engine_u8_impl.cuh"

namespace rfim {

void* engine_kernel_u8_rnd();  // engine_u8_rnd.cu

// ---------------------------------------------------------------------------
// host-side helpers
// ---------------------------------------------------------------------------
int engine_smem_u8(const Params& p) {
  int s = 16;
  for (int j = 0; j < p.n_jobs; j++) {
    const Job& J = p.jobs[j];
    if (p.td.iterations > 0) {
      const int td = (J.td_mode == 0 || J.td_mode == 3) ? TD_WARP_STAGE * TD_ROWS_PER_ITEM : TD_CTA_CHUNKS * 16;
      s = s > td ? s : td;
    }
    if (p.fd.iterations > 0) {
      const int fd = J.fd_wide ? fd_wide_smem_u8(J.C, J.nb)
                               : fd_smem_bytes(J.ws, J.pitch, J.nb, J.C, p.fd.replace == REP_RANDOM, p.fd.bin);
      s = s > fd ? s : fd;
    }
  }
  return align16i(s);
}

void* engine_kernel_u8(const Params& p) {
  const bool rnd = (p.td.iterations > 0 && p.td.replace == REP_RANDOM) ||
                   (p.fd.iterations > 0 && p.fd.replace == REP_RANDOM);
  return rnd ? engine_kernel_u8_rnd() : (void*)k_engine_u8<2, false>;
}

int launch_engine_u8(const Params& p, const LaunchCfg& cfg, void* stream) {
  void* args[] = {const_cast<Params*>(&p)};
  return (int)cudaLaunchKernel(engine_kernel_u8(p), dim3(cfg.grid), dim3(NT), args, (size_t)cfg.smem,
                               (cudaStream_t)stream);
}

}  // namespace rfim
