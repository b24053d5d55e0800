// engine.h -- launch parameters shared by the host runtime and the kernels.
#pragma once
#include <cstdint>

#include "common.cuh"

namespace rfim {

constexpr int MAX_JOBS = 160;      // beams per launch (kernel parameters stay below 32 KB)
constexpr int MAX_SEGS = 2 * MAX_JOBS;
constexpr int FD_ITEM_T = 32;      // time samples per uint8 FDSC work item (one mask word column)
// float32 FDSC work items are one sub-slab (Job::ws = 1, 2, 4 or 8 samples): the
// items that share a 128-byte line of each channel row run side by side.

enum ReplaceKind { REP_MEAN = 0, REP_MEDIAN = 1, REP_RANDOM = 2 };
enum MaskKind { MASK_NONE = 0, MASK_BITS = 1, MASK_BYTES = 2 };

// One sigma cut as the kernels see it.
struct CutDev {
  ExactK2 k2;      // uint8: exact form of fl(k*k)
  double k;        // float32 path
  float k_hi, k_lo;  // float32 path: k as float-float (k_hi + k_lo = k to ~2^-48)
  int iterations;  // 0 = method disabled
  int replace;     // ReplaceKind
  int bin;         // FDSC channels per bin
  int it0;         // index of the first iteration (keys the random draws; round r of the interleaved order)
};

// One beam: C x T samples, BCT (time fastest) or BTC (channel fastest).
struct Job {
  const void* in;   // beam base of the input
  void* out;        // beam base of the output
  void* mask;       // beam base of the mask (uint32 words for bits, bytes for bytes) or null
  const void* src_lo;  // bounds of the input buffer (for guarded vector loads)
  const void* src_hi;
  int C, T;
  // FDSC geometry
  int nb;           // number of bins
  int last_g;       // size of the last bin
  unsigned long long m_full, m_last;  // L / G and L / G_last
  int ws;           // sub-slab width (time samples) of the FDSC tile
  int pitch;        // bytes per tile row (>= C * esize, pitch/4 = 1 mod 32)
  int fd_items;     // number of FDSC work items (ceil(T / 32))
  int rows;         // TDSC rows (C)
  int td_mode;      // uint8: 0 = one warp per row, 8 rows per item; 1 = one row per item, whole CTA;
                    //        2 = one row per item, whole CTA, row read from global memory (no stage);
                    //        3 = a quarter warp per row, 32 rows per item.
                    // float32: 0 = two rows per item, a half CTA each; 1 = one row per item;
                    //          2 = one row per item, read from global memory in every pass (no stage)
  int td_items;     // number of TDSC work items
  int beam;         // index of the beam within its block (keys the random-replacement draws)
  int fd_wide;      // 1: the FDSC tile does not fit; each item cleans its columns one at a time (fd_wide_*)
  double* stats;    // or null: per row, the sum and the sum of squares of the input row ([2 * row], [2 * row + 1]),
                    // written by the first TDSC iteration (the streaming service's per-beam state)
  float* prog;      // or null (float32, fused launches with a bit mask, option "f32_records"): per row and
                    // TDSC iteration, the iteration's cut and replacement value (PROG_FLOATS floats); TDSC
                    // rows record these and their mask bits instead of writing the row, and FDSC items load
                    // the input and replay the cuts on the samples whose TDSC bit is set
};
// per row and iteration: {mu_f, lo_f, hi_f, r} (the float32 decision and the
// replacement), then {mu_lo, thr_hi, thr_lo, 0} (read only inside the band)
constexpr int PROG_FLOATS = 8;

// A run of consecutive queue items: `count` items of one kind for one job.
struct Seg {
  int start;  // first queue index of the run
  int job;
  int kind;   // 0 = TDSC rows, 1 = FDSC items
};

struct Params {
  Job jobs[MAX_JOBS];
  Seg segs[MAX_SEGS];
  int n_jobs, n_segs, n_items;
  CutDev td, fd;
  int mask_kind;
  int fd_reads_out;     // FDSC items read the output buffer (TDSC ran before)
  int wait_tdsc;        // FDSC items wait for their beam's TDSC rows
  int mask_or;          // FDSC ORs its bits into the mask (TDSC wrote it before)
  int withhold_job;     // test hook: job index whose TDSC completion is never published (-1 = none)
  unsigned long long spin_limit_ns;
  unsigned* counters;   // [0] queue head, [1 + j] TDSC rows done for job j
  unsigned* status;     // device status word (0 = ok, 5 = timeout)
  int dtype;            // 0 = uint8 (k_engine_u8), 1 = float32 (k_engine_f32)
  int td_mask_or;       // TDSC rows OR their flags into the mask (interleaved rounds after the first)
};

__host__ __device__ inline int align16i(int x) { return (x + 15) & ~15; }

// Shared memory of one FDSC tile (uint8): ws x pitch tile, per-(t, bin) sums,
// cached medians and byte extremes, per-column sums of D^2 and keep half-widths, item flag bits,
// list of flagged (t, bin) pairs.
// Rows of the per-(t, bin) arrays are padded to nbp = 8 (mod 32) entries, so the
// 8 lanes of 4 neighbouring columns hit 32 distinct banks.
__host__ __device__ inline int fd_nbp(int nb) { return nb + ((8 - nb) % 32 + 32) % 32; }

// Flag bits of an item.  With 32-channel bins and no random replacement, one
// word per (time sample of the item, bin), bit j = channel 32 g + j, each
// written by the one lane that resolves that bin at that sample, and turned
// into per-channel words by a 32 x 32 bit transpose at the end of the item;
// rows of nb | 1 words (odd: the 32 rows of one bin fall in distinct banks).
// Otherwise one word per channel, bit = time sample, set by shared atomics.
__host__ __device__ inline bool fd_bin_bits(int bin, bool rnd) { return bin == 32 && !rnd; }
__host__ __device__ inline int fd_flag_bytes(int C, int nb, bool bin_bits) {
  return align16i((bin_bits ? FD_ITEM_T * (nb | 1) : C) * 4);
}

// rnd: random replacement adds one word per channel (the flags of the
// iteration in progress, bit = tile row); bin: the FDSC bin size
__host__ __device__ inline int fd_smem_bytes(int ws, int pitch, int nb, int C, bool rnd, int bin) {
  const int nbp = fd_nbp(nb);
  return ws * pitch + 2 * align16i(ws * nbp * 4) + 2 * align16i(ws * nbp * 2) + align16i(ws * 8) + align16i(ws * 8) +
         fd_flag_bytes(C, nb, fd_bin_bits(bin, rnd)) + align16i(ws * nb * 4) + 4 * (NT / 32) +
         (rnd ? align16i(C * 4) : 0);
}

// FDSC on columns wider than the tile: a CTA cleans one column (time sample)
// at a time, holding the column, two flag bits per channel (this iteration's,
// and the OR over iterations) and per-bin sums, keep intervals and replacement
// values.
__host__ __device__ inline int fd_wide_smem_u8(int C, int nb) {
  const int W = (C + 31) / 32;
  return align16i(C) + 2 * align16i(W * 4) + 2 * align16i(nb * 8) + 2 * align16i(nb * 4);
}
__host__ __device__ inline int fd_wide_smem_f32(int C, int nb) {
  const int W = (C + 31) / 32;
  return align16i(C * 4) + 2 * align16i(W * 4) + align16i(nb * 8) + align16i(nb * 4);
}

// Tile row pitch: C bytes rounded up to 128, so that the XOR swizzle of the 16-byte
// units of a row (by (row >> 2) & 7) stays inside the row.
__host__ __device__ inline int fd_pitch(int C_bytes) { return ((C_bytes + 127) / 128) * 128; }

// TDSC row staging: a warp stages rows of up to TD_WARP_CHUNKS 16-byte chunks
// (8 warps share TD_WARP_STAGE * 8 bytes); longer rows, up to TD_CTA_CHUNKS
// chunks, are staged and processed by the whole CTA.
// Dynamic shared memory one CTA of the engine may use (227 KB opt-in on sm_103a,
// less 2 KB kept for the kernel's static shared variables).
constexpr int MAX_SMEM_PER_CTA = 232448 - 2048;

constexpr int TD_WARP_CHUNKS = 800;
constexpr int TD_WARP_STAGE = TD_WARP_CHUNKS * 16;
constexpr int TD_CTA_CHUNKS = 6144;
constexpr int TD_ROWS_PER_ITEM = NT / 32;
// uint8 rows are exact up to (255 T)^2 < 2^53
constexpr long long TD_MAX_T = 372181;
// Random replacement keeps two 16-bit flag words per chunk beside the staged
// row (this iteration's flags, and the OR over iterations): warp rows up to 640
// chunks, longer rows (up to 4915 chunks) by the whole CTA.  Longer rows are
// not staged (mode 2): their two flag bitmaps, one bit per sample, take the
// CTA stage, up to the exactness bound of the uint8 decisions.
__host__ __device__ inline int td_random_row_mode(long long T) {
  const long long nch = (T + 30) / 16 + 1;
  if (20 * nch <= TD_WARP_STAGE) return 0;
  if (20 * nch <= TD_CTA_CHUNKS * 16) return 1;
  if (T <= TD_MAX_T && 2 * 4 * ((T + 31) / 32) <= TD_CTA_CHUNKS * 16) return 2;
  return -1;
}

// Row mode for rows of T bytes: 0 = warp rows, 1 = CTA rows, -1 = too long.
// TDSC rows longer than the CTA stage are read from global memory in every
// pass (mode 2), up to the exactness bound of the uint8 decisions,
// (255 T)^2 < 2^53.
// Rows of up to TD_QUAD_CHUNKS chunks (about 3,150 samples) take a quarter warp
// each, four rows per warp in a quarter of the warp's stage (mode 3), so that
// the per-row steps (thresholds, reductions) are shared by fewer lanes.
constexpr int TD_QUAD_CHUNKS = TD_WARP_CHUNKS / 4;
constexpr int TD_MBARS = NT / 32 + NT / 8 + 1;  // staging mbarriers: warps, quarter warps, the CTA
inline int td_row_mode(long long T) {
  const long long nch = (T + 30) / 16 + 1;  // worst-case alignment of the row start
  if (nch <= TD_QUAD_CHUNKS) return 3;
  if (nch <= TD_WARP_CHUNKS) return 0;
  if (nch <= TD_CTA_CHUNKS) return 1;
  if (T <= TD_MAX_T) return 2;
  return -1;
}

// Launchers (engine_u8.cu).
struct LaunchCfg {
  int grid;
  int smem;
};
int engine_smem_u8(const Params& p);
void* engine_kernel_u8(const Params& p);
int launch_engine_u8(const Params& p, const LaunchCfg& cfg, void* stream);

// float32 engine: TDSC rows of up to TD32_MAX_T samples staged per CTA (longer rows
// are read from memory in every pass); FDSC tile
// of ws x C floats plus per-(t, bin) and per-column scratch.
constexpr int TD32_LIST = 1024;  // replaced values kept per iteration for the statistics update
constexpr int TD32_MAX_T = 52000;
// float32 rows beyond the stage with random replacement: two flag bitmaps,
// one bit per sample, in shared memory
__host__ __device__ inline int td32_rnd_long_bytes(long long T) { return (int)(8 * ((T + 31) / 32)); }
__host__ __device__ inline int td32_smem_bytes(int T) {
  const int nch = (T + 6) / 4 + 1;
  return 16 * nch + align16i(nch) + 4 * TD32_LIST;
}
// rnd: random replacement adds one flag word per channel; prog: one word per
// channel holds the TDSC mask word of the sub-slab (replay of TDSC's cut records)
__host__ __device__ inline int fd32_smem_bytes(int ws, int C, int nb, bool rnd = false, bool prog = false) {
  const int U = ws * nb;
  return align16i(ws * C * 4) + align16i(C * 4) + align16i(U * 8) * 2 + align16i(U * 4) + align16i(ws * 8) +
         align16i(ws * 4) * 2 + (rnd ? align16i(C * 4) : 0) + (prog ? align16i(C * 4) : 0);
}
int engine_smem_f32(const Params& p);
void* engine_kernel_f32(const Params& p);
int launch_engine_f32(const Params& p, const LaunchCfg& cfg, void* stream);

// layout conversion (transpose.cu): out[b][c][r] = in[b][r][c] for rows x cols
// planes of esize-byte elements; bit masks from BCT rows (c) to BTC rows (t).
int launch_transpose(const void* in, void* out, int batch, int rows, int cols, int esize, void* stream);
int launch_transpose_bits(const void* in_bct, void* out_btc, int batch, int C, int T, void* stream);

inline int engine_smem(const Params& p) { return p.dtype ? engine_smem_f32(p) : engine_smem_u8(p); }
inline void* engine_kernel(const Params& p) { return p.dtype ? engine_kernel_f32(p) : engine_kernel_u8(p); }
inline int launch_engine(const Params& p, const LaunchCfg& cfg, void* stream) {
  return p.dtype ? launch_engine_f32(p, cfg, stream) : launch_engine_u8(p, cfg, stream);
}

}  // namespace rfim
