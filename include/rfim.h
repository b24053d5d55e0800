/*
 * rfim.h -- C ABI of the GB300 (sm_103a) RFI mitigation library, librfim.so.
 *
 * The library cleans radio filterbanks (beam x channel x time intensities) with
 * the two thresholding methods of Sclocco, Vohl and van Nieuwpoort, "Real-Time
 * RFI Mitigation for the Apertif Radio Transient System" (arXiv:2001.03389):
 *
 *   TDSC, time-domain sigma cut (Sec. IV, TDSC paragraph; Fig. 2): for every
 *     (beam, channel), the mean mu and standard deviation sigma of the batch's
 *     time samples are computed; a sample with |x - mu| > k sigma (the test is
 *     symmetric, Fig. 2 caption) is flagged and replaced.
 *   FDSC, frequency-domain sigma cut (Sec. IV, FDSC paragraph; Fig. 3): for
 *     every (beam, time sample), channels are grouped into bins of `fdsc_bin`
 *     channels; each value minus its bin mean is compared with the mean and
 *     standard deviation of these mean-corrected values over all channels; an
 *     outlier's original value is replaced by its bin's replacement value.
 *   Replacement strategy (Sec. IV, last paragraph): the mean, or the median.
 *   Iterations (Sec. V-A: three in production): the cut is re-run on its own
 *     output, statistics recomputed from the current values.
 *   Cleaning happens in device memory and, out of place, leaves the input
 *     untouched (Sec. VI).
 *
 * Definitions the paper leaves open, as implemented (bit-exact for uint8):
 *   - sigma is the population deviation (divide by the count);
 *   - uint8 decisions are exact: TDSC flags iff
 *       (double)((T x - S)^2) > fl(k2 * (double)(T Q - S^2)),  S = sum x, Q = sum x^2,
 *     FDSC flags iff (double)(C D^2) > fl(k2 * (double)sum D^2),
 *       D = (L / G_g)(G_g x - S_g), L = lcm of the bin sizes,
 *     where k2 = fl(k * k) and fl() is one IEEE double rounding;
 *   - float32 decisions are those of the IEEE double expression
 *       fabs((double)x - mu) > k * sigma,   sigma = sqrt(sum (x - mu)^2 / n)
 *     (FDSC: x - mu replaced by the deviation from the bin mean, whose mean
 *     over the channels is 0); the library takes its sums in compensated
 *     float32 arithmetic and evaluates samples near the threshold in double,
 *     so it agrees with a plain double evaluation except for samples within
 *     about 1e-12 relative of k sigma.  float32 input must be finite;
 *   - uint8 mean replacement rounds half up, floor((2S + n) / (2n));
 *     float32 mean replacement is (float) of the double mean;
 *   - the median is the lower median (rank floor((n-1)/2), 0-based) of the
 *     current values of the row (TDSC) or bin (FDSC);
 *   - FDSC bins are contiguous channel groups [g*bin, (g+1)*bin), the last one
 *     possibly shorter; fdsc_bin == channels is one bin (bandpass corrected);
 *   - rfim_clean runs all TDSC iterations on every row, then all FDSC
 *     iterations on every column of the TDSC output.
 *
 * Row lengths: uint8 TDSC takes rows up to 372,181 samples, where (255 T)^2
 * reaches 2^53 (RFIM_ERR_RANGE beyond); rows longer than 98,273 samples do not
 * fit the on-chip stage and are read from memory in every pass (slower, same
 * results).  float32 TDSC rows longer than 52,000 samples are read from memory
 * in every pass, replaying the earlier iterations' decisions.  With random
 * replacement, uint8 rows longer than 78,609 samples and float32 rows longer
 * than 52,000 are not staged either: iteration 0 writes the output row and
 * later iterations rewrite it in place, with the flags kept as bitmaps in
 * shared memory (uint8 up to the 372,181 bound above, float32 up to 921,600
 * samples; RFIM_ERR_ARG beyond).
 *
 * Column heights: FDSC cleans tiles of 8 to 32 time samples x all channels in
 * shared memory.  Beams whose tile does not fit (uint8: about 14,700 channels
 * in 32-channel bins; float32: about 26,700) are cleaned one column at a time,
 * the column gathered into shared memory (slower, same results), up to 115,200
 * uint8 or 49,800 float32 channels in 32-channel bins (fewer with smaller bins:
 * per bin the column layout keeps its sums and replacement value);
 * RFIM_ERR_RANGE beyond.
 *
 * Conventions for every call below:
 *   - Pointers inside rfim_block are DEVICE pointers owned by the caller,
 *     except for rfim_clean_host.  `out == in` cleans in place; any other
 *     overlap of out with in is RFIM_ERR_ARG.
 *   - Calls are asynchronous on the given CUDA stream (a cudaStream_t passed as
 *     void*, NULL = legacy default stream) unless stated otherwise.  Errors are
 *     returned as status codes, never thrown; rfim_last_error(ctx) holds a
 *     message for the last failing call on that context.
 *   - A context is not thread-safe, except for the rfim_stream_* family, whose
 *     calls may come from any thread.
 *   - Device memory the context needs (work queues, descriptors, staging and
 *     streaming slots) is owned by the context and freed by rfim_destroy.
 */
#ifndef RFIM_H
#define RFIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RFIM_OK = 0,
  RFIM_ERR_ARG = 1,     /* invalid argument (null pointer, bad size, bad enum, overlap) */
  RFIM_ERR_RANGE = 2,   /* shape outside the exact-integer range of the uint8 decisions, or a
                           column too tall for shared memory (see "Column heights") */
  RFIM_ERR_OOM = 3,     /* a device or pinned-host allocation failed */
  RFIM_ERR_CUDA = 4,    /* a CUDA runtime call failed (message in rfim_last_error) */
  RFIM_ERR_TIMEOUT = 5, /* a bounded device-side wait gave up (see rfim_device_status) */
  RFIM_ERR_BUSY = 6,    /* streaming: result not ready, or no slot / memory to admit */
  RFIM_ERR_STATE = 7    /* call not valid in the current context state */
} rfim_status;

typedef enum { RFIM_U8 = 0, RFIM_F32 = 1 } rfim_dtype;

/* BCT: x[b][c][t], time fastest ("channel-major").  BTC: x[b][t][c], channel fastest. */
/*
 * Layouts: BCT = [beam][channel][time] (time fastest: TDSC rows contiguous);
 * BTC = [beam][time][channel] (channels fastest).  The kernels work on BCT; a
 * BTC block is transposed on the device into a context-owned BCT scratch copy,
 * cleaned there and transposed back (three reads and writes of the block in
 * all), with identical results.  rfim_clean_batch runs BTC blocks one after
 * the other without graph capture; rfim_clean_noalloc and the streaming
 * service take BCT only.
 */
typedef enum { RFIM_LAYOUT_BCT = 0, RFIM_LAYOUT_BTC = 1 } rfim_layout;

/*
 * Replacement strategies (Sec. IV, last paragraph): the mean, the lower median,
 * or a random unflagged sample.  RANDOM: a flagged sample takes the current
 * value of an unflagged sample of the same row (TDSC) or bin (FDSC), found by
 * rejection sampling: attempt a = 0..31 draws position
 *   u = ((h >> 32) * n) >> 32,  h = M(M(M(M(beam) ^ line) ^ index) ^ (method << 8 | it << 16 | a << 24)),
 * with M the SplitMix64 output function (Steele, Lea, Flood 2014: z += 0x9E3779B97F4A7C15,
 * then the two xor-shift-multiply rounds), n the row length (TDSC) or bin
 * size (FDSC, u relative to the bin's first channel), method 1 = TDSC (line =
 * channel, index = time sample), 2 = FDSC (line = time sample, index =
 * channel), beam = the beam's index within its block, it = the iteration; the
 * first draw that hits an unflagged sample wins, and after 32 misses the
 * sample keeps its value.  In the interleaved order ("order" option) round r
 * is iteration r of each method and draws with it = r.  Row lengths with
 * RANDOM: see "Row lengths" above.
 */
typedef enum { RFIM_REPLACE_MEAN = 0, RFIM_REPLACE_MEDIAN = 1, RFIM_REPLACE_RANDOM = 2 } rfim_replace;

/*
 * Flag-mask output.
 *   BITS:  one bit per sample along the fastest axis of the layout.  With
 *          R = beams * (slow axes) rows of N samples (N = samples for BCT,
 *          channels for BTC), sample i of row r is bit i % 32 of uint32 word
 *          r * ceil(N / 32) + i / 32; padding bits are 0.  The bit is the OR of
 *          both methods and all iterations.  Needs a 4-byte aligned pointer.
 *   BYTES: one byte per sample, same layout as the data; bit 0 = flagged by
 *          TDSC, bit 1 = flagged by FDSC (any iteration).
 */
typedef enum { RFIM_MASK_NONE = 0, RFIM_MASK_BITS = 1, RFIM_MASK_BYTES = 2 } rfim_mask_fmt;

/* One sigma cut.  k: any finite k > 0, iterations 1..16,
 * fdsc_bin: FDSC channels per bin, 1..channels (0 means 32, capped at channels);
 * ignored by TDSC. */
typedef struct {
  double k;
  int iterations;
  rfim_replace replace;
  int fdsc_bin;
} rfim_cut;

/* A block of `beams` beams of channels x samples, contiguous in the given layout. */
typedef struct {
  const void* in;  /* input intensities (uint8 or float32) */
  void* out;       /* cleaned output, same shape; may equal in */
  void* mask;      /* flag mask in mask_fmt, or NULL */
  int beams, channels, samples;
  rfim_dtype dtype;
  rfim_layout layout;
  rfim_mask_fmt mask_fmt;
} rfim_block;

typedef struct rfim_ctx rfim_ctx;

/*
 * Create a context on CUDA device `device`.
 *   hbm_budget_bytes: device memory the streaming service may hold for its
 *     slots (0 = no limit beyond what is free).
 *   tune_cache: path of the autotuner's JSON cache (read if present, written
 *     after tuning), or NULL for no persistence.
 * Returns RFIM_ERR_ARG for a null ctx or bad device, RFIM_ERR_CUDA if the
 * device cannot be used.
 */
rfim_status rfim_create(rfim_ctx** ctx, int device, size_t hbm_budget_bytes, const char* tune_cache);

/* Synchronise the context's work, free everything it owns, destroy it.  NULL is a no-op. */
rfim_status rfim_destroy(rfim_ctx* ctx);

/*
 * Set a tuning or test option (returns RFIM_ERR_ARG for an unknown key):
 *   "spin_limit_us"   limit of every device-side wait, microseconds (default 2e6);
 *   "schedule"        0 = auto (fused, or separate launches when every uint8
 *                     row takes a quarter warp: rows of at most ~3,150 samples),
 *                     1 = fused persistent (L2-resident re-read),
 *                     2 = separate launches (TDSC pass, then FDSC pass);
 *   "tile_samples"    FDSC tile width in time samples: 0 (automatic) or 1, 2, 4, 8, 16, 32
 *                     (uint8 tiles use at least 8, float32 tiles at most 8);
 *   "smem_target"     shared memory an FDSC tile may use, bytes (sets the automatic width);
 *   "fused_lag"       beams of TDSC rows queued ahead of a beam's FDSC items (0..8);
 *   "stage_group_bytes"  rfim_clean_host: bytes of beams copied and cleaned per
 *                     group (default 32 MB; at least one beam per group);
 *   "stage_streams"   rfim_clean_host: CUDA streams the groups rotate over (1..4, default 3);
 *   "f32_records"     float32 fused launches: 1 = TDSC writes per-row cut records
 *                     (band and replacement value per iteration) instead of its
 *                     output, and FDSC replays them as it loads each tile (same
 *                     results; less traffic, more arithmetic); 0 = off (default);
 *   "order"           order of the methods in rfim_clean and rfim_clean_batch:
 *                     0 = blocked (all TDSC iterations on every row, then all
 *                     FDSC iterations on every column; default), 1 = interleaved
 *                     (round i: TDSC iteration i on every row, then FDSC
 *                     iteration i on every column; single-iteration launches);
 *   "ctas_per_sm"     persistent-kernel CTAs per SM (0 = occupancy maximum);
 *   "withhold_tdsc_done"  test hook: 1 makes the fused kernel never publish the
 *                     TDSC completion of beam 0, so its FDSC items time out
 *                     (RFIM_ERR_TIMEOUT via rfim_device_status);
 *   "fail_alloc_after"  test hook: n >= 0 lets the context's next n device or
 *                     pinned-host allocations succeed and refuses every later
 *                     one (the call returns RFIM_ERR_OOM, nothing is allocated,
 *                     and the context stays usable) until the option is set
 *                     to -1 (off, the default).  It covers every allocation
 *                     after rfim_create: BTC scratch, graph counters, float32
 *                     cut records, host staging, autotuner scratch and the
 *                     streaming slots.
 */
rfim_status rfim_set_option(rfim_ctx* ctx, const char* key, long long value);

/*
 * TDSC on every (beam, channel) row of the block (Sec. IV, Fig. 2).
 * Writes out (all samples) and mask (TDSC flags), asynchronously on stream.
 */
rfim_status rfim_tdsc(rfim_ctx* ctx, const rfim_block* blk, const rfim_cut* cut, void* stream);

/* FDSC on every (beam, time) column of the block (Sec. IV, Fig. 3). */
rfim_status rfim_fdsc(rfim_ctx* ctx, const rfim_block* blk, const rfim_cut* cut, void* stream);

/*
 * TDSC (all iterations) then FDSC (all iterations).  By default one persistent
 * kernel whose FDSC work items re-read each beam's TDSC output while it is
 * resident in L2; blocks whose rows are all short (at most ~3,150 samples)
 * run as two launches, TDSC then FDSC, which is faster there (option
 * "schedule").  Either cut may be NULL to skip that method.
 */
rfim_status rfim_clean(rfim_ctx* ctx, const rfim_block* blk, const rfim_cut* tdsc, const rfim_cut* fdsc,
                       void* stream);

/* flags for rfim_clean_batch */
#define RFIM_BATCH_GRAPH 1u    /* capture the launch in a CUDA graph, replay it when the batch repeats */
#define RFIM_BATCH_AUTOTUNE 2u /* time candidate tilings per shape on first use, cache the winner */

/*
 * Clean n blocks of possibly different shapes (same dtype and layout) in one
 * persistent launch with a device work queue (ragged batching; two launches,
 * TDSC then FDSC, when every row is short, and a launch per 160 beams).
 * Results equal n separate rfim_clean calls bit for bit.  The descriptor table is uploaded
 * with the launch; with RFIM_BATCH_GRAPH the upload and launch are captured
 * once per distinct batch (same pointers and shapes) and replayed afterwards.
 */
rfim_status rfim_clean_batch(rfim_ctx* ctx, const rfim_block* blocks, int n, const rfim_cut* tdsc,
                             const rfim_cut* fdsc, unsigned flags, void* stream);

/*
 * rfim_clean on HOST buffers (pinned memory recommended): the context copies
 * beams to device staging buffers, cleans them and copies results back,
 * overlapping the copies of one beam group with the cleaning of another on a
 * ring of streams ("stage_group_bytes", "stage_streams").  Synchronous:
 * returns when out and mask are written.
 */
rfim_status rfim_clean_host(rfim_ctx* ctx, const rfim_block* host_blk, const rfim_cut* tdsc,
                            const rfim_cut* fdsc);

/*
 * rfim_clean for callers that cannot allocate memory.  The paper has no
 * counterpart: this entry point exists for host code that must not call
 * cudaMalloc -- a real-time pipeline that reserves all device memory at start
 * and forbids allocation in its processing loop, or a plugin inside a framework
 * that owns the allocator and gives this code no context object.
 *
 * Same arguments and results as rfim_clean (TDSC then FDSC, either cut may be
 * NULL), on the CURRENT CUDA device, asynchronously on `stream`, with default
 * tuning.  No context: the work-queue counters live in a fixed device array
 * inside the library (1 + RFIM_NOALLOC_MAX_BEAMS + 1 words per device, held
 * by every device that loads the library until the process exits).
 *   - At most RFIM_NOALLOC_MAX_BEAMS beams per call; more returns RFIM_ERR_RANGE.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) and caches it; make that first call before any
 *     stream capture on the device.
 *   - Every call on a device shares the array and clears it on its stream
 *     first.  Calls whose work overlaps on the GPU (different streams without
 *     ordering) race on it and must not be issued; order them on one stream.
 *   - A device-side wait that gives up (after 2 s) leaves its output
 *     incomplete and sets a status word in the same array; the call itself
 *     has already returned, so read the word with rfim_noalloc_status.
 *   - Calls no cudaMalloc, cudaFree or other allocating routine.
 */
#define RFIM_NOALLOC_MAX_BEAMS 160
rfim_status rfim_clean_noalloc(const rfim_block* blk, const rfim_cut* tdsc, const rfim_cut* fdsc, void* stream);

/*
 * Status of the latest rfim_clean_noalloc call on the CURRENT device (each
 * call clears the word on its stream first): synchronises `stream` (the one
 * that call used), reads the shared array's status word and clears it.
 * RFIM_OK, or RFIM_ERR_TIMEOUT if a device-side wait of that call gave up.
 * Allocates nothing either (the word is copied to a host variable); like the
 * calls it reports on, it must not overlap other rfim_clean_noalloc work on
 * the device.
 */
rfim_status rfim_noalloc_status(void* stream);

/*
 * Synchronise `stream` and return the device status word of the context's
 * kernels since the last check: RFIM_OK, or RFIM_ERR_TIMEOUT if a device-side
 * wait gave up (the affected output is then incomplete).  Clears the word.
 * Batches of the streaming service that timed out since the last check (their
 * chunks complete with RFIM_ERR_TIMEOUT) are reported here too, and cleared.
 */
rfim_status rfim_device_status(rfim_ctx* ctx, void* stream);

/* ------------------------------------------------------------------------ */
/* Streaming service (continuous batching of beam chunks).                   */
/* Each chunk is one batch in the paper's sense (Sec. IV): its statistics come */
/* from the chunk alone, so a chunk's result is the same alone or in a mix.  */
/* ------------------------------------------------------------------------ */

/*
 * Open the streaming service: n_beams beams of `channels` x `chunk_samples`
 * chunks (BCT layout per chunk) of dtype, cleaned with the given cuts (either
 * may be NULL; rfim_clean semantics, bit mask output).
 *   - Slots: each holds one chunk's cleaned output and bit mask in device
 *     memory.  As many are allocated as the context's HBM budget allows
 *     (rfim_create; 0 = a quarter of the free device memory), at most four per
 *     beam.  A chunk is admitted only when a slot is free.
 *   - A dispatcher thread launches everything waiting (up to 160 chunks) as
 *     one micro-batch (TDSC and FDSC as two launches for short chunks) on
 *     whichever of four CUDA streams is idle, so batches
 *     overlap on the device; completion is signalled from the stream.
 *   - Per-beam state on the device: each beam keeps the slot of its latest
 *     completed chunk (cleaned data, mask and the per-channel statistics of
 *     its input, see rfim_stream_beam_state) until a newer chunk of the beam
 *     completes; at most half of the slots are held this way.  Statistics of
 *     earlier chunks never enter a decision (each chunk is its own batch).
 *   - The options "spin_limit_us" and "withhold_tdsc_done" in force at open
 *     apply to the service's launches.
 * Returns RFIM_ERR_STATE if the service is already open, RFIM_ERR_OOM if not
 * even one slot fits.
 */
rfim_status rfim_stream_open(rfim_ctx* ctx, int n_beams, int channels, int chunk_samples, rfim_dtype dtype,
                             const rfim_cut* tdsc, const rfim_cut* fdsc);

/*
 * Submit one chunk of beam `beam` (0 <= beam < n_beams).
 *   chunk: a DEVICE pointer is read in place by the kernels (zero copy): its
 *     contents must be complete when the call is made and stay unchanged
 *     until the ticket completes.  A HOST pointer is copied into the slot
 *     before the call returns.
 *   arrival_time_s: the chunk's scheduled arrival on the CLOCK_MONOTONIC
 *     scale, seconds; latency is measured from it (so a late push counts).
 * Returns RFIM_ERR_BUSY if no slot is free (retry after releasing tickets),
 * RFIM_ERR_STATE if the service is not open.
 */
rfim_status rfim_stream_push(rfim_ctx* ctx, int beam, const void* chunk, double arrival_time_s,
                             unsigned long long* ticket);

/*
 * Poll a ticket.  When cleaned, *out_dev and *mask_dev (bit mask, one row of
 * ceil(chunk_samples / 32) words per channel) point to context-owned device
 * memory valid until rfim_stream_release.  wait_us: how long to wait for
 * completion (0 = do not wait).  Returns RFIM_ERR_BUSY if not done in time,
 * RFIM_ERR_ARG for an unknown ticket, and for a chunk whose batch failed the
 * reason (RFIM_ERR_TIMEOUT: a device-side wait of its launch gave up, so its
 * output is incomplete; the ticket must still be released).
 */
rfim_status rfim_stream_poll(rfim_ctx* ctx, unsigned long long ticket, void** out_dev, void** mask_dev,
                             int wait_us);

/* Return a completed ticket's slot to the pool (RFIM_ERR_BUSY while it is in flight). */
rfim_status rfim_stream_release(rfim_ctx* ctx, unsigned long long ticket);

/*
 * The per-beam state the service keeps on the device: beam `beam`'s latest
 * completed chunk (the newest by push order among those cleaned so far).
 *   chunk_index (nullable): that chunk's index among the beam's pushes (0, 1, ...).
 *   stats (nullable, host memory of 2 * channels doubles): for each channel c,
 *     stats[2c] = sum over the chunk's samples of the INPUT value and
 *     stats[2c + 1] = the sum of their squares, as the first TDSC iteration
 *     found them (exact for uint8; float-float sums rounded to double for
 *     float32); zeros when the service runs no TDSC.  Copied synchronously.
 *   out_dev / mask_dev (nullable): that chunk's cleaned data and bit mask in
 *     device memory, valid until the beam's next chunk completes.
 * The statistics are records for the caller (mean S/T, variance Q/T - mean^2
 * of each channel in the previous chunk); the cleaning never reads them.
 * Returns RFIM_ERR_BUSY while the beam has no completed chunk (or no state
 * slot was free for it), RFIM_ERR_ARG for a bad beam, RFIM_ERR_STATE if the
 * service is not open.
 */
rfim_status rfim_stream_beam_state(rfim_ctx* ctx, int beam, unsigned long long* chunk_index, double* stats,
                                   const void** out_dev, const void** mask_dev);

/*
 * Replay an arrival schedule through the open service: chunk i (of beam
 * beams[i], pointer chunks[i]) is pushed at its scheduled time arrival_s[i]
 * (CLOCK_MONOTONIC seconds, non-decreasing; the call waits until then, or
 * pushes at once when behind schedule), completed tickets are released as it
 * goes, and the call returns when all n are done.  A load generator for
 * recorded or simulated arrivals; latencies accumulate in rfim_stream_stats.
 */
rfim_status rfim_stream_replay(rfim_ctx* ctx, int n, const int* beams, const void* const* chunks,
                               const double* arrival_s);

/*
 * Latency percentiles (seconds, from scheduled arrival to completion seen by
 * the service) over the chunks completed since rfim_stream_open or the last
 * reset, their count, and their input GB/s (input bytes / time from the
 * earliest arrival to the last completion); any pointer may be NULL.
 * reset != 0 clears the statistics after reading.
 */
rfim_status rfim_stream_stats(rfim_ctx* ctx, double* p50, double* p99, double* p999, double* gbps,
                              unsigned long long* chunks, int reset);

/* Drain outstanding work and stop the service's threads; frees its slots. */
rfim_status rfim_stream_close(rfim_ctx* ctx);

/* Static description of a status code. */
const char* rfim_status_str(rfim_status s);

/* Message of the last failing call on ctx ("" if none); valid until the next call. */
const char* rfim_last_error(rfim_ctx* ctx);

/* Library version string, e.g. "rfim-gb300 0.1 sm_103a". */
const char* rfim_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RFIM_H */
