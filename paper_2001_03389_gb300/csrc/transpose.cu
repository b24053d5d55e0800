// transpose.cu -- layout conversion between BTC (channel fastest) and BCT
// (time fastest) blocks, for the BTC entry points: the block is transposed
// into a BCT scratch buffer, cleaned there, and transposed back.
#include <cuda_runtime.h>

#include <cstdint>

#include "engine.h"

namespace rfim {

// out[b][c][r] = in[b][r][c] for rows x cols matrices of element type E.
// Tiles of 32 x 32 elements through shared memory; 32 x 8 threads, each
// moving four elements.
template <typename E>
__global__ void __launch_bounds__(256) k_transpose(const E* __restrict__ in, E* __restrict__ out, int rows, int cols) {
  __shared__ E tile[32][33];
  const size_t plane = (size_t)rows * cols;
  const E* src = in + (size_t)blockIdx.z * plane;
  E* dst = out + (size_t)blockIdx.z * plane;
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 32; k += 8) {
    const int r = r0 + ty + k, c = c0 + tx;
    if (r < rows && c < cols) tile[ty + k][tx] = src[(size_t)r * cols + c];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 32; k += 8) {
    const int c = c0 + ty + k, r = r0 + tx;
    if (r < rows && c < cols) dst[(size_t)c * rows + r] = tile[tx][ty + k];
  }
}

// Bit masks: in is the BCT mask of a beam (rows c, words of 32 samples), out
// the BTC mask (rows t, words of 32 channels).  One warp per 32 x 32 bit block:
// lane i holds channel c0 + i's word; the ballot over bit j is sample t0 + j's word.
__global__ void __launch_bounds__(256) k_transpose_bits(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                        int C, int T) {
  const int WT = (T + 31) >> 5, WC = (C + 31) >> 5;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nblk = WT * WC;
  if (warp >= nblk) return;  // whole warps only: the grid is a multiple of 32 threads
  const int wt = warp % WT, wc = warp / WT;
  const uint32_t* src = in + (size_t)blockIdx.y * C * WT;
  uint32_t* dst = out + (size_t)blockIdx.y * T * WC;
  const int c = wc * 32 + lane;
  const uint32_t w = c < C ? src[(size_t)c * WT + wt] : 0u;
#pragma unroll 4
  for (int j = 0; j < 32; j++) {
    const uint32_t col = __ballot_sync(0xffffffffu, (w >> j) & 1u);
    const int t = wt * 32 + j;
    if (lane == 0 && t < T) dst[(size_t)t * WC + wc] = col;
  }
}

int launch_transpose(const void* in, void* out, int batch, int rows, int cols, int esize, void* stream) {
  dim3 grid((cols + 31) / 32, (rows + 31) / 32, batch);
  cudaStream_t st = (cudaStream_t)stream;
  if (esize == 1)
    k_transpose<uint8_t><<<grid, 256, 0, st>>>((const uint8_t*)in, (uint8_t*)out, rows, cols);
  else
    k_transpose<float><<<grid, 256, 0, st>>>((const float*)in, (float*)out, rows, cols);
  return (int)cudaGetLastError();
}

int launch_transpose_bits(const void* in_bct, void* out_btc, int batch, int C, int T, void* stream) {
  const long long blocks = (long long)((T + 31) / 32) * ((C + 31) / 32);
  const long long threads = blocks * 32;
  dim3 grid((unsigned)((threads + 255) / 256), batch);
  k_transpose_bits<<<grid, 256, 0, (cudaStream_t)stream>>>((const uint32_t*)in_bct, (uint32_t*)out_btc, C, T);
  return (int)cudaGetLastError();
}

}  // namespace rfim
