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

// Bytes, when rows and cols are multiples of 4 and the planes 4-byte aligned:
// tiles of 64 columns x 256 rows.  A thread loads four 4 x 4 blocks as row
// words (16 lanes read 64 contiguous bytes of a row; all 16 loads in flight),
// transposes each in registers (byte permutes) and leaves the column words in
// shared memory, from where 32 lanes store 128 contiguous bytes of an output
// row.
constexpr int TR_ROWS = 256;  // rows of a tile
__global__ void __launch_bounds__(256) k_transpose_u8x4(const uint8_t* __restrict__ in, uint8_t* __restrict__ out,
                                                        int rows, int cols) {
  __shared__ uint32_t tile[64][TR_ROWS / 4 + 1];  // [column within the tile][row quad]; +1 word against bank conflicts
  const size_t plane = (size_t)rows * cols;
  const uint8_t* src = in + (size_t)blockIdx.z * plane;
  uint8_t* dst = out + (size_t)blockIdx.z * plane;
  const int c0 = blockIdx.x * 64, r0 = blockIdx.y * TR_ROWS;
  const int cq = threadIdx.x & 15, rq = threadIdx.x >> 4;
  const int c = c0 + 4 * cq;
  uint32_t w[4][4];
#pragma unroll
  for (int p = 0; p < 4; p++)
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int r = r0 + 4 * (rq + 16 * p) + j;
      w[p][j] = (r < rows && c < cols) ? __ldg(reinterpret_cast<const uint32_t*>(src + (size_t)r * cols + c)) : 0u;
    }
#pragma unroll
  for (int p = 0; p < 4; p++) {
    transpose4x4(w[p][0], w[p][1], w[p][2], w[p][3]);  // w[p][i]: column c + i, rows r0 + 4 (rq + 16 p) .. + 3
#pragma unroll
    for (int i = 0; i < 4; i++) tile[4 * cq + i][rq + 16 * p] = w[p][i];
  }
  __syncthreads();
  const int wq = threadIdx.x & 63, r = r0 + 4 * wq;
#pragma unroll
  for (int k = 0; k < 16; k++) {
    const int cc = (threadIdx.x >> 6) + 4 * k, oc = c0 + cc;
    if (oc < cols && r < rows) *reinterpret_cast<uint32_t*>(dst + (size_t)oc * rows + r) = tile[cc][wq];
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
  uint32_t mine = 0;  // lane j keeps sample t0 + j's word; the 32 stores then go out together
#pragma unroll 8
  for (int j = 0; j < 32; j++) {
    const uint32_t col = __ballot_sync(0xffffffffu, (w >> j) & 1u);
    if (lane == j) mine = col;
  }
  const int t = wt * 32 + lane;
  if (t < T) dst[(size_t)t * WC + wc] = mine;
}

int launch_transpose(const void* in, void* out, int batch, int rows, int cols, int esize, void* stream) {
  dim3 grid((cols + 31) / 32, (rows + 31) / 32, batch);
  cudaStream_t st = (cudaStream_t)stream;
  if (esize == 1 && (rows & 3) == 0 && (cols & 3) == 0 && (((uintptr_t)in | (uintptr_t)out) & 3) == 0) {
    dim3 g4((cols + 63) / 64, (rows + TR_ROWS - 1) / TR_ROWS, batch);
    k_transpose_u8x4<<<g4, 256, 0, st>>>((const uint8_t*)in, (uint8_t*)out, rows, cols);
  } else if (esize == 1)
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
