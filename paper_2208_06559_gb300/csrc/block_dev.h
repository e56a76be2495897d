// block_dev.h -- block-wide sums and prefix sums of 3-vectors (FP64), for
// kernels that rebuild positions from link vectors.  The block size must be
// a multiple of 32 and at most 1024; every thread of the block calls them.
#pragma once

namespace bd {

// Sum of a 3-vector over the block (result in every thread).
__device__ __forceinline__ void block_sum3(double v[3], double (*red)[3]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < 3; ++c) red[warp][c] = v[c];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double x = lane < (int)(blockDim.x >> 5) ? red[lane][c] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) red[0][c] = x;
    }
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 3; ++c) v[c] = red[0][c];
  __syncthreads();
}

// Exclusive prefix sum of a 3-vector over the threads of the block.
__device__ __forceinline__ void block_exscan3(double v[3], double (*red)[3]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double inc[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    inc[c] = v[c];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double x = __shfl_up_sync(0xffffffffu, inc[c], o);
      if (lane >= o) inc[c] += x;
    }
  }
  if (lane == 31)
#pragma unroll
    for (int c = 0; c < 3; ++c) red[warp][c] = inc[c];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double x = red[lane][c];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      red[lane][c] = x;  // inclusive scan of the warp totals
    }
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 3; ++c) v[c] = inc[c] - v[c] + (warp > 0 ? red[warp - 1][c] : 0.0);
  __syncthreads();
}

}  // namespace bd
