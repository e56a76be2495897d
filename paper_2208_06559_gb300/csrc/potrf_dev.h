// potrf_dev.h -- device routines for the FP32 factorisation of a square
// diagonal tile held in shared memory (row pitch LDA = 129 floats), shared by
// the tensor-core Cholesky (128-wide tiles) and the FP32 factorisation of the
// rod-coupling matrix (64-wide tiles).
//
// Recursive halving down to 16 x 16: for a block [[A11, .], [A21, A22]]
//   factor A11 -> L11, W11;  L21 = A21 W11^T;  A22 -= L21 L21^T;
//   factor A22 -> L22, W22;  W21 = -W22 (L21 W11);
// so the tile's factor L and its inverse W are produced together.  Every
// product is split evenly over the kPotrfThreads threads with register
// blocking; the 16 x 16 leaves are factored by one warp in registers (lane r
// holds row r, pivots broadcast by shuffles) together with their inverses.
#pragma once
#include <stdint.h>

namespace bd {

constexpr int LDA = 129;  // 128 + 1
constexpr int SB = 16;
constexpr int kPotrfThreads = 512;

// 16 x 16 leaf at offset o: L (into A) and W_oo (into W), one warp.  Lane r
// holds row r of the block; at step j the column j just scaled is published
// to shared memory (in place in A) and read back by every lane as broadcasts,
// so the serial chain is one store, one warp barrier and independent loads
// per pivot.  The inverse is formed column by column (lane = column) from L
// in shared memory.
__device__ __forceinline__ void leaf16(float* A, float* W, int o, int* bad) {
  const int lane = threadIdx.x & 31;
  if ((threadIdx.x >> 5) == 0) {
    const int r = lane & (SB - 1);
    const bool own = lane < SB;
    float* Ab = A + o * LDA + o;  // block origin
    float a[SB];
#pragma unroll
    for (int q = 0; q < SB; ++q) a[q] = (q <= r) ? Ab[r * LDA + q] : 0.0f;
    bool badl = false;
#pragma unroll
    for (int j = 0; j < SB; ++j) {
      // pivot: lane j's diagonal entry, read from shared memory after lane j
      // wrote it in the previous step (step 0: the loaded value)
      const float djj = (j == 0) ? Ab[0] : Ab[j * LDA + j];
      const bool ok = djj > 0.0f;
      badl |= !ok;
      const float inv = rsqrtf(ok ? djj : 1.0f);
      if (r == j) a[j] = (ok ? djj : 1.0f) * inv;
      else if (r > j) a[j] *= inv;
      if (own && r >= j) Ab[r * LDA + j] = a[j];  // column j of L
      __syncwarp();
      float lq[SB];
#pragma unroll
      for (int q = j + 1; q < SB; ++q) lq[q] = Ab[q * LDA + j];
#pragma unroll
      for (int q = j + 1; q < SB; ++q)
        if (r >= q) a[q] -= a[j] * lq[q];
      // next pivot entry becomes visible to everyone
      if (j + 1 < SB && own && r == j + 1) Ab[r * LDA + j + 1] = a[j + 1];
      __syncwarp();
    }
    if (own) {
#pragma unroll
      for (int q = 0; q < SB; ++q)
        if (q <= r) Ab[r * LDA + q] = a[q];
    }
    __syncwarp();
    if (own) {  // column `lane` of the inverse
      float w[SB];
#pragma unroll
      for (int i = 0; i < SB; ++i) {
        float sacc = (i == r) ? 1.0f : 0.0f;
#pragma unroll
        for (int m = 0; m < i; ++m) sacc -= Ab[i * LDA + m] * w[m];
        w[i] = (i >= r) ? sacc / Ab[i * LDA + i] : 0.0f;
      }
#pragma unroll
      for (int i = 0; i < SB; ++i) W[(o + i) * LDA + o + lane] = w[i];
    }
    if (__any_sync(0xffffffffu, badl && own) && lane == 0) *bad = 1;
  }
  __syncthreads();
}

// C (H x H, at rows rc, cols cc of buffer Cb) op= X * Y with
//   TRANS_Y: Y element (m, c) read as Yb[(ry + c) * LDA + cy + m]  (Y^T stored)
//   else   : Y element (m, c) read as Yb[(ry + m) * LDA + cy + c]
// and X element (r, m) = Xb[(rx + r) * LDA + cx + m].  MODE 0: C = acc,
// 1: C -= acc (lower triangle only when LOWER), 2: C = -acc.  Thread blocks
// of RB x CB outputs; results are held in registers until every thread has
// finished reading, so C may alias an input.
template <int H, bool TRANS_Y, int MODE, bool LOWER>
__device__ __forceinline__ void tile_gemm(float* Cb, int rc, int cc, const float* Xb, int rx, int cx,
                                          const float* Yb, int ry, int cy) {
  constexpr int OUT = H * H;
  constexpr int PER = OUT / kPotrfThreads > 0 ? OUT / kPotrfThreads : 1;  // outputs per thread
  constexpr int RB = PER >= 8 ? 4 : (PER >= 2 ? 2 : 1);
  constexpr int CB = PER / RB > 0 ? PER / RB : 1;
  constexpr int NCB = H / CB;       // column blocks
  constexpr int NT = (H / RB) * NCB;  // threads used
  float acc[RB][CB];
#pragma unroll
  for (int i = 0; i < RB; ++i)
#pragma unroll
    for (int j = 0; j < CB; ++j) acc[i][j] = 0.0f;
  const int t = threadIdx.x;
  const bool active = t < NT;
  const int r0 = (t / NCB) * RB, c0 = (t % NCB) * CB;
  if (active) {
#pragma unroll 4
    for (int m = 0; m < H; ++m) {
      float xv[RB], yv[CB];
#pragma unroll
      for (int i = 0; i < RB; ++i) xv[i] = Xb[(rx + r0 + i) * LDA + cx + m];
#pragma unroll
      for (int j = 0; j < CB; ++j)
        yv[j] = TRANS_Y ? Yb[(ry + c0 + j) * LDA + cy + m] : Yb[(ry + m) * LDA + cy + c0 + j];
#pragma unroll
      for (int i = 0; i < RB; ++i)
#pragma unroll
        for (int j = 0; j < CB; ++j) acc[i][j] += xv[i] * yv[j];
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int i = 0; i < RB; ++i)
#pragma unroll
      for (int j = 0; j < CB; ++j) {
        float* cp = Cb + (rc + r0 + i) * LDA + cc + c0 + j;
        if (MODE == 0) *cp = acc[i][j];
        else if (MODE == 2) *cp = -acc[i][j];
        else if (!LOWER || c0 + j <= r0 + i) *cp -= acc[i][j];
      }
  }
  __syncthreads();
}

template <int H>
__device__ void potrf_rec(float* A, float* W, float* Tm, int o, int* bad) {
  if constexpr (H == SB) {
    leaf16(A, W, o, bad);
  } else {
    constexpr int h = H / 2;
    const int o2 = o + h;
    potrf_rec<h>(A, W, Tm, o, bad);
    // L21 = A21 W11^T  (in place over A21)
    tile_gemm<h, true, 0, false>(A, o2, o, A, o2, o, W, o, o);
    // A22 -= L21 L21^T (lower)
    tile_gemm<h, true, 1, true>(A, o2, o2, A, o2, o, A, o2, o);
    potrf_rec<h>(A, W, Tm, o2, bad);
    // Tm = L21 W11 ;  W21 = -W22 Tm
    tile_gemm<h, false, 0, false>(Tm, o2, o, A, o2, o, W, o, o);
    tile_gemm<h, false, 2, false>(W, o2, o, W, o2, o2, Tm, o2, o);
  }
}


}  // namespace bd
