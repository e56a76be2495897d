// potrf_dev.h -- FP32 factorisation of a square diagonal tile together with
// its inverse, used by the tensor-core Cholesky (128-wide tiles) and the FP32
// factorisation of the rod-coupling matrix (64-wide tiles).
#pragma once
#include <stdint.h>

namespace bd {

// ------------------------------------------------------------------------
// Register-blocked right-looking factorisation of an H x H SPD tile together
// with its inverse W = L^{-1}, four pivots per super-step.
//
// Thread t < NBLK owns the 4 x 4 block (bi, bk), bk <= bi, of the lower
// triangle in 16 registers c[][]: first the block of A (updated until it
// becomes a block of L), then the block of W.  Super-step b:
//   1. the owner of (b, b) factors its block, A_bb = L_bb L_bb^T, and forms
//      Linv = L_bb^{-1} (4 x 4, in registers);
//   2. panel  (i, b), i > b:  L_ib = A_ib Linv^T, published; c := 0 (W_ib);
//      block row b of W:       W_bm = Linv W_bm (m < b), W_bb = Linv,
//      written out and published;
//   3. every block with bi > b:  c -= L_{bi,b} Q with Q = L_{bk,b}^T for the
//      trailing A (bk > b) or Q = W_{b,bk} for the block rows of W below b
//      (bk <= b) -- the same 4 x 4 x 4 product for every active thread.
// Steps 2-3 of W are forward substitution L W = I by block rows in
// right-looking order.  Two barriers per super-step.
template <int H>
struct RegPotrf {
  static constexpr int NBK = H / 4;
  static constexpr int NBLK = NBK * (NBK + 1) / 2;
  static constexpr int kThreads = (NBLK + 31) / 32 * 32;
  static constexpr int kSmemFloats = 8 * H + 20;  // sP[4][H], sY[4][H], sLinv[16], flag
  static constexpr int kFlag = 8 * H + 16;        // float offset of the bad-pivot flag
};

// src/Lout: tile origin and row pitch (floats; may alias: each thread reads
// its block before the first barrier and writes only its own block later).
// Lout receives the lower triangle of L only (the strict upper triangle of
// the destination is left untouched).  Wout ([H][ldw]) receives L^{-1} with
// zeros above the diagonal.  Row pitches and origins must be 16-byte aligned.
// sm[kFlag] (an int) is nonzero afterwards if a pivot was not positive.
template <int H>
__device__ __forceinline__ void potrf_regs(const float* src, long long lds, float* Lout, long long ldl,
                                           float* __restrict__ Wout, int ldw, float* sm) {
  using P = RegPotrf<H>;
  // Planes, so that a warp's float4 loads of consecutive blocks are
  // consecutive 16-byte words (no bank conflicts):
  float* sP = sm;             // [4][H]: sP[k][4i + r] = L_ib[r][k]
  float* sY = sm + 4 * H;     // [4][H]: sY[t][4m + s] = W_bm[t][s] (block row b of W)
  float* sLinv = sm + 8 * H;  // [4][4]
  int* bad = reinterpret_cast<int*>(sm + P::kFlag);
  const int t = threadIdx.x;
  const bool owner = t < P::NBLK;
  int bi = 0, bk = 0;
  if (owner) {
    bi = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
    while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
    while (bi * (bi + 1) / 2 > t) --bi;
    bk = t - bi * (bi + 1) / 2;
  }
  const bool diag = owner && bi == bk;
  float c[4][4];
  if (t == 0) *bad = 0;
  if (owner) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float4 v = *reinterpret_cast<const float4*>(src + (long long)(4 * bi + r) * lds + 4 * bk);
      c[r][0] = v.x; c[r][1] = v.y; c[r][2] = v.z; c[r][3] = v.w;
#pragma unroll
      for (int s = 0; s < 4; ++s)
        if (diag && s > r) c[r][s] = 0.0f;
    }
  }
  for (int b = 0; b < P::NBK; ++b) {
    // ---- 1. diagonal block
    if (diag && bi == b) {
      float Lb[4][4], Li[4][4], rq[4];
      bool badl = false;
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int s = 0; s < 4; ++s) Lb[r][s] = Li[r][s] = 0.0f;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float p = c[j][j];
        if (!(p > 0.0f)) {
          badl = true;
          p = 1.0f;
        }
        const float r = rsqrtf(p);
        rq[j] = r;
        Lb[j][j] = p * r;
#pragma unroll
        for (int i = j + 1; i < 4; ++i) Lb[i][j] = c[i][j] * r;
#pragma unroll
        for (int i = j + 1; i < 4; ++i)
#pragma unroll
          for (int s = j + 1; s <= i; ++s) c[i][s] = fmaf(-Lb[i][j], Lb[s][j], c[i][s]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        Li[j][j] = rq[j];
#pragma unroll
        for (int i = j + 1; i < 4; ++i) {
          float acc = 0.0f;
#pragma unroll
          for (int q = j; q < i; ++q) acc = fmaf(Lb[i][q], Li[q][j], acc);
          Li[i][j] = -acc * rq[i];
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
#pragma unroll
        for (int s = 0; s <= r; ++s) Lout[(long long)(4 * b + r) * ldl + 4 * b + s] = Lb[r][s];
        *reinterpret_cast<float4*>(sLinv + 4 * r) = make_float4(Li[r][0], Li[r][1], Li[r][2], Li[r][3]);
#pragma unroll
        for (int s = 0; s < 4; ++s) c[r][s] = Li[r][s];  // W_bb
      }
      if (badl) *bad = 1;
    }
    __syncthreads();
    // ---- 2. panel and block row b of W
    if (owner && (bk == b || bi == b)) {
      float Li[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float4 v = *reinterpret_cast<const float4*>(sLinv + 4 * r);
        Li[r][0] = v.x; Li[r][1] = v.y; Li[r][2] = v.z; Li[r][3] = v.w;
      }
      if (bk == b && bi > b) {
        float l[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            float acc = 0.0f;
#pragma unroll
            for (int q = 0; q <= s; ++q) acc = fmaf(c[r][q], Li[s][q], acc);
            l[r][s] = acc;
          }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const float4 v = make_float4(l[r][0], l[r][1], l[r][2], l[r][3]);
          *reinterpret_cast<float4*>(Lout + (long long)(4 * bi + r) * ldl + 4 * bk) = v;
#pragma unroll
          for (int s = 0; s < 4; ++s) c[r][s] = 0.0f;  // W_ib starts at zero
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
          *reinterpret_cast<float4*>(sP + k * H + 4 * bi) = make_float4(l[0][k], l[1][k], l[2][k], l[3][k]);
      } else if (bi == b) {
        if (bk < b) {
          float y[4][4];
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int s = 0; s < 4; ++s) {
              float acc = 0.0f;
#pragma unroll
              for (int q = 0; q <= r; ++q) acc = fmaf(Li[r][q], c[q][s], acc);
              y[r][s] = acc;
            }
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int s = 0; s < 4; ++s) c[r][s] = y[r][s];
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
          *reinterpret_cast<float4*>(Wout + (long long)(4 * b + r) * ldw + 4 * bk) =
              make_float4(c[r][0], c[r][1], c[r][2], c[r][3]);
#pragma unroll
        for (int r = 0; r < 4; ++r)
          *reinterpret_cast<float4*>(sY + r * H + 4 * bk) = make_float4(c[r][0], c[r][1], c[r][2], c[r][3]);
      }
    }
    __syncthreads();
    // ---- 3. trailing A and the block rows of W below b
    if (owner && bi > b) {
      // Q[k][s] = L_{bk,b}[s][k] = sP[k][4 bk + s]  or  W_{b,bk}[k][s] = sY[k][4 bk + s]
      const float* qb = (bk > b) ? sP : sY;
      float p[4][4], q[4][4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float4 v = *reinterpret_cast<const float4*>(sP + k * H + 4 * bi);
        p[0][k] = v.x; p[1][k] = v.y; p[2][k] = v.z; p[3][k] = v.w;
        const float4 w = *reinterpret_cast<const float4*>(qb + k * H + 4 * bk);
        q[k][0] = w.x; q[k][1] = w.y; q[k][2] = w.z; q[k][3] = w.w;
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
          for (int k = 0; k < 4; ++k) c[r][s] = fmaf(-p[r][k], q[k][s], c[r][s]);
    }
  }
  for (int e = t; e < P::NBK * P::NBK; e += blockDim.x) {
    const int ub = e / P::NBK, uk = e % P::NBK;
    if (uk > ub) {
#pragma unroll
      for (int r = 0; r < 4; ++r)
        *reinterpret_cast<float4*>(Wout + (long long)(4 * ub + r) * ldw + 4 * uk) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

}  // namespace bd
