// k_chol_tc.cu -- mixed-precision blocked Cholesky on the tensor cores
// (Sec. 3 Eq. (10)), the dominant cost of the step (89 % of the paper's step
// time, Sec. 4 Table 1).
//
// The paper calls cuSOLVER dpotrf in FP64 (its Tables 2-3 profile the
// library's internal trsm and dgemm kernels).  Here the matrix of every chain
// is FP32, row-major, padded to a multiple of 128, and for each 128-wide
// block column k three launches cover the whole batch:
//
//   potrf128 : factor the 128 x 128 diagonal tile on the CUDA cores (FP32)
//              and form its inverse W = L_kk^{-1} so that the panel solve
//              becomes a product.
//   tc_gemm<TRSM>   : L_ik = A_ik W^T for every tile below the diagonal.
//   tc_gemm<UPDATE> : A_ij -= sum_{k0<=k<k1} L_ik L_jk^T for the trailing
//              lower tiles (diagonal tiles: lower triangle only).
//
// The two products run on the 5th-generation tensor cores.  TMA loads operand
// slices (128-byte swizzle) into a 2-stage shared-memory ring guarded by
// mbarriers (three CTAs per SM overlap each other's epilogues); one thread
// issues the MMAs, accumulating in TMEM; the four warps read TMEM back with
// tcgen05.ld and stage the tile in shared memory in the same swizzled layout.
//   TRSM:   128 x 32 FP32 slices, rounded to nearest TF32 in shared memory,
//           tcgen05.mma kind::tf32 (128 x 128 x 8).  The epilogue stores the
//           TF32-rounded FP32 tile by TMA, then converts it to an FP16 copy
//           (exact for |L| >= 2^-14: the same 10-bit mantissa, and |L| <= 1
//           for D with a unit diagonal) stored by two more TMA stores.
//   UPDATE: 128 x 64 FP16 slices of those copies, tcgen05.mma kind::f16
//           (128 x 128 x 16), one TMA reduce-add into the FP32 matrix.
// Accumulation is FP32 throughout.  No multicast.
// All launches use programmatic dependent launch (pdl.h): a kernel's
// prologue (barriers, TMEM allocation) overlaps the end of its predecessor.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <stdio.h>

#include "bd_internal.h"
#include "pdl.h"
#include "potrf_dev.h"
#include "tc_ptx.h"

namespace bd {

using namespace tc;

constexpr int NB = kMixedTile;             // 128
constexpr int kStages = 2;  // 2 x 32 KiB ring: three CTAs share an SM
constexpr int kChunkBytes = NB * 32 * 4;   // 128 rows x 32 fp32 (or 64 fp16) = 16 KiB
constexpr int kStageBytes = 2 * kChunkBytes;
constexpr int kTcSmem = kStages * kStageBytes + 1024 /*align*/ + 256 /*barriers*/;

enum TcMode { TC_UPDATE = 0, TC_TRSM = 1 };

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  return (uint8_t*)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
}

// Output tile of this CTA.  UPDATE: tiles (i, j) with j in [j0, j1) and
// i in [j, T), enumerated column by column.  TRSM: tiles (i, k0), i in (k0, T).
__device__ __forceinline__ bool tile_of(int mode, int p, int T, int k0, int j0, int j1, int& i,
                                        int& j) {
  if (mode == TC_TRSM) {
    i = k0 + 1 + p;
    j = k0;
    return i < T;
  }
  const int jend = j1 < T ? j1 : T;
  for (j = j0; j < jend; ++j) {
    const int cnt = T - j;
    if (p < cnt) {
      i = j + p;
      return true;
    }
    p -= cnt;
  }
  return false;
}

template <int MODE>
__global__ void __launch_bounds__(128, 3) k_tc_gemm(const CUtensorMap* __restrict__ maps,
                                                    const CUtensorMap* __restrict__ wmap,
                                                    const CUtensorMap* __restrict__ maps16,
                                                    const ChainDesc* __restrict__ cd, int k0, int k1,
                                                    int j0, int j1, int* __restrict__ status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
  uint64_t* empty = full + kStages;
  uint64_t* done = empty + kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int* fail = reinterpret_cast<int*>(tmem_slot + 1);

  const int c = blockIdx.y;
  const ChainDesc d = cd[c];
  const int T = d.np / NB;
  int ti, tj;
  if (!tile_of(MODE, blockIdx.x, T, k0, j0, j1, ti, tj)) return;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *fail = 0;
    fence_barrier_init();
  }
  if (warp == 2) {
    tmem_alloc(tmem_slot, 128);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  grid_dep_wait();  // everything above overlaps the tail of the preceding kernel

  // TRSM: FP32 operands (32-column slices), rounded to TF32 in shared memory.
  // UPDATE: the FP16 copies of the L tiles (64-column slices, the same
  // 32 KB per stage, twice the depth); the result goes to the FP32 matrix.
  const CUtensorMap* om = maps + c;  // FP32 matrix: the output
  const CUtensorMap* am = (MODE == TC_TRSM) ? maps + c : maps16 + c;
  const CUtensorMap* bm = (MODE == TC_TRSM) ? wmap : maps16 + c;
  const int nchunks = (MODE == TC_TRSM) ? 4 : 2 * (k1 - k0);

  if (warp == 0 && lane == 0) {
    // ---- TMA producer
    prefetch_tmap(am);
    if (MODE == TC_TRSM) prefetch_tmap(bm);
    else prefetch_tmap(om);
    for (int q = 0; q < nchunks; ++q) {
      const int s = q % kStages, round = q / kStages;
      if (round > 0 && !mbar_wait(&empty[s], (round - 1) & 1)) {
        atomicExch(fail, 1);
        break;
      }
      uint8_t* sa = smem + s * kStageBytes;
      uint8_t* sb = sa + kChunkBytes;
      mbar_arrive_expect_tx(&full[s], kStageBytes);
      const int kx = k0 * NB + (MODE == TC_TRSM ? 32 : 64) * q;  // column of the K slice in the matrix
      tma_load_2d(sa, am, &full[s], kx, ti * NB);
      if (MODE == TC_TRSM)
        tma_load_2d(sb, bm, &full[s], 32 * q, d.wrow + k0 * NB);
      else
        tma_load_2d(sb, bm, &full[s], kx, tj * NB);
    }
  } else if (warp == 1) {
    // ---- MMA issuer (lane 0).  TRSM: the whole warp first meets the two
    // rounding warps on the stage's named barrier.
    constexpr uint32_t idesc = idesc_mma(MODE == TC_TRSM ? 2u /*tf32*/ : 0u /*f16*/, 128u, 128u);
    bool ok = true;
    for (int q = 0; q < nchunks; ++q) {
      const int s = q % kStages, round = q / kStages;
      if (MODE == TC_TRSM) {
        if (s == 0) named_bar_sync<1, 96>();
        else named_bar_sync<2, 96>();
        if (*(volatile int*)fail) ok = false;
      } else if (lane == 0 && ok && !mbar_wait(&full[s], round & 1)) {
        atomicExch(fail, 1);
        ok = false;
      }
      if (MODE == TC_UPDATE && !__shfl_sync(0xffffffffu, ok, 0)) break;
      if (lane == 0 && ok) {
        tc_fence_after();
        const uint32_t sa = smem_u32(smem + s * kStageBytes);
        const uint64_t ad = desc_sw128(sa), bdsc = desc_sw128(sa + kChunkBytes);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {  // K = 8 tf32 / 16 f16 per MMA = 32 bytes of the 128-byte row
          if (MODE == TC_TRSM)
            mma_tf32(tmem, ad + 2 * kk, bdsc + 2 * kk, idesc, (q > 0 || kk > 0) ? 1u : 0u);
          else
            mma_f16(tmem, ad + 2 * kk, bdsc + 2 * kk, idesc, (q > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(&empty[s]);
      }
      __syncwarp();
    }
    if (lane == 0 && ok) mma_commit(done);
  } else if (MODE == TC_TRSM && warp >= 2) {
    // ---- warps 2-3 round both operand slices of each stage to TF32 in
    // place (elementwise, so the swizzled layout does not matter) and hand
    // the stage to the issuer; they always arrive, so the issuer never waits
    // on them unboundedly.
    const int t = threadIdx.x - 64;
    for (int q = 0; q < nchunks; ++q) {
      const int s = q % kStages, round = q / kStages;
      if (!*(volatile int*)fail && !mbar_wait(&full[s], round & 1)) atomicExch(fail, 1);
      if (!*(volatile int*)fail) {
        float4* st = reinterpret_cast<float4*>(smem + s * kStageBytes);
#pragma unroll 8
        for (int e = t; e < kStageBytes / 16; e += 64) {
          float4 v = st[e];
          v.x = tf32_rna(v.x); v.y = tf32_rna(v.y); v.z = tf32_rna(v.z); v.w = tf32_rna(v.w);
          st[e] = v;
        }
        fence_proxy_async_smem();
      }
      if (s == 0) named_bar_arrive<1, 96>();
      else named_bar_arrive<2, 96>();
    }
  }
  __syncwarp();
  grid_dep_launch();  // the next kernel may start its prologue during this epilogue

  // ---- epilogue (all four warps; warp w owns TMEM lanes / tile rows 32w..)
  const bool got = mbar_wait(done, 0);
  __syncwarp();
  tc_fence_after();
  float* stage_out = reinterpret_cast<float*>(smem);  // 4 chunks x 16 KiB, reusing stages 0-1
  const int row = threadIdx.x;
  const bool diag = (MODE == TC_UPDATE) && (ti == tj);
  if (got) {
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
      uint32_t v[32];
      tmem_ld_32cols(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(q * 32), v);
      tmem_ld_wait();
      float* chunk = stage_out + q * (kChunkBytes / 4) + row * 32;
#pragma unroll
      for (int j4 = 0; j4 < 8; ++j4) {
        float4 f;
        float* fp = reinterpret_cast<float*>(&f);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int col = 32 * q + 4 * j4 + e;
          float val = __uint_as_float(v[4 * j4 + e]);
          if (MODE == TC_UPDATE) {
            val = -val;
            if (diag && col > row) val = 0.0f;
          } else {
            val = tf32_rna(val);  // L tiles enter later products exactly
          }
          fp[e] = val;
        }
        *reinterpret_cast<float4*>(chunk + 4 * (j4 ^ (row & 7))) = f;
      }
    }
  } else {
    atomicExch(fail, 1);
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    if (*fail == 0) {
      for (int q = 0; q < 4; ++q) {
        const float* src = stage_out + q * (kChunkBytes / 4);
        if (MODE == TC_UPDATE)
          tma_reduce_add_2d(om, src, tj * NB + 32 * q, ti * NB);
        else
          tma_store_2d(om, src, k0 * NB + 32 * q, ti * NB);
      }
      bulk_commit();
      // the panel solve only needs the staged tile read before it reuses the
      // shared memory for the FP16 copy; its last wait covers both stores
      if (MODE == TC_TRSM) bulk_wait_read_all();
      else bulk_wait_all();
    } else {
      atomicCAS(status + c, BD_OK, BD_ERR_TIMEOUT);
    }
  }
  __syncthreads();
  if (MODE == TC_TRSM && *(volatile int*)fail == 0) {
    // The FP16 copy of the L tile for the trailing updates, through the same
    // shared memory (the FP32 tile's store has completed): each thread
    // converts its own row, 128-byte rows of 64 halves swizzled like the
    // FP32 chunks, FP16 chunk h (columns 64 h ..) over FP32 chunk 2 + h --
    // chunks 2 and 3 are read before either is overwritten.
    uint32_t hi_half[32];
    const float* rowf = stage_out + row * 32;
    auto granule = [&](int g, uint32_t* out4) {  // columns 8 g .. 8 g + 7 -> 4 half2 words
      const int q = g >> 2, j4 = (2 * g) & 7;    // FP32 chunk, first float4 within it
      const float4 a = *reinterpret_cast<const float4*>(rowf + q * (kChunkBytes / 4) + 4 * (j4 ^ (row & 7)));
      const float4 b = *reinterpret_cast<const float4*>(rowf + q * (kChunkBytes / 4) + 4 * ((j4 + 1) ^ (row & 7)));
      const half2 h0 = __floats2half2_rn(a.x, a.y), h1 = __floats2half2_rn(a.z, a.w);
      const half2 h2 = __floats2half2_rn(b.x, b.y), h3 = __floats2half2_rn(b.z, b.w);
      out4[0] = *reinterpret_cast<const uint32_t*>(&h0);
      out4[1] = *reinterpret_cast<const uint32_t*>(&h1);
      out4[2] = *reinterpret_cast<const uint32_t*>(&h2);
      out4[3] = *reinterpret_cast<const uint32_t*>(&h3);
    };
#pragma unroll
    for (int g = 0; g < 8; ++g) granule(8 + g, hi_half + 4 * g);  // columns 64 .. 127
    uint8_t* h16 = smem + 2 * kChunkBytes + row * 128;            // FP16 chunk 0 (over FP32 chunk 2)
    uint32_t lo_half[4];
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      granule(g, lo_half);
      *reinterpret_cast<uint4*>(h16 + 16 * (g ^ (row & 7))) = make_uint4(lo_half[0], lo_half[1], lo_half[2], lo_half[3]);
    }
#pragma unroll
    for (int g = 0; g < 8; ++g)
      *reinterpret_cast<uint4*>(h16 + kChunkBytes + 16 * (g ^ (row & 7))) =
          make_uint4(hi_half[4 * g], hi_half[4 * g + 1], hi_half[4 * g + 2], hi_half[4 * g + 3]);
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int h = 0; h < 2; ++h)
        tma_store_2d(maps16 + c, smem + (2 + h) * kChunkBytes, k0 * NB + 64 * h, ti * NB);
      bulk_commit();
      bulk_wait_all();
    }
    __syncthreads();
  }
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tmem, 128);
  }
}

// ------------------------------------------------------------ potrf128
// One CTA (544 threads, 528 owning a 4 x 4 block of the lower triangle) per
// chain factors the 128 x 128 diagonal tile k in place and writes
// W = L_kk^{-1} (lower, zeros above) to rows wrow + 128 k .. of Winv (kept for
// the refinement's triangular solve), by the register-blocked right-looking
// elimination of [A | I] in potrf_dev.h: 128 steps, one barrier each.  All in
// FP32: on this part FP64 issues at 1/64 of the FP32 rate, and the FP32
// rounding of this tile (~1e-7 relative) is far below the TF32 rounding of
// the products around it.
using RegPotrf128 = RegPotrf<NB>;

__global__ void __launch_bounds__(RegPotrf128::kThreads) k_potrf128(float* __restrict__ M,
                                                                   float* __restrict__ Winv,
                                                                   const ChainDesc* __restrict__ cd, int k,
                                                                   int* __restrict__ status) {
  __shared__ __align__(16) float sm[RegPotrf128::kSmemFloats];
  const int c = blockIdx.x;
  const ChainDesc d = cd[c];
  if (k * NB >= d.np) return;
  float* base = M + d.moff + (long long)(k * NB) * d.np + k * NB;
  float* wout = Winv + ((long long)d.wrow + (long long)k * NB) * NB;
  grid_dep_wait();
  potrf_regs<NB>(base, d.np, base, d.np, wout, NB, sm);
  grid_dep_launch();
  if (threadIdx.x == 0 && *reinterpret_cast<const int*>(sm + RegPotrf128::kFlag)) atomicCAS(status + c, BD_OK, BD_ERR_NOT_PD);
}

// ------------------------------------------------------------ K update
// Trailing update of the FP32 factorisation of the rod-coupling matrix K
// (64-wide block columns, k_chol_k64.cu) after block column k:
// K_ij -= L_ik L_jk^T over 128 x 128 output blocks of the trailing lower
// triangle (rows and columns from 64 (k + 1); blocks on the diagonal update
// their lower triangle only), on the tensor cores with FP32 accuracy.  Each
// operand slice x is split in shared memory into big = tf32(x) and
// small = tf32(x - big), both rounded to nearest, and the product is formed
// as small_A big_B + big_A small_B + big_A big_B (kind::tf32, FP32
// accumulation in TMEM); the dropped small_A small_B is below 2^-22 of it.
// (K sets the tension iteration's convergence rate and its condition number
// grows like N^2 for stretched chains, so a plain TF32 product would not
// do.)  The 64-column panel is taken in two 32-column slices through one
// 64 KB stage (three CTAs per SM); the result is added into K by TMA
// reduce-add.
constexpr int kKuSmem = 4 * kChunkBytes + 1024 /*align*/ + 256 /*barriers*/;

__device__ __forceinline__ void split_tf32(float4* x, float4* xs) {
  const float4 v = *x;
  float4 hi, lo;
  hi.x = tf32_rna(v.x); hi.y = tf32_rna(v.y); hi.z = tf32_rna(v.z); hi.w = tf32_rna(v.w);
  lo.x = tf32_rna(v.x - hi.x); lo.y = tf32_rna(v.y - hi.y); lo.z = tf32_rna(v.z - hi.z); lo.w = tf32_rna(v.w - hi.w);
  *x = hi;
  *xs = lo;
}

__global__ void __launch_bounds__(128, 3) k_tc_kupdate(const CUtensorMap* __restrict__ kmaps,
                                                       const ChainDesc* __restrict__ cd, int k,
                                                       int* __restrict__ status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + 4 * kChunkBytes);
  uint64_t* done = full + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);

  const int c = blockIdx.y;
  const ChainDesc d = cd[c];
  const int r0 = 64 * (k + 1);
  if (r0 >= d.mp) return;
  const int nb = (d.mp - r0 + NB - 1) / NB;
  const int p = blockIdx.x;
  if (p >= nb * (nb + 1) / 2) return;
  int a = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
  while (a * (a + 1) / 2 > p) --a;
  while ((a + 1) * (a + 2) / 2 <= p) ++a;
  const int b = p - a * (a + 1) / 2;
  const int row0 = r0 + NB * a, col0 = r0 + NB * b;
  const CUtensorMap* km = kmaps + c;

  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    mbar_init(full, 1);
    mbar_init(done, 1);
    fence_barrier_init();
    prefetch_tmap(km);
  }
  if (warp == 2) {
    tmem_alloc(tmem_slot, 128);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  grid_dep_wait();  // the panel L_.k comes from the preceding triangular solve

  uint8_t* sa = smem;
  uint8_t* sb = smem + kChunkBytes;
  uint8_t* sas = smem + 2 * kChunkBytes;
  uint8_t* sbs = smem + 3 * kChunkBytes;
  constexpr uint32_t idesc = idesc_mma(2u /*tf32*/, 128u, 128u);
  bool ok = true;
  for (int q = 0; q < 2 && ok; ++q) {
    if (threadIdx.x == 0) {
      mbar_arrive_expect_tx(full, 2 * kChunkBytes);
      tma_load_2d(sa, km, full, 64 * k + 32 * q, row0);
      tma_load_2d(sb, km, full, 64 * k + 32 * q, col0);
    }
    ok = mbar_wait(full, q & 1);
    if (ok) {
      float4* xa = reinterpret_cast<float4*>(sa);
      float4* xb = reinterpret_cast<float4*>(sb);
      float4* xas = reinterpret_cast<float4*>(sas);
      float4* xbs = reinterpret_cast<float4*>(sbs);
#pragma unroll 4
      for (int e = threadIdx.x; e < kChunkBytes / 16; e += 128) {
        split_tf32(xa + e, xas + e);
        split_tf32(xb + e, xbs + e);
      }
      fence_proxy_async_smem();
    }
    ok = __syncthreads_and(ok) != 0;
    if (ok && threadIdx.x == 0) {
      tc_fence_after();
      const uint64_t ab = desc_sw128(smem_u32(sa)), bb = desc_sw128(smem_u32(sb));
      const uint64_t as = desc_sw128(smem_u32(sas)), bs = desc_sw128(smem_u32(sbs));
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) mma_tf32(tmem, as + 2 * kk, bb + 2 * kk, idesc, (q > 0 || kk > 0) ? 1u : 0u);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) mma_tf32(tmem, ab + 2 * kk, bs + 2 * kk, idesc, 1u);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) mma_tf32(tmem, ab + 2 * kk, bb + 2 * kk, idesc, 1u);
      mma_commit(done);
    }
    if (ok) ok = mbar_wait(done, q & 1);  // the stage is free again
    ok = __syncthreads_and(ok) != 0;
  }
  grid_dep_launch();

  // ---- epilogue: -acc (lower triangle of a diagonal block) into K
  tc_fence_after();
  float* stage_out = reinterpret_cast<float*>(smem);  // 4 chunks x 16 KiB over the stage
  const int row = threadIdx.x;
  const bool diag = (a == b);
  if (ok) {
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
      uint32_t v[32];
      tmem_ld_32cols(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(q * 32), v);
      tmem_ld_wait();
      float* chunk = stage_out + q * (kChunkBytes / 4) + row * 32;
#pragma unroll
      for (int j4 = 0; j4 < 8; ++j4) {
        float4 f;
        float* fp = reinterpret_cast<float*>(&f);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int col = 32 * q + 4 * j4 + e;
          fp[e] = (diag && col > row) ? 0.0f : -__uint_as_float(v[4 * j4 + e]);
        }
        *reinterpret_cast<float4*>(chunk + 4 * (j4 ^ (row & 7))) = f;
      }
    }
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    if (ok) {
      // (mp is a multiple of 64: a 32-column box is wholly inside K or
      // wholly right of it, and only those inside are issued; rows past mp
      // are clipped by the TMA unit)
      for (int q = 0; q < 4; ++q)
        if (col0 + 32 * q < d.mp) tma_reduce_add_2d(km, stage_out + q * (kChunkBytes / 4), col0 + 32 * q, row0);
      bulk_commit();
      bulk_wait_all();
    } else {
      atomicCAS(status + c, BD_OK, BD_ERR_TIMEOUT);
    }
  }
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tmem, 128);
  }
}

bool is_kupdate_tc_kernel(const void* f) { return f == (const void*)k_tc_kupdate; }

// ------------------------------------------------------------ wait self-test
// One thread waits on a fresh mbarrier with the bounded wait every kernel of
// the library uses.  Without an arrival nothing completes the phase and the
// wait gives up after its limit; *out receives BD_ERR_TIMEOUT (BD_OK when the
// thread arrived first).
__global__ void k_wait_selftest(int arrive, int* __restrict__ out) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_barrier_init();
  if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
  *out = mbar_wait(&bar, 0) ? BD_OK : BD_ERR_TIMEOUT;
}

cudaError_t launch_wait_selftest(int arrive, int* out, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(arrive, out);
  return cudaGetLastError();
}

cudaError_t launch_kupdate_tc(const CUtensorMap* kmaps, const ChainDesc* cd, int n_chains, int max_mp, int k,
                              int* status, cudaStream_t s) {
  const int r0 = 64 * (k + 1);
  if (r0 >= max_mp) return cudaSuccess;
  const int nb = (max_mp - r0 + NB - 1) / NB;
  return launch_pdl(k_tc_kupdate, dim3(nb * (nb + 1) / 2, n_chains), dim3(128), kKuSmem, s, kmaps, cd, k, status);
}

// ------------------------------------------------------------ host side
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// FP32 row-major [rows][cols] matrix, 32 x 128 boxes, 128-byte swizzle.
static bool encode_f32(CUtensorMap* out, void* base, uint64_t cols, uint64_t rows, uint64_t ld) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {ld * 4};
  cuuint32_t box[2] = {32, (cuuint32_t)NB};
  cuuint32_t es[2] = {1, 1};
  return fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static bool encode_f16(CUtensorMap* out, void* base, uint64_t cols, uint64_t rows, uint64_t ld) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {ld * 2};
  cuuint32_t box[2] = {64, (cuuint32_t)NB};  // 128-byte rows
  cuuint32_t es[2] = {1, 1};
  return fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, base, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Fills maps[0..n_chains) (one per chain's matrix), maps[n_chains] (Winv,
// [sum_c np_c][128]) and maps[n_chains + 1 + c] (chain c's FP16 copy of the
// L tiles, same layout as its matrix).
bool make_tc_maps(CUtensorMap* host_maps, float* M, float* Winv, __half* M16, const ChainDesc* h_cd,
                  int n_chains) {
  uint64_t wrows = 0;
  for (int c = 0; c < n_chains; ++c) {
    if (!encode_f32(&host_maps[c], M + h_cd[c].moff, h_cd[c].np, h_cd[c].np, h_cd[c].np)) return false;
    if (!encode_f16(&host_maps[n_chains + 1 + c], M16 + h_cd[c].moff, h_cd[c].np, h_cd[c].np, h_cd[c].np))
      return false;
    wrows += h_cd[c].np;
  }
  return encode_f32(&host_maps[n_chains], Winv, NB, wrows, NB);
}

// maps[c]: chain c's FP32 matrix K ([mp][mp]), 32 x 128 boxes.
bool make_k_maps(CUtensorMap* host_maps, float* K, const ChainDesc* h_cd, int n_chains) {
  for (int c = 0; c < n_chains; ++c)
    if (!encode_f32(&host_maps[c], K + h_cd[c].koff, h_cd[c].mp, h_cd[c].mp, h_cd[c].mp)) return false;
  return true;
}

cudaError_t tc_configure() {
  cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<TC_UPDATE>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_gemm<TC_TRSM>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_kupdate, cudaFuncAttributeMaxDynamicSharedMemorySize, kKuSmem);
  return e;
}

// Right-looking with super-panels of `panel` tile columns: inside a panel,
// column k first receives the updates of the panel's earlier columns
// (K = 128 (k - K0)), is factored and solved; the trailing matrix is updated
// once per panel with K = 128 panel, so every trailing tile is read and
// written `panel` times less often than with single-column steps.
static int update_tiles(int T, int j0, int j1) {
  int n = 0;
  for (int j = j0; j < j1 && j < T; ++j) n += T - j;
  return n;
}

cudaError_t launch_chol_tc(float* M, float* Winv, const CUtensorMap* maps, const CUtensorMap* wmap,
                           const CUtensorMap* maps16, const ChainDesc* cd, int n_chains, int max_tiles,
                           int panel, int* status, cudaStream_t s) {
  const int T = max_tiles;
  if (panel < 1) panel = 1;
  cudaError_t e = cudaSuccess;
  for (int K0 = 0; K0 < T && e == cudaSuccess; K0 += panel) {
    const int K1 = K0 + panel < T ? K0 + panel : T;
    for (int k = K0; k < K1 && e == cudaSuccess; ++k) {
      if (k > K0)
        e = launch_pdl(k_tc_gemm<TC_UPDATE>, dim3(update_tiles(T, k, k + 1), n_chains), dim3(128), kTcSmem, s,
                       maps, (const CUtensorMap*)nullptr, maps16, cd, K0, k, k, k + 1, status);
      if (e == cudaSuccess)
        e = launch_pdl(k_potrf128, dim3(n_chains), dim3(RegPotrf128::kThreads), 0, s, M, Winv, cd, k, status);
      const int below = T - 1 - k;
      if (below > 0 && e == cudaSuccess)
        e = launch_pdl(k_tc_gemm<TC_TRSM>, dim3(below, n_chains), dim3(128), kTcSmem, s, maps, wmap, maps16, cd, k,
                       k + 1, 0, 0, status);
    }
    if (K1 < T && e == cudaSuccess)
      e = launch_pdl(k_tc_gemm<TC_UPDATE>, dim3(update_tiles(T, K1, T), n_chains), dim3(128), kTcSmem, s, maps,
                     (const CUtensorMap*)nullptr, maps16, cd, K0, K1, K1, T, status);
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace bd
