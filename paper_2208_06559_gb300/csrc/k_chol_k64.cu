// k_chol_k64.cu -- FP32 Cholesky of the rod-coupling matrix K on the CUDA
// cores, 64 x 64 tiles, for the mixed-precision path.
//
// K = U^T C^T D C U (order N - 1) is the Jacobian of the tension iteration at
// Q = u; it only sets the convergence rate, but for stretched chains its
// condition number grows like N^2, so its factor must be FP32-accurate (the
// TF32 tensor-core path is not).  Per block column k:
//   potrf64 : one CTA factors the 64 x 64 diagonal tile and forms its inverse
//             (the register-blocked routine of the 128-wide path);
//   trsm64  : L_ik = A_ik W_kk^T, 64 x 64 per CTA, 8 x 8 outputs per thread;
//   update  : A_ij -= L_ik L_jk^T for the trailing lower tiles, on the tensor
//             cores with split TF32 operands (k_chol_tc.cu), or on the CUDA
//             cores (update64).
// The 64 x 64 diagonal-tile inverses are kept for the tension solve.
#include "bd_internal.h"
#include "pdl.h"
#include "potrf_dev.h"

namespace bd {

constexpr int K64 = 64;
using RegPotrf64 = RegPotrf<K64>;

__global__ void __launch_bounds__(RegPotrf64::kThreads) k_potrf64(float* __restrict__ K, float* __restrict__ Kinv,
                                                                 const ChainDesc* __restrict__ cd, int k,
                                                                 int* __restrict__ status) {
  __shared__ __align__(16) float sm[RegPotrf64::kSmemFloats];
  const int c = blockIdx.x;
  const ChainDesc d = cd[c];
  if (k * K64 >= d.mp) return;
  float* base = K + d.koff + (long long)(k * K64) * d.mp + k * K64;
  float* wout = Kinv + (d.kwrow + (long long)k * K64) * K64;
  grid_dep_wait();
  potrf_regs<K64>(base, d.mp, base, d.mp, wout, K64, sm);
  grid_dep_launch();
  if (threadIdx.x == 0 && *reinterpret_cast<const int*>(sm + RegPotrf64::kFlag)) atomicCAS(status + c, BD_OK, BD_ERR_CONSTRAINT);
}

// 64 x 64 output tile, 64 threads, 8 x 8 outputs each.  The operands are
// copied row-major into shared memory with cp.async, all copies in flight at
// once; the update's output tile is copied into the first operand's buffer
// once the products are done (two tiles of shared memory: six CTAs per SM).  Thread (i, j) =
// (t % 8, t / 8) owns rows i + 8a and columns j + 8b (a, b < 8): per four k
// it reads eight 16-byte row slices of each operand (rows 4 banks apart
// across a warp: no bank conflicts) for 256 FMAs.  The result is written back
// from shared memory in coalesced 16-byte rows.
// TRSM: X = A_ik W_kk^T (overwrites A_ik).  UPDATE: A_ij -= L_ik L_jk^T
// (diagonal tiles: lower triangle only).
constexpr int kG64Threads = 64;
constexpr int kG64P = K64 + 4;  // pitch: 16-byte aligned rows, 4 banks apart
constexpr int kG64Tile = K64 * kG64P;

template <bool TRSM>
constexpr int g64_smem() {
  return 2 * kG64Tile * (int)sizeof(float);
}

__device__ __forceinline__ void g64_cp16(float* smem, const float* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}

template <bool TRSM>
__global__ void __launch_bounds__(kG64Threads) k_gemm64(float* __restrict__ K, const float* __restrict__ Kinv,
                                                        const ChainDesc* __restrict__ cd, int k) {
  extern __shared__ __align__(16) float g64s[];
  float (*Xs)[kG64P] = reinterpret_cast<float (*)[kG64P]>(g64s);
  float (*Ys)[kG64P] = reinterpret_cast<float (*)[kG64P]>(g64s + kG64Tile);
  float (*Cs)[kG64P] = Xs;  // the output tile, after the products
  const ChainDesc d = cd[blockIdx.y];
  const int T = d.mp / K64;
  int i, j;
  if (TRSM) {
    i = k + 1 + blockIdx.x;
    j = k;
    if (i >= T) return;
  } else {
    const int s = T - k - 1;
    const int p = blockIdx.x;
    if (s <= 0 || p >= s * (s + 1) / 2) return;
    int ii = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
    while (ii * (ii + 1) / 2 > p) --ii;
    while ((ii + 1) * (ii + 2) / 2 <= p) ++ii;
    i = k + 1 + ii;
    j = k + 1 + (p - ii * (ii + 1) / 2);
  }
  float* base = K + d.koff;
  const long long mp = d.mp;
  const float* xs = base + (long long)(i * K64) * mp + k * K64;
  const float* ys = TRSM ? Kinv + (d.kwrow + (long long)k * K64) * K64 : base + (long long)(j * K64) * mp + k * K64;
  const long long ldy = TRSM ? K64 : mp;
  float* out = base + (long long)(i * K64) * mp + (TRSM ? k : j) * K64;
  const int t = threadIdx.x;
  grid_dep_wait();
#pragma unroll
  for (int q = 0; q < K64 * K64 / 4 / kG64Threads; ++q) {
    const int e = t + kG64Threads * q;
    const int r = e >> 4, c4 = (e & 15) * 4;
    g64_cp16(&Xs[r][c4], xs + r * mp + c4);
    g64_cp16(&Ys[r][c4], ys + r * ldy + c4);
  }
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  const int ti = t & 7, tj = t >> 3;
  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.0f;
#pragma unroll 1
  for (int q = 0; q < K64; q += 4) {
    float4 xv[8], yv[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) xv[a] = *reinterpret_cast<const float4*>(&Xs[ti + 8 * a][q]);
#pragma unroll
    for (int b = 0; b < 8; ++b) yv[b] = *reinterpret_cast<const float4*>(&Ys[tj + 8 * b][q]);
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        float v = acc[a][b];
        v = fmaf(xv[a].x, yv[b].x, v);
        v = fmaf(xv[a].y, yv[b].y, v);
        v = fmaf(xv[a].z, yv[b].z, v);
        v = fmaf(xv[a].w, yv[b].w, v);
        acc[a][b] = v;
      }
  }
  grid_dep_launch();
  __syncthreads();  // every read of Xs is done: it takes the output tile
  if (!TRSM) {
#pragma unroll
    for (int q = 0; q < K64 * K64 / 4 / kG64Threads; ++q) {
      const int e = t + kG64Threads * q;
      const int r = e >> 4, c4 = (e & 15) * 4;
      g64_cp16(&Cs[r][c4], out + r * mp + c4);
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
    __syncthreads();
  }
  const bool diag = !TRSM && (i == j);
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int r = ti + 8 * a, cc = tj + 8 * b;
      if (TRSM)
        Cs[r][cc] = acc[a][b];
      else if (!diag || cc <= r)
        Cs[r][cc] -= acc[a][b];
    }
  __syncthreads();
#pragma unroll 4
  for (int q = 0; q < K64 * K64 / 4 / kG64Threads; ++q) {
    const int e = t + kG64Threads * q;
    const int r = e >> 4, c4 = (e & 15) * 4;
    *reinterpret_cast<float4*>(out + (long long)r * mp + c4) = *reinterpret_cast<const float4*>(&Cs[r][c4]);
  }
}

cudaError_t k64_configure() {
  cudaError_t e = cudaFuncSetAttribute(k_gemm64<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, g64_smem<false>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gemm64<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, g64_smem<true>());
  return e;
}

bool is_k64_kernel(const void* f) {
  return f == (const void*)k_potrf64 || f == (const void*)k_gemm64<true> || f == (const void*)k_gemm64<false> ||
         is_kupdate_tc_kernel(f);
}

// kmaps (TMA maps of every chain's K) selects the tensor-core trailing update
// (k_chol_tc.cu, split TF32 operands, FP32-accurate); without them the
// update runs on the CUDA cores (k_gemm64<false>).
cudaError_t launch_chol_k64(float* K, float* Kinv, const CUtensorMap* kmaps, const ChainDesc* cd, int n_chains,
                            int max_tiles, int* status, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < max_tiles && e == cudaSuccess; ++k) {
    e = launch_pdl(k_potrf64, dim3(n_chains), dim3(RegPotrf64::kThreads), 0, s, K, Kinv, cd, k, status);
    const int below = max_tiles - 1 - k;
    if (below > 0 && e == cudaSuccess)
      e = launch_pdl(k_gemm64<true>, dim3(below, n_chains), dim3(kG64Threads), g64_smem<true>(), s, K, Kinv, cd, k);
    if (below > 0 && e == cudaSuccess) {
      if (kmaps)
        e = launch_kupdate_tc(kmaps, cd, n_chains, K64 * max_tiles, k, status, s);
      else
        e = launch_pdl(k_gemm64<false>, dim3(below * (below + 1) / 2, n_chains), dim3(kG64Threads),
                       g64_smem<false>(), s, K, Kinv, cd, k);
    }
  }
  return e;
}

}  // namespace bd
