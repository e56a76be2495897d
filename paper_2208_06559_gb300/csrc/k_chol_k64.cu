// k_chol_k64.cu -- FP32 Cholesky of the rod-coupling matrix K on the CUDA
// cores, 64 x 64 tiles, for the mixed-precision path.
//
// K = U^T C^T D C U (order N - 1) is the Jacobian of the tension iteration at
// Q = u; it only sets the convergence rate, but for stretched chains its
// condition number grows like N^2, so its factor must be FP32-accurate (the
// TF32 tensor-core path is not).  Per block column k:
//   potrf64 : one CTA factors the 64 x 64 diagonal tile and forms its inverse
//             (the register-blocked routine of the 128-wide path);
//   trsm64  : L_ik = A_ik W_kk^T, 64 x 64 per CTA, 4 x 4 outputs per thread;
//   update64: A_ij -= L_ik L_jk^T for the trailing lower tiles.
// The 64 x 64 diagonal-tile inverses are kept for the tension solve.
#include "bd_internal.h"
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
  potrf_regs<K64>(base, d.mp, base, d.mp, wout, K64, sm);
  if (threadIdx.x == 0 && *reinterpret_cast<const int*>(sm + RegPotrf64::kFlag)) atomicCAS(status + c, BD_OK, BD_ERR_CONSTRAINT);
}

// 64 x 64 output tile, 256 threads, 4 x 4 outputs each.
// TRSM: X = A_ik W_kk^T (overwrites A_ik).  UPDATE: A_ij -= L_ik L_jk^T.
template <bool TRSM>
__global__ void __launch_bounds__(256) k_gemm64(float* __restrict__ K, const float* __restrict__ Kinv,
                                                const ChainDesc* __restrict__ cd, int k) {
  __shared__ float X[K64][K64 + 1];
  __shared__ float Y[K64][K64 + 1];
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
  const int t = threadIdx.x;
  for (int e = t; e < K64 * K64 / 4; e += 256) {
    const int r = e >> 4, c4 = (e & 15) * 4;
    const float4 a = *reinterpret_cast<const float4*>(xs + r * mp + c4);
    const float4 b = *reinterpret_cast<const float4*>(ys + r * ldy + c4);
    X[r][c4] = a.x; X[r][c4 + 1] = a.y; X[r][c4 + 2] = a.z; X[r][c4 + 3] = a.w;
    Y[r][c4] = b.x; Y[r][c4 + 1] = b.y; Y[r][c4 + 2] = b.z; Y[r][c4 + 3] = b.w;
  }
  __syncthreads();
  const int r0 = (t >> 4) * 4, c0 = (t & 15) * 4;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
#pragma unroll 4
  for (int m = 0; m < K64; ++m) {
    float xv[4], yv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) xv[a] = X[r0 + a][m];
#pragma unroll
    for (int b = 0; b < 4; ++b) yv[b] = Y[c0 + b][m];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] += xv[a] * yv[b];
  }
  float* out = base + (long long)(i * K64) * mp + (TRSM ? k : j) * K64;
  const bool diag = !TRSM && (i == j);
  if (TRSM) __syncthreads();  // all reads of A_ik done before it is overwritten (X holds it)
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      float* o = out + (long long)(r0 + a) * mp + c0 + b;
      if (TRSM) *o = acc[a][b];
      else if (!diag || c0 + b <= r0 + a) *o -= acc[a][b];
    }
}

cudaError_t k64_configure() { return cudaSuccess; }

bool is_k64_kernel(const void* f) {
  return f == (const void*)k_potrf64 || f == (const void*)k_gemm64<true> || f == (const void*)k_gemm64<false>;
}

cudaError_t launch_chol_k64(float* K, float* Kinv, const ChainDesc* cd, int n_chains, int max_tiles,
                            int* status, cudaStream_t s) {
  for (int k = 0; k < max_tiles; ++k) {
    k_potrf64<<<n_chains, RegPotrf64::kThreads, 0, s>>>(K, Kinv, cd, k, status);
    const int below = max_tiles - 1 - k;
    if (below > 0) {
      k_gemm64<true><<<dim3(below, n_chains), 256, 0, s>>>(K, Kinv, cd, k);
      k_gemm64<false><<<dim3(below * (below + 1) / 2, n_chains), 256, 0, s>>>(K, Kinv, cd, k);
    }
  }
  return cudaGetLastError();
}

}  // namespace bd
