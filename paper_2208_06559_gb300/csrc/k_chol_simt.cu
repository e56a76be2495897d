// k_chol_simt.cu -- blocked right-looking Cholesky on the CUDA cores
// (Sec. 3 Eq. (10): D = sigma sigma^T with sigma lower triangular).
//
// The paper calls cuSOLVER's dpotrf, whose internal trsm and dgemm kernels it
// profiles in Sec. 4 (Tables 2-3).  This is the library's own blocked
// factorisation for the FP64 path and for the rod-coupling matrix K of the
// tension solve: tiles of 32 x 32, and per block column k three launches over
// every chain of the batch at once:
//   potrf : one warp factors the diagonal tile in registers (lane r holds
//           row r; pivots broadcast with shuffles) and forms its inverse
//           W_kk = L_kk^{-1}, stored for the panel solve and for later
//           triangular solves with the factor;
//   trsm  : L_ik = A_ik W_kk^T for the tiles below it (a product);
//   update: A_ij -= L_ik L_jk^T for the trailing lower tiles (i >= j > k).
// The matrix is row-major; only the lower triangle is read or written, so the
// strict upper triangle (which holds D) survives the factorisation.
#include <math.h>

#include "bd_internal.h"

namespace bd {

constexpr int TS = kSimtTile;

template <typename T>
__device__ __forceinline__ void matrix_of(const ChainDesc& d, bool kmat, T* M, T*& base, int& np,
                                          long long& wrow) {
  base = M + (kmat ? d.koff : d.moff);
  np = kmat ? d.mp : d.np;
  wrow = kmat ? d.kwrow : d.swrow;
}

template <typename T>
__global__ void __launch_bounds__(32) k_potrf(T* M, T* Winv, const ChainDesc* __restrict__ cd, int k,
                                              bool kmat, int* status) {
  __shared__ T Ls[TS][TS + 1];
  const ChainDesc d = cd[blockIdx.x];
  T* base;
  int np;
  long long wrow;
  matrix_of(d, kmat, M, base, np, wrow);
  if (k * TS >= np) return;
  base += (long long)(k * TS) * np + k * TS;
  const int lane = threadIdx.x;
  T a[TS];
#pragma unroll
  for (int c = 0; c < TS; ++c) a[c] = (c <= lane) ? base[(long long)lane * np + c] : T(0);
  bool bad = false;
#pragma unroll
  for (int j = 0; j < TS; ++j) {
    const T djj = __shfl_sync(0xffffffffu, a[j], j);
    const bool ok = djj > T(0);  // false for NaN too
    bad |= !ok;
    const T piv = sqrt(ok ? djj : T(1));
    const T inv = T(1) / piv;
    if (lane == j) a[j] = piv;
    else if (lane > j) a[j] *= inv;
#pragma unroll
    for (int c = j + 1; c < TS; ++c) {
      const T lc = __shfl_sync(0xffffffffu, a[j], c);
      if (lane >= c) a[c] -= a[j] * lc;
    }
  }
#pragma unroll
  for (int c = 0; c < TS; ++c) Ls[lane][c] = (c <= lane) ? a[c] : T(0);
  __syncwarp();
  // column `lane` of W = L^{-1}: L w = e_lane, w_i = 0 for i < lane
  T w[TS];
#pragma unroll
  for (int i = 0; i < TS; ++i) {
    T s = (i == lane) ? T(1) : T(0);
#pragma unroll
    for (int m = 0; m < i; ++m) s -= Ls[i][m] * w[m];
    w[i] = (i >= lane) ? s / Ls[i][i] : T(0);
  }
#pragma unroll
  for (int c = 0; c < TS; ++c)
    if (c <= lane) base[(long long)lane * np + c] = a[c];
  T* W = Winv + (wrow + (long long)k * TS) * TS;
#pragma unroll
  for (int i = 0; i < TS; ++i) W[i * TS + lane] = w[i];  // W[i][lane]
  const unsigned any_bad = __ballot_sync(0xffffffffu, bad);
  if (lane == 0 && any_bad)
    atomicCAS(status + blockIdx.x, BD_OK, kmat ? BD_ERR_CONSTRAINT : BD_ERR_NOT_PD);
}

// L_ik = A_ik W_kk^T, one 32 x 32 tile per CTA, 2 x 2 outputs per thread.
template <typename T>
__global__ void __launch_bounds__(256) k_trsm(T* M, const T* __restrict__ Winv,
                                              const ChainDesc* __restrict__ cd, int k, bool kmat) {
  __shared__ T A[TS][TS + 1];
  __shared__ T W[TS][TS + 1];
  const ChainDesc d = cd[blockIdx.y];
  T* base;
  int np;
  long long wrow;
  matrix_of(d, kmat, M, base, np, wrow);
  const int i = k + 1 + blockIdx.x;
  if (i * TS >= np) return;
  T* aik = base + (long long)(i * TS) * np + k * TS;
  const T* wk = Winv + (wrow + (long long)k * TS) * TS;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 16 x 16
  for (int e = ty * 16 + tx; e < TS * TS; e += 256) {
    const int r = e / TS, c = e % TS;
    A[r][c] = aik[(long long)r * np + c];
    W[r][c] = wk[e];
  }
  __syncthreads();
  T x00 = 0, x01 = 0, x10 = 0, x11 = 0;
#pragma unroll 8
  for (int m = 0; m < TS; ++m) {
    const T a0 = A[ty][m], a1 = A[ty + 16][m];
    const T w0 = W[tx][m], w1 = W[tx + 16][m];
    x00 += a0 * w0;
    x01 += a0 * w1;
    x10 += a1 * w0;
    x11 += a1 * w1;
  }
  aik[(long long)ty * np + tx] = x00;
  aik[(long long)ty * np + tx + 16] = x01;
  aik[(long long)(ty + 16) * np + tx] = x10;
  aik[(long long)(ty + 16) * np + tx + 16] = x11;
}

// A_ij -= L_ik L_jk^T, 32 x 32 output tile per CTA, 2 x 2 outputs per thread.
template <typename T>
__global__ void __launch_bounds__(256) k_update(T* M, const ChainDesc* __restrict__ cd, int k,
                                                bool kmat) {
  __shared__ T Li[TS][TS + 1];
  __shared__ T Lj[TS][TS + 1];
  const ChainDesc d = cd[blockIdx.y];
  T* base;
  int np;
  long long wrow;
  matrix_of(d, kmat, M, base, np, wrow);
  const int s = np / TS - k - 1;
  const int p = blockIdx.x;
  if (s <= 0 || p >= s * (s + 1) / 2) return;
  int ii = (int)((sqrt(8.0 * p + 1.0) - 1.0) * 0.5);
  while (ii * (ii + 1) / 2 > p) --ii;
  while ((ii + 1) * (ii + 2) / 2 <= p) ++ii;
  const int jj = p - ii * (ii + 1) / 2;
  const int i = k + 1 + ii, j = k + 1 + jj;
  const T* lik = base + (long long)(i * TS) * np + k * TS;
  const T* ljk = base + (long long)(j * TS) * np + k * TS;
  T* aij = base + (long long)(i * TS) * np + j * TS;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 16 x 16
  for (int e = ty * 16 + tx; e < TS * TS; e += 256) {
    const int r = e / TS, c = e % TS;
    Li[r][c] = lik[(long long)r * np + c];
    Lj[r][c] = ljk[(long long)r * np + c];
  }
  __syncthreads();
  T a00 = 0, a01 = 0, a10 = 0, a11 = 0;
#pragma unroll 8
  for (int q = 0; q < TS; ++q) {
    const T x0 = Li[ty][q], x1 = Li[ty + 16][q];
    const T y0 = Lj[tx][q], y1 = Lj[tx + 16][q];
    a00 += x0 * y0;
    a01 += x0 * y1;
    a10 += x1 * y0;
    a11 += x1 * y1;
  }
  const bool diag = (i == j);
  const int r0 = ty, r1 = ty + 16, c0 = tx, c1 = tx + 16;
  if (!diag || r0 >= c0) aij[(long long)r0 * np + c0] -= a00;
  if (!diag || r0 >= c1) aij[(long long)r0 * np + c1] -= a01;
  if (!diag || r1 >= c0) aij[(long long)r1 * np + c0] -= a10;
  if (!diag || r1 >= c1) aij[(long long)r1 * np + c1] -= a11;
}

template <typename T>
cudaError_t launch_chol_simt(T* M, T* Winv, const ChainDesc* cd, int n_chains, int max_tiles,
                             bool kmat, int* status, cudaStream_t s) {
  for (int k = 0; k < max_tiles; ++k) {
    k_potrf<T><<<n_chains, 32, 0, s>>>(M, Winv, cd, k, kmat, status);
    const int below = max_tiles - 1 - k;
    if (below > 0) {
      k_trsm<T><<<dim3(below, n_chains), dim3(16, 16), 0, s>>>(M, Winv, cd, k, kmat);
      k_update<T><<<dim3(below * (below + 1) / 2, n_chains), dim3(16, 16), 0, s>>>(M, cd, k, kmat);
    }
  }
  return cudaGetLastError();
}

template cudaError_t launch_chol_simt<double>(double*, double*, const ChainDesc*, int, int, bool,
                                              int*, cudaStream_t);
template cudaError_t launch_chol_simt<float>(float*, float*, const ChainDesc*, int, int, bool, int*,
                                             cudaStream_t);

}  // namespace bd
