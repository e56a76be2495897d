// k_chol_simt.cu -- blocked right-looking Cholesky on the CUDA cores
// (Sec. 3 Eq. (10): D = sigma sigma^T with sigma lower triangular).
//
// The paper calls cuSOLVER's dpotrf, whose internal trsm and dgemm kernels it
// profiles in Sec. 4 (Tables 2-3).  This is the library's own blocked
// factorisation for the FP64 path and for the rod-coupling matrix K: tiles of
// 32 x 32, and per block column k three launches over every chain of the
// batch at once:
//   potrf : factor the diagonal tile (always in FP64 arithmetic);
//   trsm  : L_ik = A_ik L_kk^{-T} for the tiles below it;
//   update: A_ij -= L_ik L_jk^T for the trailing lower tiles (i >= j > k).
// The matrix is row-major; only the lower triangle is read or written, so the
// strict upper triangle (which holds D) survives the factorisation.
#include <math.h>

#include "bd_internal.h"

namespace bd {

constexpr int TS = kSimtTile;

template <typename T>
__device__ __forceinline__ void matrix_of(const ChainDesc& d, bool kmat, T* M, T*& base,
                                          int& np) {
  base = M + (kmat ? d.koff : d.moff);
  np = kmat ? d.mp : d.np;
}

__device__ __forceinline__ void flag_status(int* status, int c, int code) {
  atomicCAS(status + c, BD_OK, code);
}

template <typename T>
__global__ void __launch_bounds__(256) k_potrf(T* M, const ChainDesc* __restrict__ cd, int k,
                                               bool kmat, int* status) {
  __shared__ double A[TS][TS + 1];
  __shared__ int bad;
  const ChainDesc d = cd[blockIdx.x];
  T* base;
  int np;
  matrix_of(d, kmat, M, base, np);
  if (k * TS >= np) return;
  base += (long long)(k * TS) * np + k * TS;
  const int tx = threadIdx.x, ty = threadIdx.y;
  if (tx == 0 && ty == 0) bad = 0;
  for (int r = ty; r < TS; r += 8) A[r][tx] = (tx <= r) ? (double)base[(long long)r * np + tx] : 0.0;
  __syncthreads();
  for (int j = 0; j < TS; ++j) {
    if (tx == 0 && ty == 0) {
      double dj = A[j][j];
      if (!(dj > 0.0)) {  // non-positive or NaN pivot
        bad = 1;
        dj = 1.0;
      }
      A[j][j] = sqrt(dj);
    }
    __syncthreads();
    if (ty == 0 && tx > j) A[tx][j] /= A[j][j];
    __syncthreads();
    for (int r = ty; r < TS; r += 8)
      if (r > j && tx > j && tx <= r) A[r][tx] -= A[r][j] * A[tx][j];
    __syncthreads();
  }
  for (int r = ty; r < TS; r += 8)
    if (tx <= r) base[(long long)r * np + tx] = (T)A[r][tx];
  if (tx == 0 && ty == 0 && bad) flag_status(status, blockIdx.x, kmat ? BD_ERR_CONSTRAINT : BD_ERR_NOT_PD);
}

// X L_kk^T = A_ik, one tile per CTA, one row per thread (forward substitution
// along the row), FP64 arithmetic.
template <typename T>
__global__ void __launch_bounds__(32) k_trsm(T* M, const ChainDesc* __restrict__ cd, int k,
                                             bool kmat) {
  __shared__ double Lkk[TS][TS + 1];
  __shared__ double X[TS][TS + 1];
  const ChainDesc d = cd[blockIdx.y];
  T* base;
  int np;
  matrix_of(d, kmat, M, base, np);
  const int i = k + 1 + blockIdx.x;
  if (i * TS >= np) return;
  const T* lkk = base + (long long)(k * TS) * np + k * TS;
  T* aik = base + (long long)(i * TS) * np + k * TS;
  const int t = threadIdx.x;
  for (int r = 0; r < TS; ++r) {
    Lkk[r][t] = (t <= r) ? (double)lkk[(long long)r * np + t] : 0.0;
    X[r][t] = (double)aik[(long long)r * np + t];
  }
  __syncthreads();
  for (int c = 0; c < TS; ++c) {
    double s = X[t][c];
    for (int q = 0; q < c; ++q) s -= X[t][q] * Lkk[c][q];
    X[t][c] = s / Lkk[c][c];
  }
  __syncthreads();
  for (int r = 0; r < TS; ++r) aik[(long long)r * np + t] = (T)X[r][t];
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
  matrix_of(d, kmat, M, base, np);
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
cudaError_t launch_chol_simt(T* M, const ChainDesc* cd, int n_chains, int max_tiles, bool kmat,
                             int* status, cudaStream_t s) {
  for (int k = 0; k < max_tiles; ++k) {
    k_potrf<T><<<n_chains, dim3(32, 8), 0, s>>>(M, cd, k, kmat, status);
    const int below = max_tiles - 1 - k;
    if (below > 0) {
      k_trsm<T><<<dim3(below, n_chains), 32, 0, s>>>(M, cd, k, kmat);
      k_update<T><<<dim3(below * (below + 1) / 2, n_chains), dim3(16, 16), 0, s>>>(M, cd, k, kmat);
    }
  }
  return cudaGetLastError();
}

template cudaError_t launch_chol_simt<double>(double*, const ChainDesc*, int, int, bool, int*,
                                              cudaStream_t);
template cudaError_t launch_chol_simt<float>(float*, const ChainDesc*, int, int, bool, int*,
                                             cudaStream_t);

}  // namespace bd
