// k_assemble.cu -- RPY diffusion-tensor assembly (Sec. 3 Eqs. (7)-(9)).
//
// The paper's "Diffusion Tensor" kernel (Sec. 4) releases one thread per
// scalar element of the dense 3(N+1) x 3(N+1) matrix and branches on i == j.
// Here one thread evaluates 3x3 bead-pair blocks (the separation, its norm
// and the two RPY coefficients are shared by the nine elements), a CTA stages
// a 32 x 32 bead tile (96 x 96 elements) in shared memory, and the tile is
// written twice with coalesced row stores: once at (i, j) and once transposed
// at (j, i).  The result is the full symmetric D in the chain's row-major
// matrix; the Cholesky later overwrites the lower triangle with the factor and
// the strict upper triangle keeps D.
#include <type_traits>

#include "bd_internal.h"
#include "rpy_dev.h"

namespace bd {

constexpr int kBeadTile = 32;
constexpr int kElTile = 3 * kBeadTile;  // 96 x 96 elements per tile
template <typename T>
constexpr int assemble_smem() {
  return kElTile * (kElTile + 1) * (int)sizeof(T);
}

// FP32 path: the positions arrive split into (hi, lo) float pairs (rs), and
// every difference is (x_i,hi - x_j,hi) + (x_i,lo - x_j,lo): exact for nearby
// beads (Sterbenz), FP32-accurate otherwise, with no FP64 arithmetic (the
// FP64 pipe of this part runs at 1/64 of the FP32 rate).
template <typename T>
__global__ void __launch_bounds__(256) k_assemble(const double* __restrict__ r, const float2* __restrict__ rs,
                                                  T* __restrict__ M, const ChainDesc* __restrict__ cd,
                                                  double hstar, double a) {
  using C = T;  // arithmetic type of the coefficients (FP64 or FP32)
  extern __shared__ __align__(16) uint8_t as_smem[];
  T (*S)[kElTile + 1] = reinterpret_cast<T (*)[kElTile + 1]>(as_smem);
  const ChainDesc d = cd[blockIdx.y];
  const int TB = (d.N + kBeadTile - 1) / kBeadTile;
  const int p = blockIdx.x;
  if (p >= TB * (TB + 1) / 2) return;
  int bi = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
  while (bi * (bi + 1) / 2 > p) --bi;
  while ((bi + 1) * (bi + 2) / 2 <= p) ++bi;
  const int bj = p - bi * (bi + 1) / 2;  // bj <= bi

  // 1024 bead pairs per tile, four per thread
  for (int q = 0; q < 4; ++q) {
    const int e = threadIdx.x + 256 * q;
    const int ty = e >> 5, tx = e & 31;
    const int i = bi * kBeadTile + ty, j = bj * kBeadTile + tx;
    T blk[9];
#pragma unroll
    for (int w = 0; w < 9; ++w) blk[w] = T(0);
    if (i < d.N && j < d.N) {
      if (i == j) {
        blk[0] = blk[4] = blk[8] = T(1);
      } else {
        C R[3], R2;
        if constexpr (sizeof(T) == 4) {
          const float2* ri = rs + d.swrow + 3 * i;
          const float2* rj = rs + d.swrow + 3 * j;
#pragma unroll
          for (int k = 0; k < 3; ++k) R[k] = (ri[k].x - rj[k].x) + (ri[k].y - rj[k].y);
          R2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
        } else {
          const double* ri = r + 3 * (d.boff + i);
          const double* rj = r + 3 * (d.boff + j);
          const double dx = ri[0] - rj[0], dy = ri[1] - rj[1], dz = ri[2] - rj[2];
          R[0] = dx;
          R[1] = dy;
          R[2] = dz;
          R2 = dx * dx + dy * dy + dz * dz;
        }
        C cI, cRR;
        rpy_coeffs<C>(R2, (C)hstar, (C)a, cI, cRR);
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int l = 0; l < 3; ++l) blk[3 * k + l] = (k == l ? cI : C(0)) + cRR * R[k] * R[l];
      }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int l = 0; l < 3; ++l) S[3 * ty + k][3 * tx + l] = blk[3 * k + l];
  }
  __syncthreads();

  // 16-byte row stores (4 floats or 2 doubles); rows and columns past the
  // logical order n are never written (the padded border keeps its identity
  // diagonal, and a tile may reach past the padded order of the FP64 layout)
  T* base = M + d.moff;
  const long long np = d.np;
  const int n = d.n;
  const int r0 = kElTile * bi, c0 = kElTile * bj;
  constexpr int V = 16 / (int)sizeof(T);
  constexpr int G = kElTile / V;  // vectors per tile row
  using VecT = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  auto store_rows = [&](int rbase, int cbase, bool transposed) {
    for (int e = threadIdx.x; e < kElTile * G; e += blockDim.x) {
      const int rr = e / G, g = e - rr * G;
      const int row = rbase + rr, col = cbase + V * g;
      if (row >= n || col >= n) continue;
      VecT vv;
      T* vp = reinterpret_cast<T*>(&vv);
#pragma unroll
      for (int q = 0; q < V; ++q) vp[q] = transposed ? S[V * g + q][rr] : S[rr][V * g + q];
      T* dst = base + (long long)row * np + col;
      if (col + V <= n) {
        *reinterpret_cast<VecT*>(dst) = vv;
      } else {
#pragma unroll
        for (int q = 0; q < V; ++q)
          if (col + q < n) dst[q] = vp[q];
      }
    }
  };
  store_rows(r0, c0, false);
  if (bi != bj) store_rows(c0, r0, true);
}

template <typename T>
cudaError_t launch_assemble(const double* r, T* M, const ChainDesc* cd, int n_chains, int max_N,
                            int max_np, double hstar, double a, float2* rsplit, cudaStream_t s) {
  if (sizeof(T) == 4) {
    if (!rsplit) return cudaErrorInvalidValue;
    const cudaError_t e = launch_split_f2(cd, n_chains, max_np, r, rsplit, nullptr, s);
    if (e != cudaSuccess) return e;
  }
  const int TB = (max_N + kBeadTile - 1) / kBeadTile;
  dim3 grid(TB * (TB + 1) / 2, n_chains);
  k_assemble<T><<<grid, 256, assemble_smem<T>(), s>>>(r, rsplit, M, cd, hstar, a);
  return cudaGetLastError();
}

// Identity border of a padded matrix: ones on the diagonal past the logical
// order (the rest of the border is zeroed by a memset at creation).
template <typename T>
__global__ void k_border(T* M, const ChainDesc* cd, bool kmat) {
  const ChainDesc d = cd[blockIdx.y];
  const int n = kmat ? d.m : d.n, np = kmat ? d.mp : d.np;
  T* base = M + (kmat ? d.koff : d.moff);
  for (int q = n + blockIdx.x * blockDim.x + threadIdx.x; q < np; q += gridDim.x * blockDim.x)
    base[(long long)q * np + q] = T(1);
}

template <typename T>
cudaError_t launch_fill_identity_border(T* M, const ChainDesc* cd, int n_chains, int max_np,
                                        bool kmat, cudaStream_t s) {
  (void)max_np;
  k_border<T><<<dim3(1, n_chains), 128, 0, s>>>(M, cd, kmat);
  return cudaGetLastError();
}

// Dense FP64 copy of D (which = 0) or of the factor B (which = 1) of one chain.
template <typename T>
__global__ void k_extract(const T* M, const ChainDesc* cd, int chain, int which, double* out) {
  const ChainDesc d = cd[chain];
  const T* base = M + d.moff;
  const long long total = (long long)d.n * d.n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / d.n), c = (int)(e % d.n);
    double v;
    if (which == 0) {
      v = (r == c) ? 1.0 : (double)(r < c ? base[(long long)r * d.np + c] : base[(long long)c * d.np + r]);
    } else {
      v = (r >= c) ? (double)base[(long long)r * d.np + c] : 0.0;
    }
    out[e] = v;
  }
}

template <typename T>
cudaError_t launch_extract(const T* M, const ChainDesc* cd, int chain, int which, double* out,
                           cudaStream_t s) {
  k_extract<T><<<256, 256, 0, s>>>(M, cd, chain, which, out);
  return cudaGetLastError();
}

template cudaError_t launch_assemble<double>(const double*, double*, const ChainDesc*, int, int, int,
                                             double, double, float2*, cudaStream_t);
template cudaError_t launch_assemble<float>(const double*, float*, const ChainDesc*, int, int, int,
                                            double, double, float2*, cudaStream_t);
template cudaError_t launch_fill_identity_border<double>(double*, const ChainDesc*, int, int, bool,
                                                         cudaStream_t);
template cudaError_t launch_fill_identity_border<float>(float*, const ChainDesc*, int, int, bool,
                                                        cudaStream_t);
template cudaError_t launch_extract<double>(const double*, const ChainDesc*, int, int, double*,
                                            cudaStream_t);
template cudaError_t launch_extract<float>(const float*, const ChainDesc*, int, int, double*,
                                           cudaStream_t);

cudaError_t assemble_configure() {
  cudaError_t e = cudaFuncSetAttribute(k_assemble<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       assemble_smem<double>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_assemble<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             assemble_smem<float>());
  return e;
}

}  // namespace bd
