// k_matvec.cu -- the matrix-vector products of the step.
//
// The paper forms Diff = D_{i+1,j} - D_{i,j} (and the same for sigma) as a
// dense link-space matrix, multiplies it elementwise into a dense "Mult"
// array and reduces its rows with a shared-memory tree (Sec. 4, Eqs.
// (21)-(24) and the Reduction algorithm).  Here nothing link-space is
// materialised: products are taken in bead space and held in registers, rows
// are reduced with warp shuffles, and the O(N) link differences are taken by
// the consumers.
//
//   trmv : y = s * B xi, B lower triangular (noise term of Eq. (6)), warp per row.
//   symv : u = D f with D read once from the strict upper triangle (unit
//          diagonal, Eq. (7)); deterministic two-phase reduction.
//   form_k: K_kl = u_k^T (D_kl - D_k,l+1 - D_k+1,l + D_k+1,l+1) u_l, the
//          rod-coupling matrix of the tension solve.
#include "bd_internal.h"

namespace bd {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------- trmv
// One warp per row, lanes stride the row (coalesced), FP64 accumulation.
template <typename T>
__global__ void __launch_bounds__(256) k_trmv(const T* __restrict__ M, const ChainDesc* __restrict__ cd,
                                              const double* __restrict__ x_in,
                                              const StepArgs* __restrict__ args, double scale,
                                              double* __restrict__ y) {
  const ChainDesc d = cd[blockIdx.y];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double* x = x_in;
  if (args) x = args->noise + (long long)args->step * args->stride;
  x += 3 * d.boff;
  const T* base = M + d.moff;
  for (int rr = 0; rr < 4; ++rr) {
    const int row = blockIdx.x * 32 + warp * 4 + rr;
    if (row >= d.n) return;
    const T* Lr = base + (long long)row * d.np;
    double acc = 0.0;
    for (int c = lane; c <= row; c += 32) acc += (double)Lr[c] * x[c];
    acc = warp_sum(acc);
    if (lane == 0) y[3 * d.boff + row] = scale * acc;
  }
}

template <typename T>
cudaError_t launch_trmv(const T* M, const ChainDesc* cd, int n_chains, int max_n, const double* x,
                        const StepArgs* args, double scale, double* y, cudaStream_t s) {
  k_trmv<T><<<dim3(ceil_div(max_n, 32), n_chains), 256, 0, s>>>(M, cd, x, args, scale, y);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- symv
// Phase 1: CTA per upper tile (bi <= bj) of 64 x 64.  It adds U_tile f[bj]
// into P[bj][rows of bi] and U_tile^T f[bi] into P[bi][rows of bj] (for the
// diagonal tile both, plus the unit diagonal, go to P[bi][rows of bi]).
// Each slot P[t][block b] is written by exactly one tile.
// Phase 2: u[rho] = sum_t P[t][rho] in a fixed order (deterministic).
constexpr int SY = kSymvTile;

template <typename T>
__global__ void __launch_bounds__(256) k_symv_tiles(const T* __restrict__ M,
                                                    const ChainDesc* __restrict__ cd,
                                                    const double* __restrict__ f,
                                                    double* __restrict__ P,
                                                    const int* __restrict__ state) {
  __shared__ double fr[SY], fc[SY];
  __shared__ double rowsum[SY];
  __shared__ double colpart[8][SY];
  const int c = blockIdx.y;
  if (state && state[c] >= NS_DONE) return;
  const ChainDesc d = cd[c];
  const int TSn = (d.n + SY - 1) / SY;
  const int p = blockIdx.x;
  if (p >= TSn * (TSn + 1) / 2) return;
  int bj = (int)((sqrt(8.0 * p + 1.0) - 1.0) * 0.5);
  while (bj * (bj + 1) / 2 > p) --bj;
  while ((bj + 1) * (bj + 2) / 2 <= p) ++bj;
  const int bi = p - bj * (bj + 1) / 2;  // bi <= bj
  const int r0 = bi * SY, c0 = bj * SY;
  const double* fb = f + 3 * d.boff;
  if (threadIdx.x < SY) {
    const int q = threadIdx.x;
    fr[q] = (r0 + q < d.n) ? fb[r0 + q] : 0.0;
    fc[q] = (c0 + q < d.n) ? fb[c0 + q] : 0.0;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool diag = (bi == bj);
  const T* base = M + d.moff;
  double cp0 = 0.0, cp1 = 0.0;
  for (int rr = warp * 8; rr < warp * 8 + 8; ++rr) {
    const int row = r0 + rr;
    double v0 = 0.0, v1 = 0.0;
    if (row < d.n) {
      const T* Ur = base + (long long)row * d.np + c0;
      const int ca = lane, cb = lane + 32;
      if (c0 + ca < d.n && (!diag || ca > rr)) v0 = (double)Ur[ca];
      if (c0 + cb < d.n && (!diag || cb > rr)) v1 = (double)Ur[cb];
    }
    const double rs = warp_sum(v0 * fc[lane] + v1 * fc[lane + 32]);
    if (lane == 0) rowsum[rr] = rs;
    cp0 += v0 * fr[rr];
    cp1 += v1 * fr[rr];
  }
  colpart[warp][lane] = cp0;
  colpart[warp][lane + 32] = cp1;
  __syncthreads();
  if (threadIdx.x < SY) {
    const int q = threadIdx.x;
    double cs = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) cs += colpart[w][q];
    const long long ld = (long long)TSn * SY;
    double* Pc = P + d.soff;
    if (diag) {
      Pc[bi * ld + r0 + q] = rowsum[q] + cs + fr[q];
    } else {
      Pc[bj * ld + r0 + q] = rowsum[q];  // rows of bi, from column block bj
      Pc[bi * ld + c0 + q] = cs;         // rows of bj, from column block bi
    }
  }
}

__global__ void k_symv_reduce(const ChainDesc* __restrict__ cd, const double* __restrict__ P,
                              double* __restrict__ u, const int* __restrict__ state) {
  const int c = blockIdx.y;
  if (state && state[c] >= NS_DONE) return;
  const ChainDesc d = cd[c];
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= d.n) return;
  const int TSn = (d.n + SY - 1) / SY;
  const long long ld = (long long)TSn * SY;
  const double* Pc = P + d.soff;
  double s = 0.0;
  for (int t = 0; t < TSn; ++t) s += Pc[t * ld + row];
  u[3 * d.boff + row] = s;
}

template <typename T>
cudaError_t launch_symv(const T* M, const ChainDesc* cd, int n_chains, int max_np, const double* f,
                        double* scratch, double* u, const int* state, cudaStream_t s) {
  const int TSn = ceil_div(max_np, SY);
  k_symv_tiles<T><<<dim3(TSn * (TSn + 1) / 2, n_chains), 256, 0, s>>>(M, cd, f, scratch, state);
  k_symv_reduce<<<dim3(ceil_div(max_np, 256), n_chains), 256, 0, s>>>(cd, scratch, u, state);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- form_k
// One thread per K_kl (k >= l).  D_ab for a != b is read from the strict
// upper triangle at (min, max) (RPY blocks are symmetric 3 x 3), D_aa = I.
template <typename T>
__device__ __forceinline__ void d_block_times(const T* base, long long np, int a, int b,
                                              const double* v, double out[3]) {
  if (a == b) {
    out[0] = v[0];
    out[1] = v[1];
    out[2] = v[2];
    return;
  }
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  const T* p = base + (long long)(3 * lo) * np + 3 * hi;
#pragma unroll
  for (int k = 0; k < 3; ++k)
    out[k] = (double)p[k * np] * v[0] + (double)p[k * np + 1] * v[1] + (double)p[k * np + 2] * v[2];
}

template <typename T>
__global__ void __launch_bounds__(256) k_form_k(const T* __restrict__ M, T* __restrict__ K,
                                                const ChainDesc* __restrict__ cd,
                                                const double* __restrict__ uhat) {
  const ChainDesc d = cd[blockIdx.y];
  const int m = d.m;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long npairs = (long long)m * (m + 1) / 2;
  if (idx >= npairs) return;
  int k = (int)((sqrt(8.0 * (double)idx + 1.0) - 1.0) * 0.5);
  while ((long long)k * (k + 1) / 2 > idx) --k;
  while ((long long)(k + 1) * (k + 2) / 2 <= idx) ++k;
  const int l = (int)(idx - (long long)k * (k + 1) / 2);  // l <= k
  const double* uk = uhat + 3 * (d.roff + k);
  const double* ul = uhat + 3 * (d.roff + l);
  const T* base = M + d.moff;
  const long long np = d.np;
  double t0[3], t1[3], t2[3], t3[3];
  d_block_times(base, np, k, l, ul, t0);
  d_block_times(base, np, k, l + 1, ul, t1);
  d_block_times(base, np, k + 1, l, ul, t2);
  d_block_times(base, np, k + 1, l + 1, ul, t3);
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < 3; ++q) s += uk[q] * (t0[q] - t1[q] - t2[q] + t3[q]);
  K[d.koff + (long long)k * d.mp + l] = (T)s;
}

template <typename T>
cudaError_t launch_form_k(const T* M, T* K, const ChainDesc* cd, int n_chains, int max_m,
                          const double* u, cudaStream_t s) {
  const long long npairs = (long long)max_m * (max_m + 1) / 2;
  k_form_k<T><<<dim3(ceil_div(npairs, 256), n_chains), 256, 0, s>>>(M, K, cd, u);
  return cudaGetLastError();
}

template cudaError_t launch_trmv<double>(const double*, const ChainDesc*, int, int, const double*,
                                         const StepArgs*, double, double*, cudaStream_t);
template cudaError_t launch_trmv<float>(const float*, const ChainDesc*, int, int, const double*,
                                        const StepArgs*, double, double*, cudaStream_t);
template cudaError_t launch_symv<double>(const double*, const ChainDesc*, int, int, const double*,
                                         double*, double*, const int*, cudaStream_t);
template cudaError_t launch_symv<float>(const float*, const ChainDesc*, int, int, const double*,
                                        double*, double*, const int*, cudaStream_t);
template cudaError_t launch_form_k<double>(const double*, double*, const ChainDesc*, int, int,
                                           const double*, cudaStream_t);
template cudaError_t launch_form_k<float>(const float*, float*, const ChainDesc*, int, int,
                                          const double*, cudaStream_t);

}  // namespace bd
