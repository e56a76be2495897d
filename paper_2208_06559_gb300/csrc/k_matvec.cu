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
#include "rpy_dev.h"

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
// FP64 path: K_kl = u_k^T (D_kl - D_k,l+1 - D_k+1,l + D_k+1,l+1) u_l for rods
// k >= l (the mixed path forms K from the positions, k_form_k_pos).
// CTA per 32 x 32 rod tile (kt >= lt): the 99 x 99 element region of D that
// the tile needs (beads 32 lt .. 32 lt + 32 against 32 kt .. 32 kt + 32) is
// staged in shared memory from the strict upper triangle with coalesced row
// loads; D_ab for a > b is the mirror block (RPY blocks are symmetric), D_aa = I.
constexpr int KR = 32;        // rods per tile side
constexpr int KE = 3 * KR + 3;  // 99 elements

template <typename T>
constexpr int form_k_smem() {
  return (int)(KE * (KE + 1) * sizeof(T) + 2 * KR * 3 * sizeof(T));
}

// Arithmetic in the storage type T.
template <typename T>
__global__ void __launch_bounds__(256) k_form_k(const T* __restrict__ M, T* __restrict__ K,
                                                const ChainDesc* __restrict__ cd,
                                                const double* __restrict__ uhat) {
  extern __shared__ __align__(16) uint8_t fk_smem[];
  T (*uk)[3] = reinterpret_cast<T (*)[3]>(fk_smem);
  T (*ul)[3] = reinterpret_cast<T (*)[3]>(fk_smem + KR * 3 * sizeof(T));
  T (*R)[KE + 1] = reinterpret_cast<T (*)[KE + 1]>(fk_smem + 2 * KR * 3 * sizeof(T));
  const ChainDesc d = cd[blockIdx.y];
  const int m = d.m;
  const int TK = (m + KR - 1) / KR;
  const int p = blockIdx.x;
  if (p >= TK * (TK + 1) / 2) return;
  int kt = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
  while (kt * (kt + 1) / 2 > p) --kt;
  while ((kt + 1) * (kt + 2) / 2 <= p) ++kt;
  const int lt = p - kt * (kt + 1) / 2;  // lt <= kt
  const T* base = M + d.moff;
  const long long np = d.np;
  // R[x][y] = U[3*32*lt + x][3*32*kt + y]: rows from the l side (smaller bead
  // indices), columns from the k side; only entries with row < col are D.
  const int row0 = 3 * KR * lt, col0 = 3 * KR * kt;
  // every element copied asynchronously (zero-filled outside the strict
  // upper triangle), so all of a thread's loads are in flight at once
  for (int x = threadIdx.x >> 5; x < KE; x += 8) {
    const int rr = row0 + x;
    for (int y = threadIdx.x & 31; y < KE; y += 32) {
      const int cc = col0 + y;
      const bool in = rr < d.n && cc < d.n && rr < cc;
      const T* src = in ? base + (long long)rr * np + cc : base;
      const unsigned dst = (unsigned)__cvta_generic_to_shared(&R[x][y]);
      if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(in ? 4 : 0)
                     : "memory");
      else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(in ? 8 : 0)
                     : "memory");
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  if (threadIdx.x < KR) {
    const int t = threadIdx.x;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      uk[t][q] = (KR * kt + t < m) ? (T)uhat[3 * (d.roff + KR * kt + t) + q] : T(0);
      ul[t][q] = (KR * lt + t < m) ? (T)uhat[3 * (d.roff + KR * lt + t) + q] : T(0);
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  // D_ab v for bead a on the k side (a = 32 kt + ia), b on the l side
  // (b = 32 lt + ib), ia, ib in [0, 32].
  auto blk_times = [&](int ia, int ib, const T* v, T out[3]) {
    const int a = KR * kt + ia, b = KR * lt + ib;
    if (a == b) {
      out[0] = v[0];
      out[1] = v[1];
      out[2] = v[2];
      return;
    }
    if (b < a) {  // D_ab = D_ba = U[3b..][3a..]
#pragma unroll
      for (int k = 0; k < 3; ++k)
        out[k] = R[3 * ib + k][3 * ia] * v[0] + R[3 * ib + k][3 * ia + 1] * v[1] +
                 R[3 * ib + k][3 * ia + 2] * v[2];
    } else {  // a < b: only on a diagonal tile (kt == lt): U[3a..][3b..]
#pragma unroll
      for (int k = 0; k < 3; ++k)
        out[k] = R[3 * ia + k][3 * ib] * v[0] + R[3 * ia + k][3 * ib + 1] * v[1] +
                 R[3 * ia + k][3 * ib + 2] * v[2];
    }
  };
  for (int e = threadIdx.x; e < KR * KR; e += blockDim.x) {
    const int ia = e / KR, ib = e % KR;  // rod k = 32 kt + ia, rod l = 32 lt + ib
    const int k = KR * kt + ia, l = KR * lt + ib;
    if (k >= m || l >= m || l > k) continue;
    T t0[3], t1[3], t2[3], t3[3];
    blk_times(ia, ib, ul[ib], t0);
    blk_times(ia, ib + 1, ul[ib], t1);
    blk_times(ia + 1, ib, ul[ib], t2);
    blk_times(ia + 1, ib + 1, ul[ib], t3);
    T sum = T(0);
#pragma unroll
    for (int q = 0; q < 3; ++q) sum += uk[ia][q] * (t0[q] - t1[q] - t2[q] + t3[q]);
    K[d.koff + (long long)k * d.mp + l] = sum;
  }
}

// K for the mixed path straight from the positions, so that it needs neither
// D nor the assembly and runs beside it: per 32 x 32 rod tile (kt >= lt) the
// 3 x 3 blocks D_xy = cI I + cRR R R^T of the 33 x 33 bead pairs the tile
// touches (Eqs. (8)-(9), FP32 from positions split into float pairs; D_aa =
// I) are formed once in shared memory as their six distinct entries; then
// per rod pair the second difference
//   B_kl = D_k,l - D_k,l+1 - D_k+1,l + D_k+1,l+1   (symmetric 3 x 3, = B_lk)
// gives
//   G_kl = B_kl u_l,  G_lk = B_kl u_k  (the rod-space mobility C D C^T U,
//                                        three planes [3][mp][mp], optional)
//   K_kl = u_k . G_kl  (lower triangle).
// K only preconditions the tension iteration; G, when formed, is the
// mobility the mixed path's tension iteration uses (its FP32 rounding is a
// ~1e-7 relative change of the model, far below the TF32 factor's).
constexpr int KB = KR + 1;  // beads per tile side

// WHAT selects the outputs (bit 0: K, bit 1: G); the variants are separate
// kernels so that the step graph can give the K chain's launches their own
// priority.
template <int WHAT>
__global__ void __launch_bounds__(256) k_form_k_pos(const double* __restrict__ r, float* __restrict__ K,
                                                    float* __restrict__ G,
                                                    const ChainDesc* __restrict__ cd,
                                                    const double* __restrict__ uhat, float hstar, float arad) {
  if (!(WHAT & 1)) K = nullptr;
  if (!(WHAT & 2)) G = nullptr;
  __shared__ float Ds[6][KB][KB];  // xx, xy, xz, yy, yz, zz of D_xy
  __shared__ float ph[2][KB][3], pl[2][KB][3];  // split positions: [0] k side, [1] l side
  __shared__ float uk[KR][3], ul[KR][3];
  __shared__ float St[3][KR][KR + 1];            // G_lk staged for a coalesced transposed store
  const ChainDesc d = cd[blockIdx.y];
  const int m = d.m, N = d.N;
  const int TK = (m + KR - 1) / KR;
  const int p = blockIdx.x;
  if (p >= TK * (TK + 1) / 2) return;
  int kt = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
  while (kt * (kt + 1) / 2 > p) --kt;
  while ((kt + 1) * (kt + 2) / 2 <= p) ++kt;
  const int lt = p - kt * (kt + 1) / 2;  // lt <= kt
  const int t = threadIdx.x;
  const double* rc = r + 3 * d.boff;
  if (t < 2 * KB * 3) {
    const int side = t / (KB * 3), e = t % (KB * 3), bead = e / 3, q = e % 3;
    const int gb = (side == 0 ? KR * kt : KR * lt) + bead;
    const double v = gb < N ? rc[3 * gb + q] : 0.0;
    const float h = (float)v;
    ph[side][bead][q] = h;
    pl[side][bead][q] = (float)(v - (double)h);
  }
  if (t < KR) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      uk[t][q] = (KR * kt + t < m) ? (float)uhat[3 * (d.roff + KR * kt + t) + q] : 0.0f;
      ul[t][q] = (KR * lt + t < m) ? (float)uhat[3 * (d.roff + KR * lt + t) + q] : 0.0f;
    }
  }
  __syncthreads();
  const float inv_a = 1.0f / arad;
  for (int e = t; e < KB * KB; e += blockDim.x) {
    const int x = e / KB, y = e % KB;
    const int a = KR * kt + x, b = KR * lt + y;
    float dv[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (a < N && b < N) {
      if (a == b) {
        dv[0] = dv[3] = dv[5] = 1.0f;
      } else {
        float R[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) R[q] = (ph[0][x][q] - ph[1][y][q]) + (pl[0][x][q] - pl[1][y][q]);
        float ci, cr;
        rpy_coeffs_rsqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2], hstar, arad, inv_a, ci, cr);
        const float c0 = cr * R[0], c1 = cr * R[1];
        dv[0] = fmaf(c0, R[0], ci);
        dv[1] = c0 * R[1];
        dv[2] = c0 * R[2];
        dv[3] = fmaf(c1, R[1], ci);
        dv[4] = c1 * R[2];
        dv[5] = fmaf(cr * R[2], R[2], ci);
      }
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) Ds[q][x][y] = dv[q];
  }
  __syncthreads();
  const long long mp = d.mp;
  float* Gc = G ? G + 3 * d.koff : nullptr;  // plane q at Gc + q mp^2
  for (int e = t; e < KR * KR; e += blockDim.x) {
    const int ia = e / KR, ib = e % KR;  // rod k = 32 kt + ia, rod l = 32 lt + ib
    const int k = KR * kt + ia, l = KR * lt + ib;
    const bool valid = k < m && l < m && l <= k;
    float B[6];
#pragma unroll
    for (int q = 0; q < 6; ++q)
      B[q] = (Ds[q][ia][ib] - Ds[q][ia][ib + 1]) + (Ds[q][ia + 1][ib + 1] - Ds[q][ia + 1][ib]);
    const float u0 = uk[ia][0], u1 = uk[ia][1], u2 = uk[ia][2];
    const float v0 = ul[ib][0], v1 = ul[ib][1], v2 = ul[ib][2];
    const float bv[3] = {B[0] * v0 + B[1] * v1 + B[2] * v2, B[1] * v0 + B[3] * v1 + B[4] * v2,
                         B[2] * v0 + B[4] * v1 + B[5] * v2};  // B u_l
    if (valid) {
      if (K) K[d.koff + (long long)k * mp + l] = u0 * bv[0] + u1 * bv[1] + u2 * bv[2];
      if (Gc) {
#pragma unroll
        for (int q = 0; q < 3; ++q) Gc[q * mp * mp + (long long)k * mp + l] = bv[q];
      }
    }
    if (Gc) {
      const bool lower = valid && l < k;
      St[0][ia][ib] = lower ? B[0] * u0 + B[1] * u1 + B[2] * u2 : 0.0f;  // B u_k
      St[1][ia][ib] = lower ? B[1] * u0 + B[3] * u1 + B[4] * u2 : 0.0f;
      St[2][ia][ib] = lower ? B[2] * u0 + B[4] * u1 + B[5] * u2 : 0.0f;
    }
  }
  if (!Gc) return;
  __syncthreads();
  // G_lk for the tile's pairs with l < k: row l, column k (transposed store)
  for (int e = t; e < KR * KR; e += blockDim.x) {
    const int ib = e / KR, ia = e % KR;
    const int k = KR * kt + ia, l = KR * lt + ib;
    if (k < m && l < m && l < k) {
#pragma unroll
      for (int q = 0; q < 3; ++q) Gc[q * mp * mp + (long long)l * mp + k] = St[q][ia][ib];
    }
  }
}

cudaError_t launch_form_k_pos(const double* r, float* K, float* G, const ChainDesc* cd, int n_chains,
                              int max_m, const double* u, double hstar, double a, cudaStream_t s) {
  const int TK = ceil_div(max_m, KR);
  const dim3 grid(TK * (TK + 1) / 2, n_chains);
  if (K && G)
    k_form_k_pos<3><<<grid, 256, 0, s>>>(r, K, G, cd, u, (float)hstar, (float)a);
  else if (K)
    k_form_k_pos<1><<<grid, 256, 0, s>>>(r, K, G, cd, u, (float)hstar, (float)a);
  else if (G)
    k_form_k_pos<2><<<grid, 256, 0, s>>>(r, K, G, cd, u, (float)hstar, (float)a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_form_k(const T* M, T* K, const ChainDesc* cd, int n_chains, int max_m,
                          const double* u, cudaStream_t s) {
  const int TK = ceil_div(max_m, KR);
  k_form_k<T><<<dim3(TK * (TK + 1) / 2, n_chains), 256, form_k_smem<T>(), s>>>(M, K, cd, u);
  return cudaGetLastError();
}

template cudaError_t launch_trmv<double>(const double*, const ChainDesc*, int, int, const double*,
                                         const StepArgs*, double, double*, cudaStream_t);
template cudaError_t launch_trmv<float>(const float*, const ChainDesc*, int, int, const double*,
                                        const StepArgs*, double, double*, cudaStream_t);
template cudaError_t launch_symv<double>(const double*, const ChainDesc*, int, int, const double*,
                                         double*, double*, const int*, cudaStream_t);
template cudaError_t launch_form_k<double>(const double*, double*, const ChainDesc*, int, int,
                                           const double*, cudaStream_t);

}  // namespace bd

namespace bd {

// ---------------------------------------------------- symv, FP32 storage
// u = D f for D stored in FP32 with FP32 arithmetic only (the FP64 pipe of
// this part runs at 1/64 of the FP32 rate), to a relative error of a few
// FP32 unit round-offs of the result, with no growth in the length of the sum:
//   k_split_f2      : f (FP64) -> (fh, fl) float pairs once per product,
//                     zero-padded to the chain's padded order;
//   k_symv_tiles_f32: per 64 x 64 tile of the upper triangle, groups of four
//                     products d*fh are summed in FP32 (three roundings of
//                     the group sum) and each group sum is added to a
//                     compensated (two-sum) accumulator; the d*fl terms go to
//                     a plain float beside it; row sums and column sums of
//                     the tile go out as (hi, lo) pairs;
//   k_symv_reduce_df: per row, compensated sum of its tile partials, one
//                     conversion to FP64.
// A tile is staged in shared memory (128 threads: thread t < 64 sums row t,
// thread t >= 64 column t - 64), so each element is read from HBM once and
// used twice; small CTAs let about a dozen share an SM, overlapping one
// tile's loads with another's sums.  Diagonal tiles are symmetrised in
// shared memory (mirror of the upper part, unit diagonal) and only row sums
// are taken.
constexpr int SF = 64;
constexpr int SFP = SF + 4;  // row pitch: 16-byte aligned rows for float4 access

struct DF {
  float hi, lo;
};

// a += d0 f0 + d1 f1 + d2 f2 + d3 f3, f = (h0, l0, h1, l1), (h2, l2, h3, l3):
// the high products summed in FP32, the sum added to a with a two-sum, the
// low products accumulated in `lo` (folded into a.lo at the end).
__device__ __forceinline__ void df_add4(DF& a, float& lo, float d0, float d1, float d2, float d3, float4 f01,
                                        float4 f23) {
  const float p = fmaf(d3, f23.z, fmaf(d2, f23.x, fmaf(d1, f01.z, d0 * f01.x)));
  lo = fmaf(d3, f23.w, fmaf(d2, f23.y, fmaf(d1, f01.w, fmaf(d0, f01.y, lo))));
  const float s = a.hi + p;
  const float bp = s - a.hi;
  a.lo += (a.hi - (s - bp)) + (p - bp);
  a.hi = s;
}

// (bj, bi), bi <= bj, of upper-triangle tile p (column-major enumeration),
// in FP32 with an exact integer correction.
__device__ __forceinline__ void upper_tile_of(int p, int& bi, int& bj) {
  int j = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
  while (j * (j + 1) / 2 > p) --j;
  while ((j + 1) * (j + 2) / 2 <= p) ++j;
  bj = j;
  bi = p - j * (j + 1) / 2;
}

__global__ void k_split_f2(const ChainDesc* __restrict__ cd, const double* __restrict__ f,
                           float2* __restrict__ fs, const int* __restrict__ state) {
  const int c = blockIdx.y;
  if (state && state[c] >= NS_DONE) return;
  const ChainDesc d = cd[c];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.np) return;
  const double v = (e < d.n) ? f[3 * d.boff + e] : 0.0;
  const float h = (float)v;
  fs[d.swrow + e] = make_float2(h, (float)(v - (double)h));
}

// Asynchronous 16- and 8-byte global -> shared copies (cp.async), grouped.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

constexpr int kSymvCtasPerSm = 5;

// Tile `id` of the batch (chain-major, tpc tiles per chain slot): its chain,
// block row and column; false if the chain has fewer tiles or is not active.
__device__ __forceinline__ bool symv_tile(int id, int tpc, const ChainDesc* __restrict__ cd,
                                          const int* __restrict__ state, int& c, int& bi, int& bj) {
  c = id / tpc;
  const int p = id - c * tpc;
  if (state && state[c] >= NS_DONE) return false;
  const int TSn = (cd[c].n + SF - 1) / SF;
  if (p >= TSn * (TSn + 1) / 2) return false;
  upper_tile_of(p, bi, bj);
  return true;
}

// Persistent: CTA b takes tiles b, b + grid, ...; the next tile (and its two
// f segments) is copied into the other shared-memory stage while the current
// one is summed.
__global__ void __launch_bounds__(128) k_symv_tiles_f32(const float* __restrict__ M,
                                                        const ChainDesc* __restrict__ cd, int n_chains,
                                                        int tpc, const float2* __restrict__ fs,
                                                        float2* __restrict__ P,
                                                        const int* __restrict__ state) {
  __shared__ __align__(16) float S[2][SF][SFP];
  __shared__ __align__(16) float2 fr[2][SF], fc[2][SF];  // (hi, lo) of f at the tile's rows / columns
  const int t = threadIdx.x;
  const int total = n_chains * tpc;
  auto issue = [&](int id, int buf) {
    int c, bi, bj;
    if (id < total && symv_tile(id, tpc, cd, state, c, bi, bj)) {
      const ChainDesc& d = cd[c];
      const float* base = M + d.moff + (long long)(bi * SF) * d.np + bj * SF;
#pragma unroll
      for (int q = 0; q < SF * SF / 4 / 128; ++q) {
        const int e = t + 128 * q;
        const int r = e >> 4, c4 = e & 15;
        cp_async16(&S[buf][r][4 * c4], base + (long long)r * d.np + 4 * c4);
      }
      if (t < SF)
        cp_async8(&fr[buf][t], fs + d.swrow + bi * SF + t);
      else
        cp_async8(&fc[buf][t - SF], fs + d.swrow + bj * SF + (t - SF));
    }
    cp_async_commit();
  };
  int k = 0;
  issue(blockIdx.x, 0);
  for (int id = blockIdx.x; id < total; id += gridDim.x, ++k) {
    const int buf = k & 1;
    issue(id + gridDim.x, buf ^ 1);
    cp_async_wait1();
    __syncthreads();
    int c, bi, bj;
    if (symv_tile(id, tpc, cd, state, c, bi, bj)) {
      const ChainDesc& d = cd[c];
      const int TSn = (d.n + SF - 1) / SF;
      const bool diag = (bi == bj);
      float (*Sb)[SFP] = S[buf];
      if (diag) {  // uniform over the CTA
        for (int e = t; e < SF * SF; e += 128) {
          const int r = e >> 6, cc = e & 63;
          if (cc < r) Sb[r][cc] = Sb[cc][r];
        }
        __syncthreads();
        if (t < SF) Sb[t][t] = 1.0f;
        __syncthreads();
      }
      const int r0 = bi * SF, c0 = bj * SF;
      const long long ld = (long long)TSn * SF;
      float2* Pc = P + d.soff;
      const float4* fc4 = reinterpret_cast<const float4*>(fc[buf]);  // (h0, l0, h1, l1)
      const float4* fr4 = reinterpret_cast<const float4*>(fr[buf]);
      {
        if (t < SF) {
          DF acc{0.f, 0.f};
          float lo = 0.f;
#pragma unroll 4
          for (int q4 = 0; q4 < SF / 4; ++q4) {
            const float4 v = *reinterpret_cast<const float4*>(&Sb[t][4 * q4]);
            df_add4(acc, lo, v.x, v.y, v.z, v.w, fc4[2 * q4], fc4[2 * q4 + 1]);
          }
          Pc[bj * ld + r0 + t] = make_float2(acc.hi, acc.lo + lo);  // rows of bi from column block bj
        } else if (!diag) {
          const int q = t - SF;
          DF acc{0.f, 0.f};
          float lo = 0.f;
#pragma unroll 4
          for (int r = 0; r < SF; r += 4)
            df_add4(acc, lo, Sb[r][q], Sb[r + 1][q], Sb[r + 2][q], Sb[r + 3][q], fr4[r >> 1], fr4[(r >> 1) + 1]);
          Pc[bi * ld + c0 + q] = make_float2(acc.hi, acc.lo + lo);  // rows of bj from column block bi
        }
      }
    }
    __syncthreads();  // stage `buf` is refilled by the issue of the next iteration
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

__global__ void k_symv_reduce_df(const ChainDesc* __restrict__ cd, const float2* __restrict__ P,
                                 double* __restrict__ u, const int* __restrict__ state) {
  const int c = blockIdx.y;
  if (state && state[c] >= NS_DONE) return;
  const ChainDesc d = cd[c];
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= d.n) return;
  const int TSn = (d.n + SF - 1) / SF;
  const long long ld = (long long)TSn * SF;
  const float2* Pc = P + d.soff;
  float hi = 0.f, lo = 0.f;
  for (int t = 0; t < TSn; ++t) {
    const float2 v = Pc[t * ld + row];
    const float s = hi + v.x;
    const float bp = s - hi;
    lo += ((hi - (s - bp)) + (v.x - bp)) + v.y;
    hi = s;
  }
  u[3 * d.boff + row] = (double)hi + (double)lo;
}

cudaError_t launch_split_f2(const ChainDesc* cd, int n_chains, int max_np, const double* v,
                            float2* out, const int* state, cudaStream_t s) {
  k_split_f2<<<dim3(ceil_div(max_np, 256), n_chains), 256, 0, s>>>(cd, v, out, state);
  return cudaGetLastError();
}

cudaError_t launch_symv_f32(const float* M, const ChainDesc* cd, int n_chains, int max_np,
                            const double* f, float2* fsplit, double* scratch, double* u,
                            const int* state, cudaStream_t s) {
  const int TSn = ceil_div(max_np, SF);
  float2* P = reinterpret_cast<float2*>(scratch);
  k_split_f2<<<dim3(ceil_div(max_np, 256), n_chains), 256, 0, s>>>(cd, f, fsplit, state);
  static int n_sm = 0;
  if (!n_sm) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n_sm <= 0)
      n_sm = 1;
  }
  const int tpc = TSn * (TSn + 1) / 2;
  const long long total = (long long)tpc * n_chains;
  const int grid = (int)(total < (long long)kSymvCtasPerSm * n_sm ? total : (long long)kSymvCtasPerSm * n_sm);
  k_symv_tiles_f32<<<grid, 128, 0, s>>>(M, cd, n_chains, tpc, fsplit, P, state);
  k_symv_reduce_df<<<dim3(ceil_div(max_np, 256), n_chains), 256, 0, s>>>(cd, P, u, state);
  return cudaGetLastError();
}

bool is_kchain_form_kernel(const void* f) {
  return f == (const void*)k_form_k_pos<3> || f == (const void*)k_form_k_pos<1>;
}

cudaError_t matvec_configure() {
  return cudaFuncSetAttribute(k_form_k<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              form_k_smem<double>());
}

}  // namespace bd
