// k_solve_sb.cu -- the mixed path's tension solve K delta = rhs with
// 256-wide super-blocks.
//
// K = L L^T (FP32 factor, 64-wide diagonal-block inverses W_J kept by the
// factorisation).  Once per step, after the factor, k_sb_inverse forms the
// explicit inverses V_S = L_SS^{-1} of the 256 x 256 diagonal super-blocks
// from the 64-wide pieces (column block j of V_S: V_jj = W_j and, down the
// column, V_ij = -W_i sum_{k=j}^{i-1} L_ik V_kj).  Every tension iteration
// then takes 2 x ceil(m / 256) super-steps instead of 2 x ceil(m / 64)
// dependent block steps:
//   forward  z_S = V_S (rhs_S - L[S, 0:256S] z)
//   backward x_S = V_S^T (z_S - L[256(S+1):m, S]^T x)
// Each super-step is two passes of independent 16-byte loads over all
// threads of a cluster of CL CTAs (2, 4 or 8; the off-diagonal part split by
// 64-wide column blocks or rows taken round-robin, the V_S product by rows
// round-robin), with the partial results exchanged through distributed
// shared memory and combined in rank order, so every CTA holds identical z
// and x.
// Rank 0 writes T += x, the update itself (for the incremental rod-space
// products) and F(T).
#include <cooperative_groups.h>

#include "bd_internal.h"
#include "pdl.h"

namespace bd {

constexpr int kSB = 256;             // super-block order
constexpr int kSBBlocks = kSB / 64;  // 64-wide blocks per super-block
constexpr int kTP = 65;              // shared-memory pitch of a 64 x 64 tile
constexpr int kSbInvThreads = 256;
constexpr int kSbInvSmem = 3 * 64 * kTP * (int)sizeof(float);
constexpr int kSbThreads = 1024;
constexpr int kSbMaxM = 8192;        // rods per chain (N <= 8192 beads)

// One CTA per (chain, super-block S, column block j): V_S's column block j,
// rows j .. end of the super-block, top-down.  Each finished block V_ij goes
// straight to V and is read back (from L2) as an operand of the blocks below
// it, so only three 64 x 64 tiles live in shared memory (four CTAs per SM).
__global__ void __launch_bounds__(kSbInvThreads) k_sb_inverse(const float* __restrict__ K,
                                                              const float* __restrict__ Kinv,
                                                              float* __restrict__ V,
                                                              const ChainDesc* __restrict__ cd) {
  extern __shared__ float sbi_smem[];
  float (*At)[kTP] = reinterpret_cast<float (*)[kTP]>(sbi_smem);
  float (*Bt)[kTP] = reinterpret_cast<float (*)[kTP]>(sbi_smem + 64 * kTP);
  float (*Wt)[kTP] = reinterpret_cast<float (*)[kTP]>(sbi_smem + 2 * 64 * kTP);
  const ChainDesc d = cd[blockIdx.y];
  const int S = blockIdx.x / kSBBlocks, j = blockIdx.x % kSBBlocks;
  const int nb = d.mp / 64;
  const int nbS = min(kSBBlocks, nb - kSBBlocks * S);
  if (nbS <= 0 || j >= nbS) return;
  const long long mp = d.mp;
  const float* L = K + d.koff;
  const float* W = Kinv + d.kwrow * 64;  // W_J row r at (64 J + r) * 64
  float* Vs = V + (d.kwrow + (long long)kSB * S) * kSB;  // V_S row r at r * kSB
  const int t = threadIdx.x, tr = t >> 4, tc = t & 15;
  const int J0 = kSBBlocks * S;
  grid_dep_wait();
  auto vblk = [&](int i) { return Vs + (long long)(64 * i) * kSB + 64 * j; };  // V_ij, row pitch kSB
  // V_jj = W_j (zero above the diagonal)
  for (int e = t; e < 64 * 16; e += kSbInvThreads) {
    const int r = e >> 4, c4 = (e & 15) * 4;
    *reinterpret_cast<float4*>(vblk(j) + (long long)r * kSB + c4) =
        *reinterpret_cast<const float4*>(W + (long long)(64 * (J0 + j) + r) * 64 + c4);
  }
  __syncthreads();  // V_jj is visible to the whole CTA before it is read back
  for (int i = j + 1; i < nbS; ++i) {
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
    for (int k = j; k < i; ++k) {  // acc += L_ik V_kj
      const float* Lik = L + (long long)(64 * (J0 + i)) * mp + 64 * (J0 + k);
      const float* Vk = vblk(k);
      for (int e = t; e < 64 * 64; e += kSbInvThreads) {
        const int r = e >> 6, cc = e & 63;
        At[r][cc] = Lik[(long long)r * mp + cc];
        Bt[r][cc] = __ldcg(Vk + (long long)r * kSB + cc);
      }
      __syncthreads();
#pragma unroll 4
      for (int q = 0; q < 64; ++q) {
        float av[4], bv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = At[4 * tr + a][q];
#pragma unroll
        for (int b = 0; b < 4; ++b) bv[b] = Bt[q][4 * tc + b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
      }
      __syncthreads();
    }
    // V_ij = -W_i acc
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) At[4 * tr + a][4 * tc + b] = acc[a][b];
    for (int e = t; e < 64 * 64; e += kSbInvThreads) {
      const int r = e >> 6, cc = e & 63;
      Wt[r][cc] = W[(long long)(64 * (J0 + i) + r) * 64 + cc];
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
#pragma unroll 4
    for (int q = 0; q < 64; ++q) {
      float av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = Wt[4 * tr + a][q];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = At[q][4 * tc + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
    }
    float* Vi = vblk(i);
#pragma unroll
    for (int a = 0; a < 4; ++a)
      *reinterpret_cast<float4*>(Vi + (long long)(4 * tr + a) * kSB + 4 * tc) =
          make_float4(-acc[a][0], -acc[a][1], -acc[a][2], -acc[a][3]);
    __syncthreads();  // V_ij visible; At and Wt free for the next row block
  }
}

__device__ __forceinline__ float dot4(const float4 a, const float4 b) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the cluster's CTAs of their partial results p[t] (distributed
// shared memory), in rank order in every CTA, so that all hold the same value.
template <int CL>
__device__ __forceinline__ float cluster_sum(cooperative_groups::cluster_group& cl, float* p, int rank, int t) {
  float s = 0.0f;
#pragma unroll
  for (int q = 0; q < CL; ++q) s += (q == rank) ? p[t] : cl.map_shared_rank(p, q)[t];
  return s;
}

template <int CL>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(kSbThreads)
    k_newton_solve_sb(const float* __restrict__ K, const float* __restrict__ V,
                      const ChainDesc* __restrict__ cd, Phys ph, const double* __restrict__ uhat,
                      const double* __restrict__ rhs, double* __restrict__ Tn, double* __restrict__ F,
                      int* __restrict__ state, int* __restrict__ iters, double* __restrict__ dT) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  extern __shared__ __align__(16) float sb_smem[];
  float* bs = sb_smem;            // [kSbMaxM] right-hand side
  float* zs = sb_smem + kSbMaxM;  // [kSbMaxM] z, overwritten by x super-block by super-block
  __shared__ __align__(16) float red[16][kSB];
  __shared__ __align__(16) float xb[2][kSB];  // exchanged partial results, by exchange parity
  __shared__ __align__(16) float sv[kSB];
  const int c = blockIdx.x / CL;
  grid_dep_wait();
  const int st = state[c];
  if (st != NS_ACTIVE && st != NS_EXTRA) return;  // the same for both CTAs of the cluster
  const ChainDesc d = cd[c];
  const int m = d.m;
  const long long mp = d.mp;
  const float* L = K + d.koff;
  const float* Vc = V + d.kwrow * kSB;
  const int nsb = (m + kSB - 1) / kSB;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  for (int e = t; e < nsb * kSB; e += kSbThreads) {
    bs[e] = (e < m) ? (float)rhs[d.roff + e] : 0.0f;
    zs[e] = 0.0f;
  }
  __syncthreads();
  int ex = 0;
  // ---- forward: z = L^{-1} rhs
  for (int S = 0; S < nsb; ++S) {
    const int R0 = kSB * S, nS = min(kSB, m - R0);
    const int nbj = R0 / 64;  // column blocks left of the super-block
    {
      const int half = lane >> 4, q = lane & 15;
      // rows r and r + 32 together; this CTA's column blocks j = rank, rank + CL, ...
      for (int r = warp; r < nS; r += 64) {
        const int r2 = r + 32;
        const float* La = L + (long long)(R0 + r) * mp + 4 * q;
        const float* Lb = L + (long long)(R0 + (r2 < nS ? r2 : r)) * mp + 4 * q;
        float a0 = 0.0f, a1 = 0.0f;
#pragma unroll 2
        for (int j = rank + CL * half; j < nbj; j += 2 * CL) {
          const float4 la = __ldg(reinterpret_cast<const float4*>(La + 64 * j));
          const float4 lb = __ldg(reinterpret_cast<const float4*>(Lb + 64 * j));
          const float4 zv = *reinterpret_cast<const float4*>(zs + 64 * j + 4 * q);
          a0 += dot4(la, zv);
          a1 += dot4(lb, zv);
        }
        a0 = warp_sum(a0);
        a1 = warp_sum(a1);
        if (lane == 0) {
          xb[ex & 1][r] = a0;
          if (r2 < nS) xb[ex & 1][r2] = a1;
        }
      }
    }
    cl.sync();
    if (t < kSB) {
      float s = 0.0f;
      if (t < nS) s = bs[R0 + t] - cluster_sum<CL>(cl, &xb[ex & 1][0], rank, t);
      sv[t] = s;
    }
    ++ex;
    __syncthreads();
    {
      // z_S = V_S s, rows r = CL k + rank; row r has nonzeros in columns <= r
      const float* VS = Vc + (long long)R0 * kSB;
      for (int k = warp; CL * k + rank < nS; k += 32) {
        const int r = CL * k + rank;
        const float* Vr = VS + (long long)r * kSB;
        const int n4 = 16 * (r / 64 + 1);
        float a = 0.0f;
        for (int q4 = lane; q4 < n4; q4 += 32)
          a += dot4(__ldg(reinterpret_cast<const float4*>(Vr + 4 * q4)),
                    *reinterpret_cast<const float4*>(sv + 4 * q4));
        a = warp_sum(a);
        if (lane == 0) xb[ex & 1][r] = a;
      }
    }
    cl.sync();
    if (t < nS) {
      const int owner = t % CL;
      zs[R0 + t] = owner == rank ? xb[ex & 1][t] : cl.map_shared_rank(&xb[ex & 1][0], owner)[t];
    }
    ++ex;
    __syncthreads();
  }
  // ---- backward: x = L^{-T} z
  const int cq = t & 63, rl = t >> 6;  // column quad, row lane (16)
  for (int S = nsb - 1; S >= 0; --S) {
    const int C0 = kSB * S, nS = min(kSB, m - C0);
    const int R1 = C0 + kSB;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (C0 + 4 * cq < mp) {
      const float* Lc = L + C0 + 4 * cq;
#pragma unroll 4
      for (int R = R1 + CL * rl + rank; R < m; R += 16 * CL) {
        const float4 lv = __ldg(reinterpret_cast<const float4*>(Lc + (long long)R * mp));
        const float xr = zs[R];
        acc.x = fmaf(lv.x, xr, acc.x);
        acc.y = fmaf(lv.y, xr, acc.y);
        acc.z = fmaf(lv.z, xr, acc.z);
        acc.w = fmaf(lv.w, xr, acc.w);
      }
    }
    *reinterpret_cast<float4*>(&red[rl][4 * cq]) = acc;
    __syncthreads();
    if (t < kSB) {
      float p = 0.0f;
#pragma unroll
      for (int g = 0; g < 16; ++g) p += red[g][t];
      xb[ex & 1][t] = p;
    }
    cl.sync();
    if (t < kSB) {
      float s = 0.0f;
      if (t < nS) s = zs[C0 + t] - cluster_sum<CL>(cl, &xb[ex & 1][0], rank, t);
      sv[t] = s;
    }
    ++ex;
    __syncthreads();
    // x_S = V_S^T s over rows r = CL (rl + 16 i) + rank; V_S[r][c] = 0 for c > r
    acc = make_float4(0.f, 0.f, 0.f, 0.f);
    {
      const float* VS = Vc + (long long)C0 * kSB + 4 * cq;
#pragma unroll 4
      for (int r = CL * rl + rank; r < nS; r += 16 * CL) {
        if (4 * cq <= r) {
          const float4 v = __ldg(reinterpret_cast<const float4*>(VS + (long long)r * kSB));
          const float sr = sv[r];
          acc.x = fmaf(v.x, sr, acc.x);
          acc.y = fmaf(v.y, sr, acc.y);
          acc.z = fmaf(v.z, sr, acc.z);
          acc.w = fmaf(v.w, sr, acc.w);
        }
      }
    }
    *reinterpret_cast<float4*>(&red[rl][4 * cq]) = acc;
    __syncthreads();
    if (t < kSB) {
      float p = 0.0f;
#pragma unroll
      for (int g = 0; g < 16; ++g) p += red[g][t];
      xb[ex & 1][t] = p;
    }
    cl.sync();
    if (t < nS) zs[C0 + t] = cluster_sum<CL>(cl, &xb[ex & 1][0], rank, t);
    ++ex;
    __syncthreads();
  }
  cl.sync();  // no CTA leaves while its partner may still read its shared memory
  grid_dep_launch();
  if (rank != 0) return;
  for (int k = t; k < m; k += kSbThreads) {
    Tn[d.roff + k] += (double)zs[k];
    if (dT) dT[d.roff + k] = (double)zs[k];
  }
  __syncthreads();
  for (int i = t; i < d.N; i += kSbThreads) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      double f = 0.0;
      if (i < m) f += Tn[d.roff + i] * uhat[3 * (d.roff + i) + q];
      if (i > 0) f -= Tn[d.roff + i - 1] * uhat[3 * (d.roff + i - 1) + q];
      F[3 * (d.boff + i) + q] = f;
    }
  }
  if (t == 0) iters[c] += 1;
}

cudaError_t launch_sb_inverse(const float* K, const float* Kinv, float* V, const ChainDesc* cd, int n_chains,
                              int max_mp, cudaStream_t s) {
  const int nsb = ceil_div(max_mp, kSB);
  return launch_pdl(k_sb_inverse, dim3(nsb * kSBBlocks, n_chains), dim3(kSbInvThreads), kSbInvSmem, s, K, Kinv, V,
                    cd);
}

// Cluster size of the solve: 2 CTAs per chain, doubled up to 8 while the
// solve's CTAs would fill at most three quarters of the SMs (a small batch
// of long chains streams K's factor through more SMs).
static int g_sb_sms = 0;

static int sb_cluster(int n_chains) {
  int cl = 2;
  const long long budget = (long long)(g_sb_sms > 0 ? g_sb_sms : 148) * 3 / 4;
  while (cl < 8 && (long long)n_chains * 2 * cl <= budget) cl *= 2;
  return cl;
}

cudaError_t launch_newton_solve_sb(const float* K, const float* V, const ChainDesc* cd, int n_chains, Phys ph,
                                   const double* uhat, const double* rhs, double* Tn, double* F, int* state,
                                   int* iters, double* dT, cudaStream_t s) {
  const size_t smem = 2 * kSbMaxM * sizeof(float);
  switch (sb_cluster(n_chains)) {
    case 2:
      return launch_pdl(k_newton_solve_sb<2>, dim3(2 * n_chains), dim3(kSbThreads), smem, s, K, V, cd, ph, uhat, rhs,
                        Tn, F, state, iters, dT);
    case 4:
      return launch_pdl(k_newton_solve_sb<4>, dim3(4 * n_chains), dim3(kSbThreads), smem, s, K, V, cd, ph, uhat, rhs,
                        Tn, F, state, iters, dT);
    default:
      return launch_pdl(k_newton_solve_sb<8>, dim3(8 * n_chains), dim3(kSbThreads), smem, s, K, V, cd, ph, uhat, rhs,
                        Tn, F, state, iters, dT);
  }
}

bool is_sb_inverse_kernel(const void* f) { return f == (const void*)k_sb_inverse; }

cudaError_t solve_sb_configure() {
  cudaError_t e = cudaFuncSetAttribute(k_sb_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, kSbInvSmem);
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&g_sb_sms, cudaDevAttrMultiProcessorCount, dev);
  const int smem = (int)(2 * kSbMaxM * sizeof(float));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_newton_solve_sb<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_newton_solve_sb<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_newton_solve_sb<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return e;
}

}  // namespace bd
