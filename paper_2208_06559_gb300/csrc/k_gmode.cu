// k_gmode.cu -- the mixed path's tension iteration in rod space.
//
// The residual of the rigid-rod constraint needs only the rod vectors
//   Q(T) = Q* + dt C D F(T) = Q* - dt G T,   G = C D C^T U,
// (Q* = C r*, C the bead-to-rod difference operator, U the old rod
// directions), not the bead positions.  G (three planes of (N-1) x (N-1),
// formed from the positions beside K by k_form_k_pos) holds one third of the
// elements of D's upper triangle and each is used once per product, so the
// product G T streams a third fewer bytes and needs a third of the
// compensated arithmetic of the symmetric product D F.  Once the tensions
// have converged the positions are rebuilt from the rods:
//   r_0 = r*_0 + dt (D F)_0,  r_{k+1} = r_k + Q_k(T),
// so every rod keeps the length the iteration reached.
//
//   k_gemv_g         : w = G T (or w += G dT once the chain is accurate),
//                      one warp per row of a plane, plain FP32 or
//                      double-float sums as the chain's mode;
//   k_newton_residual_g : g_k = |Q*_k - dt w_k|^2 - 1, the iteration state;
//   k_finalize_g     : positions of converged chains from the rods.
#include "bd_internal.h"
#include "block_dev.h"
#include "rpy_dev.h"
#include "pdl.h"

namespace bd {

constexpr int kGvWarps = 8;
constexpr int kGvThreads = 32 * kGvWarps;
constexpr int kGvRowsPerWarp = 8;
constexpr int kGvRows = kGvWarps * kGvRowsPerWarp;  // 64 rows of one plane per CTA
constexpr int kGvLoads = 8;                          // float4 loads in flight per lane

struct DFg {
  float hi, lo;
};

// a += g * (th + tl): the product g * th exact with an FMA, its high part
// added with a two-sum, the rounding terms and g * tl in the low word.
__device__ __forceinline__ void dfg_add_prod(DFg& a, float g, float th, float tl) {
  const float p = g * th;
  const float e = fmaf(g, th, -p);
  const float s = a.hi + p;
  const float bp = s - a.hi;
  const float err = (a.hi - (s - bp)) + (p - bp);
  a.hi = s;
  a.lo += err + e + g * tl;
}

// Rows R = pl * mp + k of the three planes; a CTA takes 64 rows of one plane
// (mp is a multiple of 64).  T (or dT) is split into (hi, lo) floats in
// shared memory, the high words of all columns first, then the low words
// (consecutive lanes read consecutive 16-byte words).  Each warp streams its
// rows with kGvLoads 16-byte loads per lane issued before use; the lane
// partials are combined with a butterfly (two-sum in double-float mode),
// after which every lane holds the same sum.
__global__ void __launch_bounds__(kGvThreads) k_gemv_g(const float* __restrict__ G,
                                                       const ChainDesc* __restrict__ cd,
                                                       const double* __restrict__ T,
                                                       const double* __restrict__ dT,
                                                       double* __restrict__ w,
                                                       const int* __restrict__ state,
                                                       const int* __restrict__ mode) {
  extern __shared__ __align__(16) float4 tsm[];  // [mp / 4] hi words, then [mp / 4] lo words
  const int c = blockIdx.y;
  grid_dep_wait();
  if (state[c] >= NS_DONE) return;
  const ChainDesc d = cd[c];
  const int mp = d.mp, m = d.m, mp4 = mp >> 2;
  const int row0 = blockIdx.x * kGvRows;
  if (row0 >= 3 * mp) return;
  const int pl = row0 / mp, k0 = row0 - pl * mp;
  if (k0 >= m) return;  // padding rows only
  const int md = mode[c];
  const double* src = (md >= MOB_INC_DF ? dT : T) + d.roff;
  const int t = threadIdx.x;
  for (int e = t; e < mp4; e += kGvThreads) {
    float h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int col = 4 * e + q;
      const double v = col < m ? src[col] : 0.0;
      h[q] = (float)v;
      l[q] = (float)(v - (double)h[q]);
    }
    tsm[e] = make_float4(h[0], h[1], h[2], h[3]);
    tsm[mp4 + e] = make_float4(l[0], l[1], l[2], l[3]);
  }
  __syncthreads();
  const int warp = t >> 5, lane = t & 31;
  const float* Gp = G + 3 * d.koff + (long long)pl * mp * mp;
  const bool df = (md == MOB_FULL_DF || md == MOB_INC_DF);
  for (int rr = 0; rr < kGvRowsPerWarp; ++rr) {
    const int k = k0 + kGvRowsPerWarp * warp + rr;
    if (k >= m) break;
    const float4* row = reinterpret_cast<const float4*>(Gp + (long long)k * mp);
    DFg acc{0.0f, 0.0f};
    for (int base = 0; base < mp4; base += 32 * kGvLoads) {
      float4 g[kGvLoads];
#pragma unroll
      for (int j = 0; j < kGvLoads; ++j) {
        const int q = base + 32 * j + lane;
        g[j] = q < mp4 ? __ldcs(row + q) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int j = 0; j < kGvLoads; ++j) {
        const int q = base + 32 * j + lane;
        if (q >= mp4) break;
        const float4 th = tsm[q];
        if (df) {
          const float4 tl = tsm[mp4 + q];
          dfg_add_prod(acc, g[j].x, th.x, tl.x);
          dfg_add_prod(acc, g[j].y, th.y, tl.y);
          dfg_add_prod(acc, g[j].z, th.z, tl.z);
          dfg_add_prod(acc, g[j].w, th.w, tl.w);
        } else {
          acc.hi = fmaf(g[j].x, th.x, acc.hi);
          acc.hi = fmaf(g[j].y, th.y, acc.hi);
          acc.hi = fmaf(g[j].z, th.z, acc.hi);
          acc.hi = fmaf(g[j].w, th.w, acc.hi);
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float h2 = __shfl_xor_sync(0xffffffffu, acc.hi, o);
      const float l2 = __shfl_xor_sync(0xffffffffu, acc.lo, o);
      const float s = acc.hi + h2;
      const float bp = s - acc.hi;
      const float err = (acc.hi - (s - bp)) + (h2 - bp);
      acc.hi = s;
      acc.lo = acc.lo + l2 + err;
    }
    if (lane == 0) {
      const double v = (double)acc.hi + (double)acc.lo;
      double* wp = w + 3 * (long long)(d.roff + k) + pl;
      if (md >= MOB_INC_DF)
        *wp += v;
      else
        *wp = v;
    }
  }
  grid_dep_launch();
}

// One CTA per chain: Q_k = Q*_k - dt w_k, g_k = |Q_k|^2 - 1, max |g|, and the
// state machine of k_newton_residual (same stopping rule, same mode switch).
__global__ void __launch_bounds__(256) k_newton_residual_g(const double* __restrict__ rstar,
                                                           const double* __restrict__ w,
                                                           const ChainDesc* __restrict__ cd, Phys ph,
                                                           double* __restrict__ rhs,
                                                           int* __restrict__ state,
                                                           int* __restrict__ status,
                                                           const int* __restrict__ iters,
                                                           int* __restrict__ mode) {
  __shared__ double red[32];
  const int c = blockIdx.x;
  grid_dep_wait();
  const int st = state[c];
  if (st >= NS_DONE) return;
  if (status[c] != BD_OK) {
    if (threadIdx.x == 0) state[c] = NS_FAILED;
    return;
  }
  const ChainDesc d = cd[c];
  const double* rs = rstar + 3 * d.boff;
  const double inv2dt = 0.5 / ph.dt;
  double gmax = 0.0;
  for (int k = threadIdx.x; k < d.m; k += blockDim.x) {
    const double* wk = w + 3 * (long long)(d.roff + k);
    const double q0 = (rs[3 * k + 3] - rs[3 * k]) - ph.dt * wk[0];
    const double q1 = (rs[3 * k + 4] - rs[3 * k + 1]) - ph.dt * wk[1];
    const double q2 = (rs[3 * k + 5] - rs[3 * k + 2]) - ph.dt * wk[2];
    const double g = q0 * q0 + q1 * q1 + q2 * q2 - 1.0;
    rhs[d.roff + k] = g * inv2dt;
    gmax = (g != g) ? INFINITY : fmax(gmax, fabs(g));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = gmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) gmax = fmax(gmax, red[i]);
    gmax = fmax(gmax, red[0]);
    int ns = st;
    const int md = mode[c];
    const bool acc_now = md != MOB_FULL_F32;
    if (st == NS_EXTRA) {
      ns = NS_DONE;
    } else if (gmax <= ph.tol && acc_now) {
      ns = NS_EXTRA;
    } else if (iters[c] >= ph.max_newton || !(gmax < INFINITY)) {
      ns = NS_FAILED;
      atomicCAS(status + c, BD_OK, BD_ERR_CONSTRAINT);
    }
    state[c] = ns;
    // The residual decides convergence only when it was evaluated accurately.
    // Products: plain FP32 while the residual is large, then one full
    // double-float product, then increments G dT of size ~|g|: double-float
    // while |g| >= 1e-10, plain FP32 below (error ~1e-7 of an increment below
    // 1e-10, far under the tolerance).
    if (md == MOB_FULL_F32)
      mode[c] = (gmax < 1e-5) ? MOB_FULL_DF : MOB_FULL_F32;
    else
      mode[c] = (gmax < 1e-10) ? MOB_INC_F32 : MOB_INC_DF;
  }
}

// One CTA (1024 threads) per chain, converged chains only: bead 0 moves by
// dt (D F)_0 (D_0j, Eqs. (7)-(9), evaluated in FP64 from the positions whose
// mobility the step uses; D_00 = I) and the rods Q_k = Q*_k - dt w_k are
// summed from it.  Failed chains keep their
// positions; the step index advances as in k_finalize.
constexpr int kFinThreads = 1024;
constexpr int kFinPer = 8;  // beads per thread (N <= 8192)

__global__ void __launch_bounds__(kFinThreads) k_finalize_g(const ChainDesc* __restrict__ cd, Phys ph,
                                                            const double* __restrict__ rpos,
                                                            const double* __restrict__ rstar,
                                                            const double* __restrict__ w,
                                                            const double* __restrict__ F,
                                                            double* __restrict__ r,
                                                            const int* __restrict__ state,
                                                            int* __restrict__ status, StepArgs* args) {
  __shared__ double red[32][3];
  const int c = blockIdx.x;
  const ChainDesc d = cd[c];
  const int st = state[c];
  if (threadIdx.x == 0 && st != NS_DONE && st != NS_FAILED)
    atomicCAS(status + c, BD_OK, BD_ERR_CONSTRAINT);  // loop ended early (not expected)
  if (args && c == 0 && threadIdx.x == 0) {
    args->step += 1;
    args->loops_in_step = 0;
  }
  if (st != NS_DONE) return;
  const int N = d.N, m = d.m, t = threadIdx.x;
  double* rc = r + 3 * d.boff;
  const double* rs = rstar + 3 * d.boff;
  const double* Fc = F + 3 * d.boff;
  // (D F)_0 with the RPY blocks D_0j (Sec. 3 Eqs. (8)-(9)) of rpos, in FP64
  double df[3] = {0.0, 0.0, 0.0};
  const double* rp = rpos + 3 * d.boff;
  for (int j = t; j < N; j += kFinThreads) {
    const double f0 = Fc[3 * j], f1 = Fc[3 * j + 1], f2 = Fc[3 * j + 2];
    if (j == 0) {
      df[0] += f0;
      df[1] += f1;
      df[2] += f2;
    } else {
      const double R0 = rp[0] - rp[3 * j], R1 = rp[1] - rp[3 * j + 1], R2 = rp[2] - rp[3 * j + 2];
      double cI, cRR;
      rpy_coeffs<double>(R0 * R0 + R1 * R1 + R2 * R2, ph.hstar, ph.a, cI, cRR);
      const double rf = cRR * (R0 * f0 + R1 * f1 + R2 * f2);
      df[0] += cI * f0 + rf * R0;
      df[1] += cI * f1 + rf * R1;
      df[2] += cI * f2 + rf * R2;
    }
  }
  block_sum3(df, red);
  // rods of this thread's beads i0 .. i0 + 3 (rod k joins bead k to k + 1)
  const int i0 = kFinPer * t;
  double q[kFinPer][3], off[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int j = 0; j < kFinPer; ++j) {
    const int k = i0 + j;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      q[j][a] = (k < m) ? (rs[3 * k + 3 + a] - rs[3 * k + a]) - ph.dt * w[3 * (long long)(d.roff + k) + a] : 0.0;
      off[a] += q[j][a];
    }
  }
  block_exscan3(off, red);
  const double b0[3] = {rs[0] + ph.dt * df[0], rs[1] + ph.dt * df[1], rs[2] + ph.dt * df[2]};
#pragma unroll
  for (int j = 0; j < kFinPer; ++j) {
    const int i = i0 + j;
    if (i < N) {
#pragma unroll
      for (int a = 0; a < 3; ++a) rc[3 * i + a] = b0[a] + off[a];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) off[a] += q[j][a];
  }
}

cudaError_t launch_tension_products_g(const float* G, const ChainDesc* cd, int n_chains, int max_mp,
                                      const double* T, const double* dT, double* w, const int* state,
                                      const int* mode, cudaStream_t s) {
  return launch_pdl(k_gemv_g, dim3(ceil_div(3 * max_mp, kGvRows), n_chains), dim3(kGvThreads),
                    (size_t)max_mp * 2 * sizeof(float), s, G, cd, T, dT, w, state, mode);
}

cudaError_t launch_newton_residual_g(const double* rstar, const double* w, const ChainDesc* cd,
                                     int n_chains, Phys ph, double* rhs, int* state, int* status,
                                     const int* iters, int* mode, cudaStream_t s) {
  return launch_pdl(k_newton_residual_g, dim3(n_chains), dim3(256), 0, s, rstar, w, cd, ph, rhs, state, status,
                    iters, mode);
}

cudaError_t launch_finalize_g(const ChainDesc* cd, int n_chains, Phys ph, const double* rpos, const double* rstar,
                              const double* w, const double* F, double* r, const int* state, int* status,
                              StepArgs* args, cudaStream_t s) {
  k_finalize_g<<<n_chains, kFinThreads, 0, s>>>(cd, ph, rpos, rstar, w, F, r, state, status, args);
  return cudaGetLastError();
}

cudaError_t gmode_configure() {
  // T split for chains of up to 8192 beads: 8192 x (hi, lo) floats
  return cudaFuncSetAttribute(k_gemv_g, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(8192 * 2 * sizeof(float)));
}

}  // namespace bd
