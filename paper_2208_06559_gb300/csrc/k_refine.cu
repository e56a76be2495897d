// k_refine.cu -- Brownian displacement for the mixed-precision path, with
// one step of iterative refinement against D.
//
// The noise term of Sec. 3 Eq. (6) is sqrt(2 dt) B xi with B B^T = D
// (Eq. (10)).  With a tensor-core factor Lt whose error is E = D - Lt Lt^T,
// the library uses
//     y = (s / 2) (Lt xi + D Lt^{-T} xi),  s = sqrt(2 dt),
// i.e. B_eff = (Lt + D Lt^{-T}) / 2, for which B_eff B_eff^T - D = E D'^{-1} E / 4
// (D' = Lt Lt^T): the error drops from first to second order in E, with the
// same xi, so the path stays comparable with the FP64 factor.
//
// All three products read FP32 matrices and accumulate in compensated FP32:
// each xi or z value is split into two floats; the triangular solve makes
// every product d * hi exact with an FMA and sums with two-sum (double-float,
// FP64-level), the two products by Lt and D sum groups of four products in
// FP32 before the two-sum (a few FP32 round-offs of the result, far below
// the refinement's second-order factor error) -- no FP64 arithmetic, which is
// slow on this part.
#include <cooperative_groups.h>

#include "bd_internal.h"

namespace bd {

struct DFa {
  float hi, lo;
};

__device__ __forceinline__ void dfa_add_prod(DFa& a, float d, float xh, float xl) {
  const float p = d * xh;
  const float e = fmaf(d, xh, -p);
  const float s = a.hi + p;
  const float bp = s - a.hi;
  const float err = (a.hi - (s - bp)) + (p - bp);
  a.hi = s;
  a.lo += err + e + d * xl;
}

// a += b for double-float values (two-sum of the high parts)
__device__ __forceinline__ void dfa_add(DFa& a, float bh, float bl) {
  const float s = a.hi + bh;
  const float bp = s - a.hi;
  a.lo += ((a.hi - (s - bp)) + (bh - bp)) + bl;
  a.hi = s;
}

// a += d0 x0 + d1 x1 + d2 x2 + d3 x3 with x = xh + xl: the high products
// summed in FP32 and added with a two-sum, the low ones into `lo`.
__device__ __forceinline__ void dfa_add4(DFa& a, float& lo, float d0, float d1, float d2, float d3, float h0,
                                         float h1, float h2, float h3, float l0, float l1, float l2,
                                         float l3) {
  const float p = fmaf(d3, h3, fmaf(d2, h2, fmaf(d1, h1, d0 * h0)));
  lo = fmaf(d3, l3, fmaf(d2, l2, fmaf(d1, l1, fmaf(d0, l0, lo))));
  const float s = a.hi + p;
  const float bp = s - a.hi;
  a.lo += (a.hi - (s - bp)) + (p - bp);
  a.hi = s;
}

__device__ __forceinline__ DFa dfa_warp_sum(DFa v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h = __shfl_xor_sync(0xffffffffu, v.hi, o);
    const float l = __shfl_xor_sync(0xffffffffu, v.lo, o);
    dfa_add(v, h, l);
  }
  return v;
}

// Split x (FP64) into two floats per value, x = xh + xl, into the chain's
// scratch region (xh at [0, n), xl at [n, 2n)), so the product loops below
// run on FP32 units only.
__global__ void k_split(const ChainDesc* __restrict__ cd, const double* __restrict__ x_in,
                        const StepArgs* __restrict__ args, double* __restrict__ scratch) {
  const ChainDesc d = cd[blockIdx.y];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.n) return;
  const double* x = args ? args->noise + (long long)args->step * args->stride : x_in;
  const double v = x[3 * d.boff + e];
  float* xs = reinterpret_cast<float*>(scratch + d.soff);
  const float h = (float)v;
  xs[e] = h;
  xs[d.n + e] = (float)(v - (double)h);
}

// y1 = Lt x, one warp per row, lanes stride the row.
__global__ void __launch_bounds__(256) k_trmv_f32(const float* __restrict__ M,
                                                  const ChainDesc* __restrict__ cd,
                                                  const double* __restrict__ scratch, double scale,
                                                  double* __restrict__ y) {
  const ChainDesc d = cd[blockIdx.y];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float* xh = reinterpret_cast<const float*>(scratch + d.soff);
  const float* xl = xh + d.n;
  const float* base = M + d.moff;
  for (int rr = 0; rr < 4; ++rr) {
    const int row = blockIdx.x * 32 + warp * 4 + rr;
    if (row >= d.n) return;
    const float* Lr = base + (long long)row * d.np;
    DFa acc{0.f, 0.f};
    float lo = 0.f;
    int c = lane;
    for (; c + 96 <= row; c += 128) {  // four loads in flight per lane
      const float v0 = __ldg(Lr + c), v1 = __ldg(Lr + c + 32), v2 = __ldg(Lr + c + 64),
                  v3 = __ldg(Lr + c + 96);
      dfa_add4(acc, lo, v0, v1, v2, v3, xh[c], xh[c + 32], xh[c + 64], xh[c + 96], xl[c], xl[c + 32],
               xl[c + 64], xl[c + 96]);
    }
    for (; c <= row; c += 32) dfa_add_prod(acc, Lr[c], xh[c], xl[c]);
    acc.lo += lo;
    acc = dfa_warp_sum(acc);
    if (lane == 0) y[3 * d.boff + row] = scale * ((double)acc.hi + (double)acc.lo);
  }
}

// z = Lt^{-T} x, 128-row blocks from the last to the first: after block b
// is solved (z_b = W_bb^T (x_b - acc_b), W_bb the stored inverse of the
// diagonal tile, staged in shared memory and applied by all 1024 threads,
// eight partial sums per output) every owned column a < 128 b gets
// sum_{rho in b} Lt[rho][a] z_rho: each row of Lt is read once, coalesced.
constexpr int kTrsvThreads = 1024;
constexpr int kTrsvMaxCols = 24;  // np <= 24576 (N <= 8192) with 4-CTA clusters
constexpr int kTrsvW = kMixedTile * kMixedTile;
constexpr int kTrsvSmem = (2 * kTrsvW + 2 * 8 * kMixedTile) * 4;  // W_b double buffer, partials

__device__ __forceinline__ void trsv_cp16(float* smem, const float* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}

// The solve is split over a cluster of CL CTAs per chain (trsv_cluster: 2, 4
// or 8, at least 2 for np <= 12288 and 4 up to 24576): CTA `rank` owns the columns of the 128-wide
// blocks B with B % CL == rank (local column l = t + 1024 q -> block
// CL (l / 128) + rank).  For block b the owner publishes its 128 accumulated
// sums through distributed shared memory, every CTA forms z_b (the same
// arithmetic, so identical copies), and each adds block b's contributions to
// the columns it owns.  W_{b-1} is copied (cp.async) into the other half of a
// double buffer while block b is processed.  Rank 0 writes z.
constexpr int kTrsvColsCl = 6;  // owned columns per thread: np <= 6144 CL

// Cluster size of the solve: the smallest that holds np (2 up to np = 12288,
// 4 up to 24576), doubled up to 8 while the solve's CTAs (one per SM, every
// chain a cluster) would fill at most three quarters of the SMs -- a small
// batch of long chains then streams its factor through more SMs; the rest
// stay free for the product L~ xi that runs beside it.
static int g_trsv_sms = 0;

static int trsv_cluster(int n_chains, int max_np) {
  int cl = max_np <= 2 * kTrsvColsCl * kTrsvThreads ? 2 : 4;
  const long long budget = (long long)(g_trsv_sms > 0 ? g_trsv_sms : 148) * 3 / 4;
  while (cl < 8 && (long long)n_chains * 2 * cl <= budget) cl *= 2;
  return cl;
}

template <int CL>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(kTrsvThreads)
    k_trsv_t_f32c(const float* __restrict__ M, const float* __restrict__ Winv, const ChainDesc* __restrict__ cd,
                  const double* __restrict__ x_in, const StepArgs* __restrict__ args, double* __restrict__ z) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  extern __shared__ __align__(16) float tv_smem[];
  float* Wbuf = tv_smem;                     // [2][128][128] W_bb, double buffered
  float* ph = Wbuf + 2 * kTrsvW;             // [8][128] partial hi
  float* pl = ph + 8 * kMixedTile;           // [8][128] partial lo
  __shared__ float pub_h[2][128], pub_l[2][128];  // published sums of an owned block (by parity)
  __shared__ float zh[128], zl[128], sh[128], sl[128];
  const ChainDesc d = cd[blockIdx.x / CL];
  const int T = d.np / kMixedTile;
  const double* x = args ? args->noise + (long long)args->step * args->stride : x_in;
  x += 3 * d.boff;
  const float* base = M + d.moff;
  const long long np = d.np;
  const int t = threadIdx.x;
  DFa acc[kTrsvColsCl];
#pragma unroll
  for (int q = 0; q < kTrsvColsCl; ++q) acc[q] = DFa{0.f, 0.f};
  auto col_of = [&](int q) {  // global column of owned slot q (may be >= np)
    const int l = t + kTrsvThreads * q;
    return kMixedTile * (CL * (l >> 7) + rank) + (l & 127);
  };
  auto stage_w = [&](int b, float* dst) {  // W_bb -> dst, 16 KB per quarter, one group
    const float* Wg = Winv + ((long long)d.wrow + kMixedTile * b) * kMixedTile;
#pragma unroll
    for (int q = 0; q < 4; ++q) trsv_cp16(dst + 4 * (t + kTrsvThreads * q), Wg + 4 * (t + kTrsvThreads * q));
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  stage_w(T - 1, Wbuf);
  int par = 0;
  for (int b = T - 1; b >= 0; --b, par ^= 1) {
    const int c0 = 128 * b;
    float* Ws = Wbuf + par * kTrsvW;
    if (b > 0) stage_w(b - 1, Wbuf + (par ^ 1) * kTrsvW);
    if ((b % CL) == rank) {  // publish the sums of block b's columns
#pragma unroll
      for (int q = 0; q < kTrsvColsCl; ++q) {
        const int a = col_of(q);
        if (a >= c0 && a < c0 + 128) {
          pub_h[par][a - c0] = acc[q].hi;
          pub_l[par][a - c0] = acc[q].lo;
        }
      }
    }
    cl.sync();
    if (t < 128) {
      const int owner = b % CL;
      const float* qh = owner == rank ? pub_h[par] : cl.map_shared_rank(&pub_h[par][0], owner);
      const float* ql = owner == rank ? pub_l[par] : cl.map_shared_rank(&pub_l[par][0], owner);
      const int a = c0 + t;
      const double rhs = ((a < d.n) ? x[a] : 0.0) - ((double)qh[t] + (double)ql[t]);
      sh[t] = (float)rhs;
      sl[t] = (float)(rhs - (double)sh[t]);
    }
    if (b > 0)  // W_bb landed; W_{b-1} may still be in flight
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    else
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    {  // z_i = sum_{j >= i} W[j][i] s_j: output i = t % 128, rows j in [16 p, 16 p + 16)
      const int i = t & 127, p = t >> 7;
      DFa zi{0.f, 0.f};
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        const int j = 16 * p + jj;
        if (j >= i) dfa_add_prod(zi, Ws[j * kMixedTile + i], sh[j], sl[j]);
      }
      ph[p * kMixedTile + i] = zi.hi;
      pl[p * kMixedTile + i] = zi.lo;
    }
    __syncthreads();
    if (t < 128) {
      DFa zi{ph[t], pl[t]};
#pragma unroll
      for (int p = 1; p < 8; ++p) dfa_add(zi, ph[p * kMixedTile + t], pl[p * kMixedTile + t]);
      const double v = (double)zi.hi + (double)zi.lo;
      zh[t] = (float)v;
      zl[t] = (float)(v - (double)zh[t]);
      if (rank == 0 && c0 + t < d.n) z[3 * d.boff + c0 + t] = v;
    }
    __syncthreads();
    if (b > 0) {  // contributions of block b to the owned columns a < c0
#pragma unroll
      for (int q = 0; q < kTrsvColsCl; ++q) {
        const int a = col_of(q);
        if (a < c0) {
          // next 16 rows loaded while the current 16 are summed, into two
          // independent accumulators (even and odd rows)
          const float* col = base + (long long)c0 * np + a;
          DFa s0 = acc[q], s1{0.f, 0.f};
          float v[16], vn[16];
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) v[jj] = __ldg(col + (long long)jj * np);
#pragma unroll 1
          for (int r0 = 0; r0 < 128; r0 += 16) {
            if (r0 + 16 < 128) {
#pragma unroll
              for (int jj = 0; jj < 16; ++jj) vn[jj] = __ldg(col + (long long)(r0 + 16 + jj) * np);
            }
#pragma unroll
            for (int jj = 0; jj < 16; jj += 2) {
              dfa_add_prod(s0, v[jj], zh[r0 + jj], zl[r0 + jj]);
              dfa_add_prod(s1, v[jj + 1], zh[r0 + jj + 1], zl[r0 + jj + 1]);
            }
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) v[jj] = vn[jj];
          }
          dfa_add(s0, s1.hi, s1.lo);
          acc[q] = s0;
        }
      }
    }
    __syncthreads();
  }
  cl.sync();  // no CTA leaves while a partner may still read its shared memory
}

// y = scale / 2 (y1 + w)   (scale already applied to y1 when y1 was formed
// with `scale`; here both y1 and w are unscaled).
__global__ void k_refine_combine(const ChainDesc* __restrict__ cd, const double* __restrict__ y1,
                                 const double* __restrict__ w, double half_scale,
                                 double* __restrict__ y) {
  const ChainDesc d = cd[blockIdx.y];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.n) return;
  const long long o = 3 * d.boff + e;
  y[o] = half_scale * (y1[o] + w[o]);
}

cudaError_t launch_brownian_f32_begin(const float* M, const float* Winv, const ChainDesc* cd, int n_chains,
                                      int max_np, const double* x, const StepArgs* args, double scale,
                                      bool refine, double* y, double* y1, double* z, double* scratch,
                                      cudaStream_t s, cudaStream_t s2, cudaEvent_t* ev, bool need_z) {
  k_split<<<dim3(ceil_div(max_np, 256), n_chains), 256, 0, s>>>(cd, x, args, scratch);
  if (!refine && !need_z) {
    k_trmv_f32<<<dim3(ceil_div(max_np, 32), n_chains), 256, 0, s>>>(M, cd, scratch, scale, y);
    return cudaGetLastError();
  }
  if (max_np > kTrsvThreads * kTrsvMaxCols) return cudaErrorInvalidValue;
  cudaError_t e = cudaEventRecord(ev[0], s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s2, ev[0], 0);
  if (e != cudaSuccess) return e;
  switch (trsv_cluster(n_chains, max_np)) {
    case 2: k_trsv_t_f32c<2><<<2 * n_chains, kTrsvThreads, kTrsvSmem, s2>>>(M, Winv, cd, x, args, z); break;
    case 4: k_trsv_t_f32c<4><<<4 * n_chains, kTrsvThreads, kTrsvSmem, s2>>>(M, Winv, cd, x, args, z); break;
    default: k_trsv_t_f32c<8><<<8 * n_chains, kTrsvThreads, kTrsvSmem, s2>>>(M, Winv, cd, x, args, z); break;
  }
  if (refine)
    k_trmv_f32<<<dim3(ceil_div(max_np, 32), n_chains), 256, 0, s>>>(M, cd, scratch, 1.0, y1);
  else
    k_trmv_f32<<<dim3(ceil_div(max_np, 32), n_chains), 256, 0, s>>>(M, cd, scratch, scale, y);
  e = cudaEventRecord(ev[1], s2);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_brownian_f32_end(const float* M, const ChainDesc* cd, int n_chains, int max_np, double scale,
                                    bool refine, double* y, const double* y1, const double* z, double* w,
                                    double* scratch, float2* fsplit, cudaStream_t s, cudaEvent_t* ev,
                                    bool need_z) {
  if (!refine && !need_z) return cudaSuccess;
  cudaError_t e = cudaStreamWaitEvent(s, ev[1], 0);
  if (e != cudaSuccess || !refine) return e;
  e = launch_symv_f32(M, cd, n_chains, max_np, z, fsplit, scratch, w, nullptr, s);
  if (e != cudaSuccess) return e;
  k_refine_combine<<<dim3(ceil_div(max_np, 256), n_chains), 256, 0, s>>>(cd, y1, w, 0.5 * scale, y);
  return cudaGetLastError();
}

cudaError_t launch_brownian_f32(const float* M, const float* Winv, const ChainDesc* cd, int n_chains,
                                int max_np, const double* x, const StepArgs* args, double scale,
                                bool refine, double* y, double* y1, double* z, double* w,
                                double* scratch, float2* fsplit, cudaStream_t s, cudaStream_t s2,
                                cudaEvent_t* ev, bool need_z) {
  cudaError_t e = launch_brownian_f32_begin(M, Winv, cd, n_chains, max_np, x, args, scale, refine, y, y1, z,
                                            scratch, s, s2, ev, need_z);
  if (e != cudaSuccess) return e;
  return launch_brownian_f32_end(M, cd, n_chains, max_np, scale, refine, y, y1, z, w, scratch, fsplit, s, ev,
                                 need_z);
}

cudaError_t refine_configure() {
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&g_trsv_sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaFuncSetAttribute(k_trsv_t_f32c<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrsvSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_trsv_t_f32c<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrsvSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_trsv_t_f32c<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrsvSmem);
  return e;
}

}  // namespace bd
