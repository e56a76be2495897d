// k_small.cu -- the whole FP64 rigid-rod step of short chains (N <= 32) in
// one CTA per chain, every matrix in shared memory, looping over all the
// steps of a bd_step call inside one launch.
//
// A chain of 32 beads has a 96 x 96 D: the multi-kernel step would spend
// almost all its time launching some hundred kernels per step, each with a
// few thousand FLOPs.  Here one CTA per chain runs the same FP64 step as the
// multi-kernel path, stage by stage:
//   D from the positions (Sec. 3 Eqs. (7)-(9)), its Cholesky factor
//   (Eq. (10)), y = s L xi (s = sqrt(2 dt));
//   midpoint step: z = s L^{-T} xi, r_m = r + P y / 2 (P the projection on
//   the tangent space of the constraints at r, a tridiagonal solve), D(r_m),
//   y = D(r_m) z and the rod directions of r_m; Euler step: D and the rod
//   directions of r;
//   the predictor r* = r + dt kappa.r + y, the self-only tensions
//   T0 = (|Q*| - 1) / (2 dt) (the K* -> infinity limit of Eq. (17));
//   the tension iteration with K = U^T C^T D C U, inverted once per step:
//   r(T) = r* + dt D F(T), g = |Q(T)|^2 - 1, T <- T + K^{-1} g / (2 dt) until
//   max|g| <= tol, then one more update (the oracle's stopping rule), capped
//   at max_newton updates;
//   the commit r <- r(T).
// A chain whose D or K is not positive definite, or whose iteration does not
// converge, records the error in its status word and keeps its positions for
// the remaining steps of the call, like the multi-kernel path.
//
// FP64 issues at two operations per clock per SM on this part, so the kernel
// avoids long dependent FP64 chains and barriers where it can: the Cholesky
// keeps its columns unscaled (L D L^T form, one barrier per column, the next
// pivot's reciprocal formed by the thread that updates it last), rows of the
// matrix-vector products are split over four threads, the tension solve is a
// product with K^{-1}, and matrices have odd row pitches (conflict-free
// column walks).
#include <math.h>

#include "bd_internal.h"
#include "rpy_dev.h"

namespace bd {

constexpr int kSmallThreads = 256;

namespace {

// Row pitch (doubles) of an order-n matrix: odd, so that a column walk by
// consecutive threads hits distinct banks.
__host__ __device__ __forceinline__ int small_pitch(int n) { return n | 1; }

}  // namespace

size_t small_smem_bytes(int max_N) {
  const size_t n = 3 * (size_t)max_N, m = max_N > 1 ? max_N - 1 : 1;
  const size_t pn = (size_t)small_pitch((int)n), pm = (size_t)small_pitch((int)m);
  return (2 * n * pn + 2 * m * pm + 8 * n + 13 * m + 40) * sizeof(double);
}

namespace {

__device__ __forceinline__ double sm_reduce_max(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double r = red[0];
#pragma unroll
  for (int w = 1; w < kSmallThreads / 32; ++w) r = fmax(r, red[w]);
  __syncthreads();
  return r;
}

// Lower-triangular pair (i, k), k <= i, of row-major index e.
__device__ __forceinline__ void tri_pair(int e, int& i, int& k) {
  i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while (i * (i + 1) / 2 > e) --i;
  while ((i + 1) * (i + 2) / 2 <= e) ++i;
  k = e - i * (i + 1) / 2;
}

// D (full, both triangles, row pitch p) of the N beads at r.
__device__ void assemble_small(const double* r, int N, double hstar, double a, double* D, int p) {
  const double inv_a = 1.0 / a;
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int i = e / N, j = e % N;
    double R[3] = {0.0, 0.0, 0.0}, cI = 1.0, cRR = 0.0;
    if (i != j) {
#pragma unroll
      for (int q = 0; q < 3; ++q) R[q] = r[3 * i + q] - r[3 * j + q];
      rpy_coeffs_inv<double>(R[0] * R[0] + R[1] * R[1] + R[2] * R[2], hstar, a, inv_a, cI, cRR);
    }
#pragma unroll
    for (int x = 0; x < 3; ++x)
#pragma unroll
      for (int y = 0; y < 3; ++y) D[(3 * i + x) * p + 3 * j + y] = (x == y ? cI : 0.0) + cRR * R[x] * R[y];
  }
}

// out_i = base_i + scale (A x)_i (base may be NULL) for the n rows of the
// full matrix A (pitch p, columns k < klim(i) = lower ? i + 1 : n), four
// threads per row.  Synchronises the block on exit.
__device__ void matvec_small(const double* A, int p, int n, bool lower, const double* x, double* out,
                             const double* base, double scale) {
  const int rows4 = (n + 7) / 8 * 8 * 4;  // whole warps of row quartets
  for (int e = threadIdx.x; e < rows4; e += blockDim.x) {
    const int i = e >> 2, part = e & 3;
    double acc = 0.0;
    if (i < n) {
      const int kl = lower ? i + 1 : n;
      for (int k = part; k < kl; k += 4) acc += A[i * p + k] * x[k];
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    if (i < n && part == 0) out[i] = base ? base[i] + scale * acc : scale * acc;
  }
  __syncthreads();
}

// In-place Cholesky factor of the order-n matrix at A (pitch p; the lower
// triangle is read and written), right-looking with unscaled columns: step j
// subtracts A_ij A_kj / d_j from the trailing lower triangle, d_j the pivot;
// the thread that makes the last update to A_{j+1,j+1} forms its reciprocal,
// so one barrier per column suffices.  Then rd[j] = 1 / sqrt(d_j) = 1 / L_jj
// and L_ij = A_ij rd[j].  *flag (zero on entry) is set when a pivot is not
// positive; returns false then, in every thread.
__device__ bool chol_small(double* A, int p, int n, double* rd, int* flag) {
  const int t = threadIdx.x;
  if (t == 0) {
    const double d0 = A[0];
    if (!(d0 > 0.0)) *flag = 1;
    else rd[0] = 1.0 / d0;
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (*flag) return false;
    const double rj = rd[j];  // 1 / d_j
    const int w = n - j - 1;
    for (int e = t; e < w * (w + 1) / 2; e += blockDim.x) {
      int ii, kk;
      tri_pair(e, ii, kk);
      const int i = j + 1 + ii, k = j + 1 + kk;
      const double v = A[i * p + k] - A[i * p + j] * A[k * p + j] * rj;
      A[i * p + k] = v;
      if (e == 0) {  // (j+1, j+1): the next pivot, now final
        if (!(v > 0.0)) *flag = 1;
        else rd[j + 1] = 1.0 / v;
      }
    }
    __syncthreads();
  }
  if (*flag) return false;
  for (int j = t; j < n; j += blockDim.x) rd[j] = sqrt(rd[j]);  // 1 / sqrt(d_j) = 1 / L_jj
  __syncthreads();
  for (int e = t; e < n * (n + 1) / 2; e += blockDim.x) {
    int i, j;
    tri_pair(e, i, j);
    A[i * p + j] = (i == j) ? 1.0 / rd[j] : A[i * p + j] * rd[j];
  }
  __syncthreads();
  return true;
}

// x = s L^{-T} b: L lower (pitch p), rd = 1 / diag(L), x and b distinct.
// One warp, column form from the last row: x_j is final, then every x_i,
// i < j, loses L_ji x_j (row j of L, contiguous).
__device__ void trsv_t_warp(const double* L, int p, const double* rd, int n, const double* b, double s,
                            double* x) {
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < n; i += 32) x[i] = s * b[i];
  __syncwarp();
  for (int j = n - 1; j >= 0; --j) {
    const double xj = x[j] * rd[j];
    __syncwarp();
    if (lane == 0) x[j] = xj;
    for (int i = lane; i < j; i += 32) x[i] -= L[j * p + i] * xj;
    __syncwarp();
  }
}

// W = L^{-1} (lower, pitch p) of the lower factor L (rd = 1 / diag(L)), one
// thread per column (forward substitution down the column), then
// Kinv = W^T W (full, pitch p) into the storage of L.
__device__ void inverse_from_factor(double* L, double* W, int p, int m, const double* rd) {
  const int t = threadIdx.x;
  for (int col = t; col < m; col += blockDim.x) {
    W[col * p + col] = rd[col];
    for (int i = col + 1; i < m; ++i) {
      double acc = 0.0;
      for (int k = col; k < i; ++k) acc += L[i * p + k] * W[k * p + col];
      W[i * p + col] = -acc * rd[i];
    }
  }
  __syncthreads();
  for (int e = t; e < m * m; e += blockDim.x) {
    const int k = e / m, l = e % m;
    const int lo = k > l ? k : l;
    double acc = 0.0;
    for (int i = lo; i < m; ++i) acc += W[i * p + k] * W[i * p + l];
    L[k * p + l] = acc;
  }
  __syncthreads();
}

__device__ __forceinline__ void rod_unit(const double* r, int k, double u[3]) {
  const double q0 = r[3 * k + 3] - r[3 * k], q1 = r[3 * k + 4] - r[3 * k + 1], q2 = r[3 * k + 5] - r[3 * k + 2];
  const double inv = 1.0 / sqrt(q0 * q0 + q1 * q1 + q2 * q2);
  u[0] = q0 * inv;
  u[1] = q1 * inv;
  u[2] = q2 * inv;
}

// F_i = T_i u_i - T_{i-1} u_{i-1} for the N beads.
__device__ void forces_small(const double* T, const double* u, int N, double* F) {
  const int m = N - 1;
  for (int i = threadIdx.x; i < N; i += blockDim.x)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      double f = 0.0;
      if (i < m) f += T[i] * u[3 * i + q];
      if (i > 0) f -= T[i - 1] * u[3 * (i - 1) + q];
      F[3 * i + q] = f;
    }
}

}  // namespace

__global__ void __launch_bounds__(kSmallThreads) k_step_small(double* __restrict__ rg, double* __restrict__ Tg,
                                                              int* __restrict__ status, int* __restrict__ iters,
                                                              int* __restrict__ state,
                                                              const ChainDesc* __restrict__ cd, Phys ph,
                                                              const double* __restrict__ noise, long long stride,
                                                              int n_steps, int midpoint) {
  extern __shared__ __align__(16) double sm_small[];
  const int c = blockIdx.x;
  const ChainDesc d = cd[c];
  const int N = d.N, n = d.n, m = d.m;
  const int mm = m > 0 ? m : 1;
  const int pn = small_pitch(n), pm = small_pitch(mm);
  double* sD = sm_small;              // [n][pn] D, then D(r_m) (midpoint)
  double* sL = sD + n * pn;           // [n][pn] the factor of D (lower)
  double* sK = sL + n * pn;           // [m][pm] K, its factor (lower), then K^{-1} (full)
  double* sW = sK + mm * pm;          // [m][pm] the inverse of K's factor
  double* sr = sW + mm * pm;          // positions
  double* srs = sr + n;               // r*
  double* srT = srs + n;              // r(T); r_m before the predictor
  double* sy = srT + n;               // displacement
  double* sz = sy + n;                // z = s L^{-T} xi
  double* sF = sz + n;                // bead forces
  double* srd = sF + n;               // 1 / diag of the factor of D
  double* sxi = srd + n;              // the step's noise
  double* su = sxi + n;               // [m][3] rod directions the tensions act along
  double* su0 = su + 3 * mm;          // [m][3] rod directions of r (midpoint projection)
  double* sT = su0 + 3 * mm;          // [2][m] tensions, double-buffered over the iteration
  double* srhs = sT + 2 * mm;         // g / (2 dt)
  double* srk = srhs + mm;            // 1 / diag of the factor of K
  double* sc = srk + mm;              // tridiagonal: c_i
  double* scp = sc + mm;              // tridiagonal: c'_i
  double* sx = scp + mm;              // tridiagonal: d_i, then the solution x_i
  double* red = sx + mm;              // [32]
  int* flag = reinterpret_cast<int*>(red + 32);
  const int t = threadIdx.x;
  const double s = ph.sq2dt, dt = ph.dt;

  for (int e = t; e < n; e += blockDim.x) sr[e] = rg[3 * d.boff + e];
  int st = status[c];
  int it = 0, tb = 0;   // tb: the half of sT holding the current tensions
  bool have_T = false;  // sT holds this call's tensions (written back at the end)
  for (int step = 0; step < n_steps && st == BD_OK; ++step) {
    const double* xi = noise + (long long)step * stride + 3 * d.boff;
    for (int e = t; e < n; e += blockDim.x) sxi[e] = xi[e];
    if (t == 0) *flag = 0;
    // ---- D and its factor
    assemble_small(sr, N, ph.hstar, ph.a, sD, pn);
    __syncthreads();
    for (int e = t; e < n * (n + 1) / 2; e += blockDim.x) {
      int i, k;
      tri_pair(e, i, k);
      sL[i * pn + k] = sD[i * pn + k];
    }
    __syncthreads();
    if (!chol_small(sL, pn, n, srd, flag)) {
      st = BD_ERR_NOT_PD;
      break;
    }
    // ---- y = s L xi
    matvec_small(sL, pn, n, true, sxi, sy, nullptr, s);
    const double* rdir = sr;
    if (midpoint) {
      // rod directions of r; z = s L^{-T} xi by warp 0 beside them
      for (int k = t; k < m; k += blockDim.x) rod_unit(sr, k, su0 + 3 * k);
      if (t < 32) trsv_t_warp(sL, pn, srd, n, sxi, s, sz);
      __syncthreads();
      // r_m = r + (y - A^T x) / 2 with (A A^T) x = A y: A A^T tridiagonal,
      // 2 on the diagonal and c_i = -u_i . u_{i+1} beside it (u of r),
      // d_i = u_i . (y_{i+1} - y_i).  Thomas: c'_0 = c_0 / 2, x_0 = d_0 / 2;
      // den = 2 - c_{i-1} c'_{i-1}, c'_i = c_i / den,
      // x_i = (d_i - c_{i-1} x_{i-1}) / den; then x_i -= c'_i x_{i+1}.
      for (int i = t; i < m; i += blockDim.x) {
        const double* ui = su0 + 3 * i;
        sc[i] = (i + 1 < m) ? -(ui[0] * ui[3] + ui[1] * ui[4] + ui[2] * ui[5]) : 0.0;
        sx[i] = ui[0] * (sy[3 * i + 3] - sy[3 * i]) + ui[1] * (sy[3 * i + 4] - sy[3 * i + 1]) +
                ui[2] * (sy[3 * i + 5] - sy[3 * i + 2]);
      }
      __syncthreads();
      if (t == 0 && m > 0) {
        double cprev = 0.5 * sc[0], xprev = 0.5 * sx[0];
        scp[0] = cprev;
        sx[0] = xprev;
        for (int i = 1; i < m; ++i) {
          const double a = sc[i - 1];
          const double rden = 1.0 / (2.0 - a * cprev);
          cprev = sc[i] * rden;
          xprev = (sx[i] - a * xprev) * rden;
          scp[i] = cprev;
          sx[i] = xprev;
        }
        for (int i = m - 2; i >= 0; --i) {
          xprev = sx[i] - scp[i] * xprev;
          sx[i] = xprev;
        }
      }
      __syncthreads();
      for (int i = t; i < N; i += blockDim.x)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          double p = sy[3 * i + q];
          if (i < m) p += sx[i] * su0[3 * i + q];
          if (i > 0) p -= sx[i - 1] * su0[3 * (i - 1) + q];
          srT[3 * i + q] = sr[3 * i + q] + 0.5 * p;
        }
      __syncthreads();
      // D(r_m) and y = D(r_m) z
      assemble_small(srT, N, ph.hstar, ph.a, sD, pn);
      __syncthreads();
      matvec_small(sD, pn, n, false, sz, sy, nullptr, 1.0);
      rdir = srT;
    }
    // ---- rod directions, K = U^T C^T D C U, its inverse
    for (int k = t; k < m; k += blockDim.x) rod_unit(rdir, k, su + 3 * k);
    __syncthreads();
    for (int e = t; e < m * (m + 1) / 2; e += blockDim.x) {
      int k, l;
      tri_pair(e, k, l);
      double v = 0.0;
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        double bu = 0.0;
#pragma unroll
        for (int y = 0; y < 3; ++y) {
          const double b = sD[(3 * k + x) * pn + 3 * l + y] - sD[(3 * k + x) * pn + 3 * (l + 1) + y] -
                           sD[(3 * (k + 1) + x) * pn + 3 * l + y] + sD[(3 * (k + 1) + x) * pn + 3 * (l + 1) + y];
          bu += b * su[3 * l + y];
        }
        v += su[3 * k + x] * bu;
      }
      sK[k * pm + l] = v;
    }
    __syncthreads();
    if (m > 0) {
      if (!chol_small(sK, pm, m, srk, flag)) {
        st = BD_ERR_CONSTRAINT;
        break;
      }
      inverse_from_factor(sK, sW, pm, m, srk);
    }
    // ---- predictor, T0, F(T0)
    for (int i = t; i < N; i += blockDim.x)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const double kr = ph.kappa[3 * q] * sr[3 * i] + ph.kappa[3 * q + 1] * sr[3 * i + 1] +
                          ph.kappa[3 * q + 2] * sr[3 * i + 2];
        srs[3 * i + q] = sr[3 * i + q] + dt * kr + sy[3 * i + q];
      }
    __syncthreads();
    tb = 0;
    for (int k = t; k < m; k += blockDim.x) {
      const double q0 = srs[3 * k + 3] - srs[3 * k], q1 = srs[3 * k + 4] - srs[3 * k + 1],
                   q2 = srs[3 * k + 5] - srs[3 * k + 2];
      sT[k] = (sqrt(q0 * q0 + q1 * q1 + q2 * q2) - 1.0) / (2.0 * dt);
    }
    have_T = true;
    __syncthreads();
    forces_small(sT, su, N, sF);
    __syncthreads();
    // ---- tension iteration (the state machine of the multi-kernel path)
    int ns = NS_ACTIVE;
    it = 0;
    for (;;) {
      matvec_small(sD, pn, n, false, sF, srT, srs, dt);  // r(T) = r* + dt D F
      double gmax = 0.0;
      for (int k = t; k < m; k += blockDim.x) {
        const double q0 = srT[3 * k + 3] - srT[3 * k], q1 = srT[3 * k + 4] - srT[3 * k + 1],
                     q2 = srT[3 * k + 5] - srT[3 * k + 2];
        const double g = q0 * q0 + q1 * q1 + q2 * q2 - 1.0;
        srhs[k] = g * (0.5 / dt);
        gmax = (g != g) ? INFINITY : fmax(gmax, fabs(g));
      }
      gmax = sm_reduce_max(gmax, red);
      if (ns == NS_EXTRA) {
        ns = NS_DONE;
        break;
      }
      if (gmax <= ph.tol) {
        ns = NS_EXTRA;
      } else if (it >= ph.max_newton || !(gmax < INFINITY)) {
        ns = NS_FAILED;
        break;
      }
      // T' = T + K^{-1} g / (2 dt) into the other half of sT, then F(T')
      double* Tc = sT + tb * mm;
      double* Tn = sT + (1 - tb) * mm;
      matvec_small(sK, pm, m, false, srhs, Tn, Tc, 1.0);
      tb = 1 - tb;
      forces_small(Tn, su, N, sF);
      __syncthreads();
      ++it;
    }
    if (ns != NS_DONE) {
      st = BD_ERR_CONSTRAINT;
      break;
    }
    // ---- commit
    for (int e = t; e < n; e += blockDim.x) sr[e] = srT[e];
    __syncthreads();
  }
  for (int e = t; e < n; e += blockDim.x) rg[3 * d.boff + e] = sr[e];
  if (have_T)
    for (int k = t; k < m; k += blockDim.x) Tg[d.roff + k] = sT[tb * mm + k];
  if (t == 0) {
    if (st != BD_OK) atomicCAS(status + c, BD_OK, st);
    iters[c] = it;
    state[c] = st == BD_OK ? NS_DONE : NS_FAILED;
  }
}

cudaError_t launch_step_small(double* r, double* T, int* status, int* iters, int* state, const ChainDesc* cd,
                              int n_chains, int max_N, Phys ph, const double* noise, long long stride,
                              int n_steps, bool midpoint, cudaStream_t s) {
  k_step_small<<<n_chains, kSmallThreads, small_smem_bytes(max_N), s>>>(r, T, status, iters, state, cd, ph, noise,
                                                                        stride, n_steps, midpoint ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t small_configure(int max_N) {
  return cudaFuncSetAttribute(k_step_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)small_smem_bytes(max_N));
}

}  // namespace bd
