// k_midpoint.cu -- the midpoint corrector of the rigid-rod step.
//
// Projecting one Euler step (mobility D and rod directions u of the start of
// the step) back onto the rod constraints misses part of the mean drift that
// rigid-rod diffusion with HI needs on the constraint surface: with h* > 0
// the chain then samples shifted statics.  The corrected step keeps one
// Cholesky factor D = L L^T of the start of the step and evaluates the
// mobility and the rod directions at a midpoint:
//   y   = s L xi,  z = L^{-T} xi  (so that D z = L xi),  s = sqrt(2 dt);
//   r_m = r + P y / 2,  P y = y - A^T (A A^T)^{-1} A y  (orthogonal projection
//         onto the tangent space of |Q_k| = 1; row k of A is -u_k at bead k
//         and +u_k at bead k+1, so A A^T is tridiagonal: 2 on the diagonal,
//         -u_k . u_k+1 beside it);
//   r*  = r + dt kappa.r + s D(r_m) z, then the tensions act along the rod
//         directions of r_m through D(r_m).
// The correlation of r_m with z supplies the missing drift.
//
//   k_tangent_midpoint : per chain, the tridiagonal solve by cyclic reduction
//                        in shared memory (FP64), r_m and the unit rod
//                        directions of r_m;
//   k_trsv_t_f64       : z = s L^{-T} xi for the FP64 factor, one CTA per
//                        chain, with the 32 x 32 diagonal-block inverses;
//   k_mob_delta_f32    : mixed path, y += s (D(r_m) - D(r)) z evaluated from
//                        the positions in FP32 (no matrix): the refined
//                        displacement y of the factor at r then becomes the
//                        displacement s D(r_m) z of the corrected step up to
//                        the refinement's second-order error.
#include "bd_internal.h"
#include "rpy_dev.h"

namespace bd {

constexpr int kMidThreads = 1024;
constexpr int kMidMaxP = 4096;     // cyclic reduction: rods padded to a power of two <= 4096
constexpr int kMidMaxRods = 8192;  // serial elimination beyond that (N <= 8192)
constexpr int kMidSmem = (4 * kMidMaxP > 3 * kMidMaxRods ? 4 * kMidMaxP : 3 * kMidMaxRods) * (int)sizeof(double);

__device__ __forceinline__ void rod_dir(const double* rc, int k, double u[3]) {
  const double q0 = rc[3 * k + 3] - rc[3 * k], q1 = rc[3 * k + 4] - rc[3 * k + 1],
               q2 = rc[3 * k + 5] - rc[3 * k + 2];
  const double inv = 1.0 / sqrt(q0 * q0 + q1 * q1 + q2 * q2);
  u[0] = q0 * inv;
  u[1] = q1 * inv;
  u[2] = q2 * inv;
}

// One CTA per chain.  (A A^T) x = A y by cyclic reduction over P = 2^L >= m
// equations (the padding rows are x = 0): the forward levels eliminate the
// odd-indexed neighbours in place (A A^T is symmetric positive definite, so
// the elimination needs no pivoting), the backward levels recover x.  Chains
// of more than 4096 rods, whose four work arrays would not fit in shared
// memory, take the serial elimination (Thomas) by one thread instead.  Then
// r_m = r + (y - A^T x) / 2 and u_m.  Chains with a nonzero status keep
// r_m = r.  y is yscale times `y_in`, or times the step's noise when args is
// not NULL.
__global__ void __launch_bounds__(kMidThreads) k_tangent_midpoint(const double* __restrict__ r,
                                                                  const double* __restrict__ y_in,
                                                                  const StepArgs* __restrict__ args,
                                                                  double yscale,
                                                                  const ChainDesc* __restrict__ cd,
                                                                  const int* __restrict__ status,
                                                                  double* __restrict__ rmid,
                                                                  double* __restrict__ umid) {
  extern __shared__ __align__(16) double tm_smem[];
  const int c = blockIdx.x;
  const ChainDesc d = cd[c];
  const int N = d.N, m = d.m, t = threadIdx.x;
  const double* rc = r + 3 * d.boff;
  const double* yc = (args ? args->noise + (long long)args->step * args->stride : y_in) + 3 * d.boff;
  double* rm = rmid + 3 * d.boff;
  if (status[c] != BD_OK) {
    for (int e = t; e < 3 * N; e += kMidThreads) rm[e] = rc[e];
    __syncthreads();
  } else {
    int P = 1;
    while (P < m) P <<= 1;
    if (P > kMidMaxP) {
      // c_i (super-diagonal, also the next row's sub-diagonal), c'_i, then
      // d_i -> d'_i -> x_i
      double* c0 = tm_smem;
      double* cp = tm_smem + kMidMaxRods;
      double* dd = tm_smem + 2 * kMidMaxRods;
      for (int i = t; i < m; i += kMidThreads) {
        double ui[3];
        rod_dir(rc, i, ui);
        double cu = 0.0;
        if (i + 1 < m) {
          double un[3];
          rod_dir(rc, i + 1, un);
          cu = -(ui[0] * un[0] + ui[1] * un[1] + ui[2] * un[2]);
        }
        c0[i] = cu;
        dd[i] = yscale * (ui[0] * (yc[3 * i + 3] - yc[3 * i]) + ui[1] * (yc[3 * i + 4] - yc[3 * i + 1]) +
                          ui[2] * (yc[3 * i + 5] - yc[3 * i + 2]));
      }
      __syncthreads();
      if (t == 0) {
        double cprev = c0[0] / 2.0;
        cp[0] = cprev;
        dd[0] = dd[0] / 2.0;
        for (int i = 1; i < m; ++i) {
          const double a = c0[i - 1];  // H_{i,i-1} = H_{i-1,i}
          const double den = 2.0 - a * cprev;
          cprev = c0[i] / den;
          cp[i] = cprev;
          dd[i] = (dd[i] - a * dd[i - 1]) / den;
        }
        for (int i = m - 2; i >= 0; --i) dd[i] -= cp[i] * dd[i + 1];
      }
      __syncthreads();
      for (int i = t; i < N; i += kMidThreads) {
        double p[3] = {yscale * yc[3 * i], yscale * yc[3 * i + 1], yscale * yc[3 * i + 2]};
        if (i < m) {
          double ui[3];
          rod_dir(rc, i, ui);
#pragma unroll
          for (int q = 0; q < 3; ++q) p[q] += dd[i] * ui[q];
        }
        if (i > 0) {
          double up[3];
          rod_dir(rc, i - 1, up);
#pragma unroll
          for (int q = 0; q < 3; ++q) p[q] -= dd[i - 1] * up[q];
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) rm[3 * i + q] = rc[3 * i + q] + 0.5 * p[q];
      }
      __syncthreads();
    } else {
    double* ca = tm_smem;           // sub-diagonal coefficient
    double* cb = tm_smem + P;       // diagonal
    double* cc = tm_smem + 2 * P;   // super-diagonal
    double* cd_ = tm_smem + 3 * P;  // right-hand side, then the solution
    for (int i = t; i < P; i += kMidThreads) {
      if (i < m) {
        double ui[3];
        rod_dir(rc, i, ui);
        double a = 0.0, cu = 0.0;
        if (i > 0) {
          double up[3];
          rod_dir(rc, i - 1, up);
          a = -(up[0] * ui[0] + up[1] * ui[1] + up[2] * ui[2]);
        }
        if (i + 1 < m) {
          double un[3];
          rod_dir(rc, i + 1, un);
          cu = -(ui[0] * un[0] + ui[1] * un[1] + ui[2] * un[2]);
        }
        ca[i] = a;
        cb[i] = 2.0;
        cc[i] = cu;
        cd_[i] = yscale * (ui[0] * (yc[3 * i + 3] - yc[3 * i]) + ui[1] * (yc[3 * i + 4] - yc[3 * i + 1]) +
                           ui[2] * (yc[3 * i + 5] - yc[3 * i + 2]));
      } else {
        ca[i] = 0.0;
        cb[i] = 1.0;
        cc[i] = 0.0;
        cd_[i] = 0.0;
      }
    }
    __syncthreads();
    // forward: equation i = 2s-1 (mod 2s) absorbs its neighbours i -+ s
    for (int s = 1; s < P; s <<= 1) {
      for (int i = 2 * s - 1 + 2 * s * t; i < P; i += 2 * s * kMidThreads) {
        const int l = i - s, rr = i + s;
        const double k1 = ca[i] / cb[l];
        double nb = cb[i] - cc[l] * k1, nd = cd_[i] - cd_[l] * k1, nc = 0.0;
        if (rr < P) {
          const double k2 = cc[i] / cb[rr];
          nb -= ca[rr] * k2;
          nd -= cd_[rr] * k2;
          nc = -cc[rr] * k2;
        }
        ca[i] = -ca[l] * k1;
        cb[i] = nb;
        cc[i] = nc;
        cd_[i] = nd;
      }
      __syncthreads();
    }
    if (t == 0) cd_[P - 1] = cd_[P - 1] / cb[P - 1];
    __syncthreads();
    // backward: equation i = s-1 (mod 2s) from the solved i -+ s
    for (int s = P >> 1; s >= 1; s >>= 1) {
      for (int i = s - 1 + 2 * s * t; i < P; i += 2 * s * kMidThreads) {
        double v = cd_[i];
        if (i - s >= 0) v -= ca[i] * cd_[i - s];
        if (i + s < P) v -= cc[i] * cd_[i + s];
        cd_[i] = v / cb[i];
      }
      __syncthreads();
    }
    // r_m = r + (y - A^T x) / 2: (A^T x)_i = x_{i-1} u_{i-1} - x_i u_i
    for (int i = t; i < N; i += kMidThreads) {
      double p[3] = {yscale * yc[3 * i], yscale * yc[3 * i + 1], yscale * yc[3 * i + 2]};
      if (i < m) {
        double ui[3];
        rod_dir(rc, i, ui);
        const double x = cd_[i];
#pragma unroll
        for (int q = 0; q < 3; ++q) p[q] += x * ui[q];
      }
      if (i > 0) {
        double up[3];
        rod_dir(rc, i - 1, up);
        const double x = cd_[i - 1];
#pragma unroll
        for (int q = 0; q < 3; ++q) p[q] -= x * up[q];
      }
#pragma unroll
      for (int q = 0; q < 3; ++q) rm[3 * i + q] = rc[3 * i + q] + 0.5 * p[q];
    }
    __syncthreads();
    }
  }
  for (int k = t; k < m; k += kMidThreads) {
    double u[3];
    rod_dir(rm, k, u);
    double* uo = umid + 3 * (d.roff + k);
    uo[0] = u[0];
    uo[1] = u[1];
    uo[2] = u[2];
  }
}

cudaError_t launch_tangent_midpoint(const double* r, const double* y, const StepArgs* args, double yscale,
                                    const ChainDesc* cd, int n_chains, const int* status, double* rmid,
                                    double* umid, cudaStream_t s) {
  k_tangent_midpoint<<<n_chains, kMidThreads, kMidSmem, s>>>(r, y, args, yscale, cd, status, rmid, umid);
  return cudaGetLastError();
}

// z = scale L^{-T} xi, FP64 factor in the lower triangle of the chain's
// matrix, W_bb = (L_bb)^{-1} for its 32 x 32 diagonal blocks (W[i][j] at
// Winv[(swrow + 32 b + i) * 32 + j]).  One CTA per chain, backward over the
// blocks: s_b = xi_b - sum_{i beyond block b} L[i][block b] z_i (column sums
// accumulated by the threads that own the columns, rows read coalesced),
// z_b = W_bb^T s_b.
constexpr int kTsThreads = 1024;
constexpr int kTsCols = 12;  // 3N <= 12288

__global__ void __launch_bounds__(kTsThreads) k_trsv_t_f64(const double* __restrict__ M,
                                                           const double* __restrict__ Winv,
                                                           const ChainDesc* __restrict__ cd,
                                                           const double* __restrict__ x_in,
                                                           const StepArgs* __restrict__ args, double scale,
                                                           double* __restrict__ z) {
  __shared__ double sblk[32], zblk[32];
  const int c = blockIdx.x;
  const ChainDesc d = cd[c];
  const int n = d.n, t = threadIdx.x;
  const long long np = d.np;
  const double* L = M + d.moff;
  const double* Wb = Winv + d.swrow * 32;
  const double* x = (args ? args->noise + (long long)args->step * args->stride : x_in) + 3 * d.boff;
  double* zc = z + 3 * d.boff;
  double acc[kTsCols];
#pragma unroll
  for (int q = 0; q < kTsCols; ++q) acc[q] = 0.0;
  const int nb = (n + 31) / 32;
  for (int b = nb - 1; b >= 0; --b) {
    const int c0 = 32 * b;
#pragma unroll
    for (int q = 0; q < kTsCols; ++q) {
      const int a = t + kTsThreads * q;
      if (a >= c0 && a < c0 + 32) sblk[a - c0] = ((a < n) ? x[a] : 0.0) - acc[q];
    }
    __syncthreads();
    if (t < 32) {
      const double* W = Wb + (long long)c0 * 32;
      double v = 0.0;  // z_i = sum_{j >= i} W[j][i] s_j
      for (int j = t; j < 32; ++j) v += W[j * 32 + t] * sblk[j];
      zblk[t] = v;
      if (c0 + t < n) zc[c0 + t] = scale * v;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kTsCols; ++q) {
      const int a = t + kTsThreads * q;
      if (a < c0) {
        const double* col = L + (long long)c0 * np + a;
        double sacc = 0.0;
#pragma unroll 8
        for (int rr = 0; rr < 32; ++rr)
          if (c0 + rr < n) sacc += col[rr * np] * zblk[rr];
        acc[q] += sacc;
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_trsv_t_f64(const double* M, const double* Winv, const ChainDesc* cd, int n_chains,
                              int max_n, const double* x, const StepArgs* args, double scale, double* z,
                              cudaStream_t s) {
  if (max_n > kTsThreads * kTsCols) return cudaErrorInvalidValue;
  k_trsv_t_f64<<<n_chains, kTsThreads, 0, s>>>(M, Winv, cd, x, args, scale, z);
  return cudaGetLastError();
}

// y_i += scale sum_{j != i} (B(R_m,ij) - B(R_ij)) z_j, B the RPY block of
// Sec. 3 Eqs. (8)-(9), R_ij = r_i - r_j and R_m,ij the same at the midpoint.
// FP32 arithmetic from (hi, lo) splits of the positions and FP32 copies of
// the midpoint shift r_m - r; one thread per bead i, the beads j streamed
// through shared memory 128 at a time.
constexpr int kMdThreads = 128;

__global__ void __launch_bounds__(kMdThreads) k_mob_delta_f32(const double* __restrict__ r,
                                                              const double* __restrict__ rmid,
                                                              const double* __restrict__ z,
                                                              const ChainDesc* __restrict__ cd,
                                                              const int* __restrict__ status, float hstar,
                                                              float arad, double scale,
                                                              double* __restrict__ y) {
  __shared__ float ph[kMdThreads][3], pl[kMdThreads][3], pd[kMdThreads][3], pz[kMdThreads][3];
  const int c = blockIdx.y;
  const ChainDesc d = cd[c];
  if (status[c] != BD_OK) return;
  const int N = d.N, t = threadIdx.x;
  const int i = blockIdx.x * kMdThreads + t;
  if (blockIdx.x * kMdThreads >= N) return;
  const double* rc = r + 3 * d.boff;
  const double* rmc = rmid + 3 * d.boff;
  const double* zc = z + 3 * d.boff;
  const float inv_a = 1.0f / arad;
  float ih[3] = {0.f, 0.f, 0.f}, il[3] = {0.f, 0.f, 0.f}, id[3] = {0.f, 0.f, 0.f};
  if (i < N) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const double v = rc[3 * i + q];
      ih[q] = (float)v;
      il[q] = (float)(v - (double)ih[q]);
      id[q] = (float)(rmc[3 * i + q] - v);
    }
  }
  float acc[3] = {0.f, 0.f, 0.f};
  for (int j0 = 0; j0 < N; j0 += kMdThreads) {
    const int j = j0 + t;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      float h = 0.f, l = 0.f, dd = 0.f, zz = 0.f;
      if (j < N) {
        const double v = rc[3 * j + q];
        h = (float)v;
        l = (float)(v - (double)h);
        dd = (float)(rmc[3 * j + q] - v);
        zz = (float)zc[3 * j + q];
      }
      ph[t][q] = h;
      pl[t][q] = l;
      pd[t][q] = dd;
      pz[t][q] = zz;
    }
    __syncthreads();
    const int jn = min(kMdThreads, N - j0);
    if (i < N) {
      for (int jj = 0; jj < jn; ++jj) {
        if (j0 + jj == i) continue;
        float R[3], Rm[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          R[q] = (ih[q] - ph[jj][q]) + (il[q] - pl[jj][q]);
          Rm[q] = R[q] + (id[q] - pd[jj][q]);
        }
        float c0, r0, c1, r1;
        rpy_coeffs_rsqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2], hstar, arad, inv_a, c0, r0);
        rpy_coeffs_rsqrt(Rm[0] * Rm[0] + Rm[1] * Rm[1] + Rm[2] * Rm[2], hstar, arad, inv_a, c1, r1);
        const float z0 = pz[jj][0], z1 = pz[jj][1], z2 = pz[jj][2];
        const float dR = r0 * (R[0] * z0 + R[1] * z1 + R[2] * z2);
        const float dRm = r1 * (Rm[0] * z0 + Rm[1] * z1 + Rm[2] * z2);
        const float dc = c1 - c0;
        acc[0] += dc * z0 + (dRm * Rm[0] - dR * R[0]);
        acc[1] += dc * z1 + (dRm * Rm[1] - dR * R[1]);
        acc[2] += dc * z2 + (dRm * Rm[2] - dR * R[2]);
      }
    }
    __syncthreads();
  }
  if (i < N) {
    double* yc = y + 3 * d.boff;
#pragma unroll
    for (int q = 0; q < 3; ++q) yc[3 * i + q] += scale * (double)acc[q];
  }
}

cudaError_t launch_mob_delta_f32(const double* r, const double* rmid, const double* z, const ChainDesc* cd,
                                 int n_chains, int max_N, const int* status, double hstar, double a,
                                 double scale, double* y, cudaStream_t s) {
  k_mob_delta_f32<<<dim3(ceil_div(max_N, kMdThreads), n_chains), kMdThreads, 0, s>>>(
      r, rmid, z, cd, status, (float)hstar, (float)a, scale, y);
  return cudaGetLastError();
}

cudaError_t midpoint_configure() {
  return cudaFuncSetAttribute(k_tangent_midpoint, cudaFuncAttributeMaxDynamicSharedMemorySize, kMidSmem);
}

}  // namespace bd
