// k_tangent.cu -- forward-mode derivatives (tangents) of one FP64 time step
// with respect to a parameter p (the Weissenberg number or h*), at fixed
// noise.  With r' = dr/dp carried from step to step, the step map
//   D = D(r; h*, a)            (Eqs. (7)-(9))
//   L = chol(D)                (Eq. (10))
//   y = s L xi                 (noise term of Eq. (6))
//   r* = r + dt kappa(Wi) r + y
//   g(T) = |Q(r* + dt D C(T u))|^2 - 1 = 0   (rigid rods)
//   r_new = r* + dt D C(T u)
// is differentiated exactly:
//   D'  = sum over pairs of dD_ij/dR (r'_i - r'_j) + dD/dh* h*' (dual numbers)
//   L'  = L Phi(L^{-1} D' L^{-T}),  Phi = lower triangle with half diagonal
//   y'  = s L Phi(X) xi with X = L^{-1} D' L^{-T} (symmetric)
//   r*' = r' + dt (kappa' r + kappa r') + y'
//   u'_k = (I - u_k u_k^T) Q'_k / |Q_k|
//   T' from  2 Q_k . Delta[r*' + dt D' F + dt D C(T u') + dt D C(T' u)]_k = 0,
//   solved by the same K-preconditioned iteration as the tensions,
//   r_new' = r*' + dt D' F + dt D C(T u') + dt D C(T' u).
// The midpoint step (mobility and rod directions at r_m = r + P y / 2, the
// Brownian displacement s D(r_m) z with z = L^{-T} xi) adds
//   z'   = -L^{-T} Phi(X)^T xi          (from L^T z = xi and L' = L Phi(X)),
//   (P y)' = y' - (A^T x)',  (A A^T) x = A y,
//            (A A^T) x' = (A y)' - (A A^T)' x  (A from the unit rods of r),
//   r_m' = r' + (P y)' / 2,  D_m' from r_m and r_m' (dual numbers),
//   the Brownian part s (D_m' z + D_m z'),
// and the tension part above with D_m, D_m' and the rod directions of r_m.
// The paper has no derivatives; these kernels serve bd_adjoint.
#include <math.h>

#include "bd_internal.h"

namespace bd {

// ------------------------------------------------------------ dual numbers
struct Dual {
  double v, d;
};
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
  const double q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}
__device__ __forceinline__ Dual dsqrt(Dual a) {
  const double s = sqrt(a.v);
  return {s, s > 0.0 ? a.d / (2.0 * s) : 0.0};
}
__device__ __forceinline__ Dual cst(double c) { return {c, 0.0}; }

// RPY coefficients (Eqs. (8)-(9)) with their derivative:
// D_ij = cI I + cRR R R^T; the branch is decided on the value.
__device__ __forceinline__ void rpy_dual(Dual R2, Dual h, Dual a, Dual& cI, Dual& cRR) {
  const Dual Rn = dsqrt(R2);
  if (h.v == 0.0 && h.d == 0.0) {
    cI = cst(0.0);
    cRR = cst(0.0);
  } else if (Rn.v >= 2.0 * a.v) {
    const Dual pref = cst(0.75) * h / Rn;
    const Dual a2R2 = a * a / R2;
    cI = pref * (cst(1.0) + cst(2.0 / 3.0) * a2R2);
    cRR = pref * (cst(1.0) - cst(2.0) * a2R2) / R2;
  } else {
    const Dual pref = cst(0.375) * h / a;
    cI = pref * (cst(8.0 / 3.0) - cst(0.75) * Rn / a);
    cRR = (Rn.v > 0.0) ? pref * (cst(0.25) / a) / Rn : cst(0.0);
  }
}

// D' (full symmetric n x n, row-major with pitch np) for every chain.
// One thread per ordered bead pair (i, j), writing its 3 x 3 block.
__global__ void k_assemble_dot(const double* __restrict__ r, const double* __restrict__ rdot,
                               const ChainDesc* __restrict__ cd, double* __restrict__ Md,
                               double hstar, double a, double hdot, double adot) {
  const ChainDesc d = cd[blockIdx.y];
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)d.N * d.N) return;
  const int i = (int)(idx / d.N), j = (int)(idx % d.N);
  double blk[9];
  if (i == j) {
#pragma unroll
    for (int q = 0; q < 9; ++q) blk[q] = 0.0;
  } else {
    const double* ri = r + 3 * (d.boff + i);
    const double* rj = r + 3 * (d.boff + j);
    const double* vi = rdot + 3 * (d.boff + i);
    const double* vj = rdot + 3 * (d.boff + j);
    const double R[3] = {ri[0] - rj[0], ri[1] - rj[1], ri[2] - rj[2]};
    const double dR[3] = {vi[0] - vj[0], vi[1] - vj[1], vi[2] - vj[2]};
    const Dual R2 = {R[0] * R[0] + R[1] * R[1] + R[2] * R[2],
                     2.0 * (R[0] * dR[0] + R[1] * dR[1] + R[2] * dR[2])};
    Dual cI, cRR;
    rpy_dual(R2, Dual{hstar, hdot}, Dual{a, adot}, cI, cRR);
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int l = 0; l < 3; ++l)
        blk[3 * k + l] = (k == l ? cI.d : 0.0) + cRR.d * R[k] * R[l] +
                         cRR.v * (dR[k] * R[l] + R[k] * dR[l]);
  }
  double* base = Md + d.moff;
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int l = 0; l < 3; ++l) base[(long long)(3 * i + k) * d.np + 3 * j + l] = blk[3 * k + l];
}

// ---------------------------------------------------- TRSM with many RHS
// B <- L^{-1} B for the n x n block B (pitch np) of every chain, L the lower
// factor in M (32-tiles, diagonal-tile inverses W in Winv).  Block row k:
//   scale : B_k <- W_kk B_k                      (all 32-column tiles)
//   update: B_r -= L_rk B_k for every r > k      (all 32-column tiles)
constexpr int TT = kSimtTile;

__global__ void __launch_bounds__(256) k_trsm_rhs_scale(const double* __restrict__ Winv,
                                                        const ChainDesc* __restrict__ cd, int k,
                                                        double* __restrict__ B) {
  __shared__ double W[TT][TT + 1];
  __shared__ double X[TT][TT + 1];
  const ChainDesc d = cd[blockIdx.y];
  const int nt = d.np / TT;
  if (k >= nt || (int)blockIdx.x >= nt) return;
  const double* w = Winv + (d.swrow + (long long)k * TT) * TT;
  double* b = B + d.moff + (long long)(k * TT) * d.np + blockIdx.x * TT;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int r = ty; r < TT; r += 8) {
    W[r][tx] = w[r * TT + tx];
    X[r][tx] = b[(long long)r * d.np + tx];
  }
  __syncthreads();
  for (int r = ty; r < TT; r += 8) {
    double s = 0.0;
    for (int m = 0; m <= r; ++m) s += W[r][m] * X[m][tx];
    b[(long long)r * d.np + tx] = s;
  }
}

__global__ void __launch_bounds__(256) k_trsm_rhs_update(const double* __restrict__ M,
                                                         const ChainDesc* __restrict__ cd, int k,
                                                         double* __restrict__ B) {
  __shared__ double Lr[TT][TT + 1];
  __shared__ double Bk[TT][TT + 1];
  const ChainDesc d = cd[blockIdx.z];
  const int nt = d.np / TT;
  const int rt = k + 1 + blockIdx.y, ct = blockIdx.x;
  if (rt >= nt || ct >= nt) return;
  const double* l = M + d.moff + (long long)(rt * TT) * d.np + k * TT;
  const double* bk = B + d.moff + (long long)(k * TT) * d.np + ct * TT;
  double* br = B + d.moff + (long long)(rt * TT) * d.np + ct * TT;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < TT; r += 8) {
    Lr[r][tx] = l[(long long)r * d.np + tx];
    Bk[r][tx] = bk[(long long)r * d.np + tx];
  }
  __syncthreads();
  for (int r = ty; r < TT; r += 8) {
    double s = 0.0;
#pragma unroll 8
    for (int m = 0; m < TT; ++m) s += Lr[r][m] * Bk[m][tx];
    br[(long long)r * d.np + tx] -= s;
  }
}

// B <- B^T in place (n x n block of every chain), tile pairs swapped.
__global__ void __launch_bounds__(256) k_transpose(const ChainDesc* __restrict__ cd,
                                                   double* __restrict__ B) {
  __shared__ double P[TT][TT + 1], Q[TT][TT + 1];
  const ChainDesc d = cd[blockIdx.z];
  const int nt = d.np / TT;
  const int ti = blockIdx.y, tj = blockIdx.x;
  if (ti >= nt || tj > ti) return;
  double* a = B + d.moff + (long long)(ti * TT) * d.np + tj * TT;
  double* b = B + d.moff + (long long)(tj * TT) * d.np + ti * TT;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < TT; r += 8) {
    P[r][tx] = a[(long long)r * d.np + tx];
    Q[r][tx] = b[(long long)r * d.np + tx];
  }
  __syncthreads();
  for (int r = ty; r < TT; r += 8) {
    a[(long long)r * d.np + tx] = Q[tx][r];
    if (ti != tj) b[(long long)r * d.np + tx] = P[tx][r];
  }
}

// v = Phi(X) xi: v_i = sum_{j < i} X_ij xi_j + X_ii xi_i / 2 (warp per row)
__global__ void __launch_bounds__(256) k_phi_matvec(const double* __restrict__ X,
                                                    const ChainDesc* __restrict__ cd,
                                                    const double* __restrict__ xi,
                                                    double* __restrict__ v) {
  const ChainDesc d = cd[blockIdx.y];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * 8 + warp;
  if (row >= d.n) return;
  const double* xr = X + d.moff + (long long)row * d.np;
  const double* x = xi + 3 * d.boff;
  double s = 0.0;
  for (int c = lane; c <= row; c += 32) s += (c == row ? 0.5 : 1.0) * xr[c] * x[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) v[3 * d.boff + row] = s;
}

// v = Phi(X)^T xi for symmetric X: v_i = sum_{j > i} X_ij xi_j + X_ii xi_i / 2.
__global__ void __launch_bounds__(256) k_phi_upper_matvec(const double* __restrict__ X,
                                                          const ChainDesc* __restrict__ cd,
                                                          const double* __restrict__ xi,
                                                          double* __restrict__ v) {
  const ChainDesc d = cd[blockIdx.y];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * 8 + warp;
  if (row >= d.n) return;
  const double* xr = X + d.moff + (long long)row * d.np;
  const double* x = xi + 3 * d.boff;
  double s = 0.0;
  for (int c = row + lane; c < d.n; c += 32) s += (c == row ? 0.5 : 1.0) * xr[c] * x[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) v[3 * d.boff + row] = s;
}

// w = A f for a dense n x n block (pitch np) of every chain, warp per row.
__global__ void __launch_bounds__(256) k_gemv_dense(const double* __restrict__ A,
                                                    const ChainDesc* __restrict__ cd,
                                                    const double* __restrict__ f,
                                                    double* __restrict__ w) {
  const ChainDesc d = cd[blockIdx.y];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * 8 + warp;
  if (row >= d.n) return;
  const double* ar = A + d.moff + (long long)row * d.np;
  const double* x = f + 3 * d.boff;
  double s = 0.0;
  for (int c = lane; c < d.n; c += 32) s += ar[c] * x[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) w[3 * d.boff + row] = s;
}

// r*' = r' + dt (kappa' r + kappa r') + y'  and  G = C(T u') (bead forces of
// the rod-direction change), u'_k = (I - u u^T) Q'_k / |Q_k| (old positions).
// The rod directions (and their tangents) come from rq, rqdot: the positions
// of the start of the step (Euler) or the midpoint (midpoint step).
__global__ void k_tangent_predictor(const double* __restrict__ r, const double* __restrict__ rdot,
                                    const double* __restrict__ rq_, const double* __restrict__ rqdot,
                                    const double* __restrict__ ydot, const double* __restrict__ uhat,
                                    const double* __restrict__ T, const ChainDesc* __restrict__ cd,
                                    Phys ph, const double* __restrict__ kappa_dot,
                                    double* __restrict__ rsdot, double* __restrict__ G) {
  const ChainDesc d = cd[blockIdx.y];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.N) return;
  const double* ri = r + 3 * (d.boff + i);
  const double* vi = rdot + 3 * (d.boff + i);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double s = vi[k] + ydot[3 * (d.boff + i) + k];
    for (int l = 0; l < 3; ++l) s += ph.dt * (kappa_dot[3 * k + l] * ri[l] + ph.kappa[3 * k + l] * vi[l]);
    rsdot[3 * (d.boff + i) + k] = s;
  }
  auto udot = [&](int kr, double out[3]) {
    const double* a0 = rq_ + 3 * (d.boff + kr);
    const double* v0 = rqdot + 3 * (d.boff + kr);
    const double q[3] = {a0[3] - a0[0], a0[4] - a0[1], a0[5] - a0[2]};
    const double qd[3] = {v0[3] - v0[0], v0[4] - v0[1], v0[5] - v0[2]};
    const double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
    const double* u = uhat + 3 * (d.roff + kr);
    const double uq = u[0] * qd[0] + u[1] * qd[1] + u[2] * qd[2];
    for (int k = 0; k < 3; ++k) out[k] = (qd[k] - u[k] * uq) / qn;
  };
  double g[3] = {0.0, 0.0, 0.0};
  if (i < d.m) {
    double ud[3];
    udot(i, ud);
    const double t = T[d.roff + i];
    for (int k = 0; k < 3; ++k) g[k] += t * ud[k];
  }
  if (i > 0) {
    double ud[3];
    udot(i - 1, ud);
    const double t = T[d.roff + i - 1];
    for (int k = 0; k < 3; ++k) g[k] -= t * ud[k];
  }
  for (int k = 0; k < 3; ++k) G[3 * (d.boff + i) + k] = g[k];
}

// a = r*' + dt (D' F + D G): the part of r_new' that does not depend on T'.
__global__ void k_tangent_base(const ChainDesc* __restrict__ cd, Phys ph,
                               const double* __restrict__ rsdot, const double* __restrict__ DdF,
                               const double* __restrict__ DG, double* __restrict__ a) {
  const ChainDesc d = cd[blockIdx.y];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.n) return;
  const long long o = 3 * d.boff + e;
  a[o] = rsdot[o] + ph.dt * (DdF[o] + DG[o]);
}

// One CTA per chain: z = a + dt D C(T' u) (u = D C(T' u) from the mobility
// product), R_k = 2 Q_k . (z_{k+1} - z_k) with Q the converged rods; stores
// z and rhs = R / (2 dt) for the K solve, and steps the iteration state.
__global__ void __launch_bounds__(256) k_tangent_residual(const double* __restrict__ a,
                                                          const double* __restrict__ u,
                                                          const double* __restrict__ rnew,
                                                          const ChainDesc* __restrict__ cd, Phys ph,
                                                          double rel_tol, double* __restrict__ rscale,
                                                          double* __restrict__ z,
                                                          double* __restrict__ rhs,
                                                          int* __restrict__ state,
                                                          int* __restrict__ status,
                                                          const int* __restrict__ iters) {
  __shared__ double red[32];
  const int c = blockIdx.x;
  const int st = state[c];
  if (st >= NS_DONE) return;
  const ChainDesc d = cd[c];
  const long long b3 = 3 * d.boff;
  for (int e = threadIdx.x; e < d.n; e += blockDim.x) z[b3 + e] = a[b3 + e] + ph.dt * u[b3 + e];
  __syncthreads();
  double rmax = 0.0;
  for (int k = threadIdx.x; k < d.m; k += blockDim.x) {
    const double* q = rnew + b3 + 3 * k;
    const double* zz = z + b3 + 3 * k;
    const double R = 2.0 * ((q[3] - q[0]) * (zz[3] - zz[0]) + (q[4] - q[1]) * (zz[4] - zz[1]) +
                            (q[5] - q[2]) * (zz[5] - zz[2]));
    rhs[d.roff + k] = R * (0.5 / ph.dt);
    rmax = (R != R) ? INFINITY : fmax(rmax, fabs(R));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = rmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
    // convergence relative to the residual of the first pass (T' = 0)
    if (iters[c] == 0 && st == NS_ACTIVE) rscale[c] = fmax(mx, 1e-300);
    int ns = st;
    if (st == NS_EXTRA) ns = NS_DONE;
    else if (mx <= rel_tol * rscale[c]) ns = NS_EXTRA;
    else if (iters[c] >= ph.max_newton || !(mx < INFINITY)) {
      ns = NS_FAILED;
      atomicCAS(status + c, BD_OK, BD_ERR_CONSTRAINT);
    }
    state[c] = ns;
  }
}

__global__ void k_tangent_init(const ChainDesc* __restrict__ cd, const int* __restrict__ status,
                               int* __restrict__ state, int* __restrict__ iters,
                               double* __restrict__ Tdot, double* __restrict__ Fdot) {
  const int c = blockIdx.y;
  const ChainDesc d = cd[c];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e == 0) {
    state[c] = (status[c] == BD_OK) ? NS_ACTIVE : NS_FAILED;
    iters[c] = 0;
  }
  if (e < d.m) Tdot[d.roff + e] = 0.0;
  if (e < d.n) Fdot[3 * d.boff + e] = 0.0;
}

// ------------------------------------------------- midpoint tangent
// One CTA per chain.  With u the unit rods of r, c = A y, H = A A^T
// (tridiagonal: 2, -u_k . u_k+1), x = H^{-1} c:
//   c'_k = u'_k . (y_k+1 - y_k) + u_k . (y'_k+1 - y'_k),
//   H'_k,k+1 = -(u'_k . u_k+1 + u_k . u'_k+1),  H'_kk = 0,
//   x' = H^{-1} (c' - H' x),
//   (P y)'_i = y'_i + x'_i u_i + x_i u'_i - x'_{i-1} u_{i-1} - x_{i-1} u'_{i-1},
// and r_m' = r' + (P y)' / 2.  The two solves share one cyclic reduction
// (the same elimination factors for both right-hand sides).
constexpr int kTmThreads = 1024;
constexpr int kTmMaxP = 4096;

__device__ __forceinline__ void rod_and_dot(const double* rc, const double* vc, int k, double u[3], double ud[3]) {
  const double q[3] = {rc[3 * k + 3] - rc[3 * k], rc[3 * k + 4] - rc[3 * k + 1], rc[3 * k + 5] - rc[3 * k + 2]};
  const double qd[3] = {vc[3 * k + 3] - vc[3 * k], vc[3 * k + 4] - vc[3 * k + 1], vc[3 * k + 5] - vc[3 * k + 2]};
  const double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
#pragma unroll
  for (int e = 0; e < 3; ++e) u[e] = q[e] / qn;
  const double uq = u[0] * qd[0] + u[1] * qd[1] + u[2] * qd[2];
#pragma unroll
  for (int e = 0; e < 3; ++e) ud[e] = (qd[e] - u[e] * uq) / qn;
}

__global__ void __launch_bounds__(kTmThreads) k_tangent_midpoint_dot(const double* __restrict__ r,
                                                                     const double* __restrict__ rdot,
                                                                     const double* __restrict__ y,
                                                                     const double* __restrict__ ydot,
                                                                     const ChainDesc* __restrict__ cd,
                                                                     const int* __restrict__ status,
                                                                     double* __restrict__ rmdot) {
  extern __shared__ __align__(16) double tmd_smem[];
  const int c = blockIdx.x;
  const ChainDesc d = cd[c];
  const int N = d.N, m = d.m, t = threadIdx.x;
  const long long b3 = 3 * d.boff;
  const double *rc = r + b3, *vc = rdot + b3, *yc = y + b3, *ydc = ydot + b3;
  double* out = rmdot + b3;
  if (status[c] != BD_OK) {
    for (int e = t; e < 3 * N; e += kTmThreads) out[e] = vc[e];
    return;
  }
  int P = 1;
  while (P < m) P <<= 1;
  double* ca = tmd_smem;
  double* cb = ca + P;
  double* cc = cb + P;
  double* x1 = cc + P;  // rhs c, then x
  double* x2 = x1 + P;  // rhs c' - H' x, then x'
  // pass 1: H and c; x by cyclic reduction (x2 unused yet)
  for (int i = t; i < P; i += kTmThreads) {
    double a = 0.0, cu = 0.0, rhs = 0.0;
    if (i < m) {
      double u[3], ud[3];
      rod_and_dot(rc, vc, i, u, ud);
      if (i > 0) {
        double up[3], upd[3];
        rod_and_dot(rc, vc, i - 1, up, upd);
        a = -(up[0] * u[0] + up[1] * u[1] + up[2] * u[2]);
      }
      if (i + 1 < m) {
        double un[3], und[3];
        rod_and_dot(rc, vc, i + 1, un, und);
        cu = -(u[0] * un[0] + u[1] * un[1] + u[2] * un[2]);
      }
      rhs = u[0] * (yc[3 * i + 3] - yc[3 * i]) + u[1] * (yc[3 * i + 4] - yc[3 * i + 1]) +
            u[2] * (yc[3 * i + 5] - yc[3 * i + 2]);
    }
    ca[i] = a;
    cb[i] = (i < m) ? 2.0 : 1.0;
    cc[i] = cu;
    x1[i] = rhs;
    x2[i] = 0.0;
  }
  __syncthreads();
  // The elimination runs twice: for x, then, once the right-hand side
  // c' - H' x is formed, for x'.  It overwrites the coefficients, so they are
  // formed again (load_h) before the second run.
  auto solve = [&](double* rhs) {
    for (int s = 1; s < P; s <<= 1) {
      for (int i = 2 * s - 1 + 2 * s * t; i < P; i += 2 * s * kTmThreads) {
        const int l = i - s, rr = i + s;
        const double k1 = ca[i] / cb[l];
        double nb = cb[i] - cc[l] * k1, nd = rhs[i] - rhs[l] * k1, nc = 0.0;
        if (rr < P) {
          const double k2 = cc[i] / cb[rr];
          nb -= ca[rr] * k2;
          nd -= rhs[rr] * k2;
          nc = -cc[rr] * k2;
        }
        ca[i] = -ca[l] * k1;
        cb[i] = nb;
        cc[i] = nc;
        rhs[i] = nd;
      }
      __syncthreads();
    }
    if (t == 0) rhs[P - 1] = rhs[P - 1] / cb[P - 1];
    __syncthreads();
    for (int s = P >> 1; s >= 1; s >>= 1) {
      for (int i = s - 1 + 2 * s * t; i < P; i += 2 * s * kTmThreads) {
        double v = rhs[i];
        if (i - s >= 0) v -= ca[i] * rhs[i - s];
        if (i + s < P) v -= cc[i] * rhs[i + s];
        rhs[i] = v / cb[i];
      }
      __syncthreads();
    }
  };
  auto load_h = [&]() {
    for (int i = t; i < P; i += kTmThreads) {
      double a = 0.0, cu = 0.0;
      if (i < m) {
        double u[3], ud[3];
        rod_and_dot(rc, vc, i, u, ud);
        if (i > 0) {
          double up[3], upd[3];
          rod_and_dot(rc, vc, i - 1, up, upd);
          a = -(up[0] * u[0] + up[1] * u[1] + up[2] * u[2]);
        }
        if (i + 1 < m) {
          double un[3], und[3];
          rod_and_dot(rc, vc, i + 1, un, und);
          cu = -(u[0] * un[0] + u[1] * un[1] + u[2] * un[2]);
        }
      }
      ca[i] = a;
      cb[i] = (i < m) ? 2.0 : 1.0;
      cc[i] = cu;
    }
    __syncthreads();
  };
  solve(x1);
  // rhs of the second solve: c'_k - (H' x)_k
  for (int i = t; i < P; i += kTmThreads) {
    double rhs = 0.0;
    if (i < m) {
      double u[3], ud[3];
      rod_and_dot(rc, vc, i, u, ud);
      const double dy[3] = {yc[3 * i + 3] - yc[3 * i], yc[3 * i + 4] - yc[3 * i + 1], yc[3 * i + 5] - yc[3 * i + 2]};
      const double dyd[3] = {ydc[3 * i + 3] - ydc[3 * i], ydc[3 * i + 4] - ydc[3 * i + 1],
                             ydc[3 * i + 5] - ydc[3 * i + 2]};
      rhs = ud[0] * dy[0] + ud[1] * dy[1] + ud[2] * dy[2] + u[0] * dyd[0] + u[1] * dyd[1] + u[2] * dyd[2];
      if (i > 0) {
        double up[3], upd[3];
        rod_and_dot(rc, vc, i - 1, up, upd);
        const double hd = -(upd[0] * u[0] + upd[1] * u[1] + upd[2] * u[2] + up[0] * ud[0] + up[1] * ud[1] +
                            up[2] * ud[2]);
        rhs -= hd * x1[i - 1];
      }
      if (i + 1 < m) {
        double un[3], und[3];
        rod_and_dot(rc, vc, i + 1, un, und);
        const double hd = -(ud[0] * un[0] + ud[1] * un[1] + ud[2] * un[2] + u[0] * und[0] + u[1] * und[1] +
                            u[2] * und[2]);
        rhs -= hd * x1[i + 1];
      }
    }
    x2[i] = rhs;
  }
  __syncthreads();
  load_h();
  solve(x2);
  // r_m' = r' + (P y)' / 2
  for (int i = t; i < N; i += kTmThreads) {
    double p[3] = {ydc[3 * i], ydc[3 * i + 1], ydc[3 * i + 2]};
    if (i < m) {
      double u[3], ud[3];
      rod_and_dot(rc, vc, i, u, ud);
#pragma unroll
      for (int q = 0; q < 3; ++q) p[q] += x2[i] * u[q] + x1[i] * ud[q];
    }
    if (i > 0) {
      double up[3], upd[3];
      rod_and_dot(rc, vc, i - 1, up, upd);
#pragma unroll
      for (int q = 0; q < 3; ++q) p[q] -= x2[i - 1] * up[q] + x1[i - 1] * upd[q];
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) out[3 * i + q] = vc[3 * i + q] + 0.5 * p[q];
  }
}

cudaError_t launch_tangent_midpoint_dot(const double* r, const double* rdot, const double* y, const double* ydot,
                                        const ChainDesc* cd, int n_chains, const int* status, double* rmdot,
                                        cudaStream_t s) {
  k_tangent_midpoint_dot<<<n_chains, kTmThreads, 5 * kTmMaxP * sizeof(double), s>>>(r, rdot, y, ydot, cd, status,
                                                                                    rmdot);
  return cudaGetLastError();
}

cudaError_t tangent_configure() {
  return cudaFuncSetAttribute(k_tangent_midpoint_dot, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(5 * kTmMaxP * sizeof(double)));
}

// ------------------------------------------------------------ launchers
cudaError_t launch_assemble_dot(const double* r, const double* rdot, const ChainDesc* cd, int n_chains,
                                int max_N, double* Md, double hstar, double a, double hdot,
                                double adot, cudaStream_t s) {
  const long long pairs = (long long)max_N * max_N;
  k_assemble_dot<<<dim3(ceil_div(pairs, 256), n_chains), 256, 0, s>>>(r, rdot, cd, Md, hstar, a,
                                                                       hdot, adot);
  return cudaGetLastError();
}

cudaError_t launch_trsm_rhs(const double* M, const double* Winv, const ChainDesc* cd, int n_chains,
                            int max_tiles, double* B, cudaStream_t s) {
  for (int k = 0; k < max_tiles; ++k) {
    k_trsm_rhs_scale<<<dim3(max_tiles, n_chains), 256, 0, s>>>(Winv, cd, k, B);
    const int below = max_tiles - 1 - k;
    if (below > 0) k_trsm_rhs_update<<<dim3(max_tiles, below, n_chains), 256, 0, s>>>(M, cd, k, B);
  }
  return cudaGetLastError();
}

cudaError_t launch_transpose(const ChainDesc* cd, int n_chains, int max_tiles, double* B,
                             cudaStream_t s) {
  k_transpose<<<dim3(max_tiles, max_tiles, n_chains), 256, 0, s>>>(cd, B);
  return cudaGetLastError();
}

cudaError_t launch_phi_matvec(const double* X, const ChainDesc* cd, int n_chains, int max_n,
                              const double* xi, double* v, cudaStream_t s) {
  k_phi_matvec<<<dim3(ceil_div(max_n, 8), n_chains), 256, 0, s>>>(X, cd, xi, v);
  return cudaGetLastError();
}

cudaError_t launch_gemv_dense(const double* A, const ChainDesc* cd, int n_chains, int max_n,
                              const double* f, double* w, cudaStream_t s) {
  k_gemv_dense<<<dim3(ceil_div(max_n, 8), n_chains), 256, 0, s>>>(A, cd, f, w);
  return cudaGetLastError();
}

cudaError_t launch_tangent_predictor(const double* r, const double* rdot, const double* rq, const double* rqdot,
                                     const double* ydot, const double* uhat, const double* T, const ChainDesc* cd,
                                     int n_chains, int max_N, Phys ph, const double* kappa_dot,
                                     double* rsdot, double* G, cudaStream_t s) {
  k_tangent_predictor<<<dim3(ceil_div(max_N, 128), n_chains), 128, 0, s>>>(r, rdot, rq, rqdot, ydot, uhat, T,
                                                                            cd, ph, kappa_dot, rsdot, G);
  return cudaGetLastError();
}

__global__ void k_vec_add(const ChainDesc* __restrict__ cd, const double* __restrict__ a,
                          const double* __restrict__ b, double* __restrict__ out) {
  const ChainDesc d = cd[blockIdx.y];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.n) return;
  const long long o = 3 * d.boff + e;
  out[o] = a[o] + b[o];
}

cudaError_t launch_vec_add(const ChainDesc* cd, int n_chains, int max_n, const double* a, const double* b,
                           double* out, cudaStream_t s) {
  k_vec_add<<<dim3(ceil_div(max_n, 256), n_chains), 256, 0, s>>>(cd, a, b, out);
  return cudaGetLastError();
}

cudaError_t launch_phi_upper_matvec(const double* X, const ChainDesc* cd, int n_chains, int max_n,
                                    const double* xi, double* v, cudaStream_t s) {
  k_phi_upper_matvec<<<dim3(ceil_div(max_n, 8), n_chains), 256, 0, s>>>(X, cd, xi, v);
  return cudaGetLastError();
}

cudaError_t launch_tangent_base(const ChainDesc* cd, int n_chains, int max_n, Phys ph,
                                const double* rsdot, const double* DdF, const double* DG, double* a,
                                cudaStream_t s) {
  k_tangent_base<<<dim3(ceil_div(max_n, 256), n_chains), 256, 0, s>>>(cd, ph, rsdot, DdF, DG, a);
  return cudaGetLastError();
}

cudaError_t launch_tangent_residual(const double* a, const double* u, const double* rnew,
                                    const ChainDesc* cd, int n_chains, Phys ph, double rel_tol,
                                    double* rscale, double* z, double* rhs, int* state, int* status,
                                    const int* iters, cudaStream_t s) {
  k_tangent_residual<<<n_chains, 256, 0, s>>>(a, u, rnew, cd, ph, rel_tol, rscale, z, rhs, state, status,
                                              iters);
  return cudaGetLastError();
}

cudaError_t launch_tangent_init(const ChainDesc* cd, int n_chains, int max_n, const int* status,
                                int* state, int* iters, double* Tdot, double* Fdot, cudaStream_t s) {
  k_tangent_init<<<dim3(ceil_div(max_n, 256), n_chains), 256, 0, s>>>(cd, status, state, iters, Tdot,
                                                                       Fdot);
  return cudaGetLastError();
}

}  // namespace bd
