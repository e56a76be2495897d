// k_tension.cu -- flow predictor, rod-tension solve and observables.
//
// Rigid rods are the K* -> infinity limit of the paper's semi-implicit
// Fraenkel scheme (Sec. 3 Eqs. (13)-(17)): Eq. (17) gives |Q| = 1 and, rod by
// rod, the tension (|Y| - 1) / (2 dt) that brings the predicted link vector Y
// back to unit length.  That self-only tension is the starting point here;
// the tensions of all rods are then found together so that every rod of
// r(T) = r* + dt D F(T),  F_i = T_i u_i - T_{i-1} u_{i-1}
// has unit length (u_k the rod directions at the start of the step).
//
// The residual is g_k = |Q_k(T)|^2 - 1.  Its Jacobian is
// -2 dt diag(Q(T))^T C^T D C diag(u); the solver keeps its value at Q = u,
// -2 dt K with K = U^T C^T D C U (symmetric positive definite, factored once
// per step), and iterates T <- T + K^{-1} g / (2 dt) until max|g| <= tol,
// followed by one more update, exactly the stopping rule of the oracle's
// Newton.  The root is the same; the convergence is linear with a rate of
// order |Q - u| ~ sqrt(dt) instead of quadratic.
#include <math.h>

#include "bd_internal.h"

namespace bd {

__device__ __forceinline__ double block_max(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) red[0] = v;
  }
  __syncthreads();
  const double r = red[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[0] = v;
  }
  __syncthreads();
  const double r = red[0];
  __syncthreads();
  return r;
}

// ------------------------------------------------------------ rod directions
// u_k = Q_k / |Q_k| at the positions of the start of the step: the directions
// along which the rod tensions act (and the right factor of K).
__global__ void k_rod_dirs(const double* __restrict__ r, const ChainDesc* __restrict__ cd,
                           double* __restrict__ uhat) {
  const ChainDesc d = cd[blockIdx.y];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d.m) return;
  const double* a0 = r + 3 * (d.boff + k);
  const double q0 = a0[3] - a0[0], q1 = a0[4] - a0[1], q2 = a0[5] - a0[2];
  const double inv = 1.0 / sqrt(q0 * q0 + q1 * q1 + q2 * q2);
  double* u = uhat + 3 * (d.roff + k);
  u[0] = q0 * inv;
  u[1] = q1 * inv;
  u[2] = q2 * inv;
}

cudaError_t launch_rod_dirs(const double* r, const ChainDesc* cd, int n_chains, int max_N,
                            double* uhat, cudaStream_t s) {
  k_rod_dirs<<<dim3(ceil_div(max_N, 128), n_chains), 128, 0, s>>>(r, cd, uhat);
  return cudaGetLastError();
}

// ------------------------------------------------------------ predictor
// r* = r + dt kappa.r + y; u_k = Q_k / |Q_k| at the old positions;
// T0_k = (|Q*_k| - 1) / (2 dt); F0 = F(T0).  One thread per bead.
__global__ void k_predictor(const double* __restrict__ r, const double* __restrict__ y,
                            const ChainDesc* __restrict__ cd, int n_chains, Phys ph,
                            double* __restrict__ rstar, const double* __restrict__ uhat,
                            double* __restrict__ T, double* __restrict__ F,
                            int* __restrict__ state, const int* __restrict__ status,
                            int* __restrict__ iters, int* __restrict__ accurate) {
  const int c = blockIdx.y;
  const ChainDesc d = cd[c];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    state[c] = (status[c] == BD_OK) ? NS_ACTIVE : NS_FAILED;
    iters[c] = 0;
    if (accurate) accurate[c] = 0;
  }
  if (i >= d.N) return;
  auto pred = [&](int b, double out[3]) {
    const double* rb = r + 3 * (d.boff + b);
    const double* yb = y + 3 * (d.boff + b);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double kr = ph.kappa[3 * k] * rb[0] + ph.kappa[3 * k + 1] * rb[1] + ph.kappa[3 * k + 2] * rb[2];
      out[k] = rb[k] + ph.dt * kr + yb[k];
    }
  };
  // T0 of rod j from |Q*_j| (self-only, K* -> infinity limit of Eq. (17))
  auto t0 = [&](const double* ra, const double* rb) {
    const double q0 = rb[0] - ra[0], q1 = rb[1] - ra[1], q2 = rb[2] - ra[2];
    return (sqrt(q0 * q0 + q1 * q1 + q2 * q2) - 1.0) / (2.0 * ph.dt);
  };
  double ri[3];
  pred(i, ri);
#pragma unroll
  for (int k = 0; k < 3; ++k) rstar[3 * (d.boff + i) + k] = ri[k];
  double Fi[3] = {0.0, 0.0, 0.0};
  if (i < d.m) {
    double rn[3];
    pred(i + 1, rn);
    const double Ti = t0(ri, rn);
    T[d.roff + i] = Ti;
    const double* ui = uhat + 3 * (d.roff + i);
#pragma unroll
    for (int k = 0; k < 3; ++k) Fi[k] += Ti * ui[k];
  }
  if (i > 0) {  // F_i = T_i u_i - T_{i-1} u_{i-1}; the previous rod's T0 is recomputed
    double rp[3];
    pred(i - 1, rp);
    const double Tp = t0(rp, ri);
    const double* up = uhat + 3 * (d.roff + i - 1);
#pragma unroll
    for (int k = 0; k < 3; ++k) Fi[k] -= Tp * up[k];
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) F[3 * (d.boff + i) + k] = Fi[k];
}

cudaError_t launch_predictor(const double* r, const double* y, const ChainDesc* cd, int n_chains,
                             int max_N, Phys ph, double* rstar, const double* uhat, double* T, double* F,
                             int* state, const int* status, int* iters, int* accurate, cudaStream_t s) {
  k_predictor<<<dim3(ceil_div(max_N, 128), n_chains), 128, 0, s>>>(r, y, cd, n_chains, ph, rstar,
                                                                    uhat, T, F, state, status, iters,
                                                                    accurate);
  return cudaGetLastError();
}

// --------------------------------------------------------- Newton residual
// One CTA per chain: r(T) = r* + dt u (u = D F(T)), g_k, max|g|, state.
__global__ void __launch_bounds__(256) k_newton_residual(const double* __restrict__ rstar,
                                                         const double* __restrict__ u,
                                                         const ChainDesc* __restrict__ cd, Phys ph,
                                                         double* __restrict__ rT,
                                                         double* __restrict__ rhs,
                                                         int* __restrict__ state,
                                                         int* __restrict__ status,
                                                         const int* __restrict__ iters) {
  __shared__ double red[32];
  const int c = blockIdx.x;
  const int st = state[c];
  if (st >= NS_DONE) return;
  if (status[c] != BD_OK) {  // e.g. K not positive definite
    if (threadIdx.x == 0) state[c] = NS_FAILED;
    return;
  }
  const ChainDesc d = cd[c];
  const long long b3 = 3 * d.boff;
  for (int e = threadIdx.x; e < d.n; e += blockDim.x) rT[b3 + e] = rstar[b3 + e] + ph.dt * u[b3 + e];
  __syncthreads();
  double gmax = 0.0;
  const double inv2dt = 0.5 / ph.dt;
  for (int k = threadIdx.x; k < d.m; k += blockDim.x) {
    const double* a = rT + b3 + 3 * k;
    const double q0 = a[3] - a[0], q1 = a[4] - a[1], q2 = a[5] - a[2];
    const double g = q0 * q0 + q1 * q1 + q2 * q2 - 1.0;
    rhs[d.roff + k] = g * inv2dt;
    gmax = (g != g) ? INFINITY : fmax(gmax, fabs(g));
  }
  gmax = block_max(gmax, red);
  if (threadIdx.x == 0) {
    int ns = st;
    if (st == NS_EXTRA) {
      ns = NS_DONE;
    } else if (gmax <= ph.tol) {
      ns = NS_EXTRA;
    } else if (iters[c] >= ph.max_newton || !(gmax < INFINITY)) {
      ns = NS_FAILED;
      atomicCAS(status + c, BD_OK, BD_ERR_CONSTRAINT);
    }
    state[c] = ns;
  }
}

cudaError_t launch_newton_residual(const double* rstar, const double* u, const ChainDesc* cd,
                                   int n_chains, Phys ph, double* rT, double* rhs, int* state,
                                   int* status, const int* iters, cudaStream_t s) {
  k_newton_residual<<<n_chains, 256, 0, s>>>(rstar, u, cd, ph, rT, rhs, state, status, iters);
  return cudaGetLastError();
}

// ------------------------------------------------------------ Newton solve
// One CTA (1024 threads) per chain: K delta = rhs with K = L L^T (row-major
// lower factor of order m, padded to mp) and the stored inverses W_bb of its
// 32 x 32 diagonal blocks; then T += delta, iters++, and F(T) for the next
// mobility product.
//   forward  L z = rhs : block b: s_b = rhs_b - L[b, 0:32b] z (one warp per
//                        row, lanes along the row), z_b = W_bb s_b;
//   backward L^T x = z : block b from the last: x_b = W_bb^T (z_b - acc_b),
//                        then every thread adds L[b rows][a] x_b to the
//                        columns a < 32b it owns (rows read once, coalesced).
constexpr int kSolveThreads = 1024;
constexpr int kSolveCols = 4;   // m <= 4096
constexpr int kSolveMaxM = kSolveThreads * kSolveCols;

// Accumulation type of the solve: K only preconditions the tension iteration
// (its accuracy sets the convergence rate, not the root), so the FP32 copy
// of the mixed path is solved in FP32; the FP64 path stays in FP64.
template <typename T, int BS>
__global__ void __launch_bounds__(kSolveThreads) k_newton_solve(const T* __restrict__ K,
                                                                const T* __restrict__ Kinv,
                                                                const ChainDesc* __restrict__ cd, Phys ph,
                                                                const double* __restrict__ uhat,
                                                                double* __restrict__ rhs,
                                                                double* __restrict__ Tn,
                                                                double* __restrict__ F,
                                                                int* __restrict__ state,
                                                                int* __restrict__ iters) {
  extern __shared__ __align__(16) uint8_t ns_smem[];
  T* zs = reinterpret_cast<T*>(ns_smem);  // [m] solution in the solve's type
  __shared__ T sblk[BS], zblk[BS];
  const int c = blockIdx.x;
  const int st = state[c];
  if (st != NS_ACTIVE && st != NS_EXTRA) return;
  const ChainDesc d = cd[c];
  const int m = d.m;
  const long long mp = d.mp;
  const T* L = K + d.koff;
  const T* Wb = Kinv + d.kwrow * BS;
  double* z = rhs + d.roff;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  constexpr int RPW = BS / 32;  // rows per warp in a block
  const int nb = (m + BS - 1) / BS;
  for (int e = t; e < m; e += kSolveThreads) zs[e] = (T)z[e];
  __syncthreads();
  // forward L y = rhs
  for (int b = 0; b < nb; ++b) {
    const int r0 = BS * b;
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
      const int lr = warp * RPW + q, row = r0 + lr;
      T acc = T(0);
      if (row < m) {
        const T* Lr = L + row * mp;
        for (int cc = lane; cc < r0; cc += 32) acc += Lr[cc] * zs[cc];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) sblk[lr] = (row < m) ? zs[row] - acc : T(0);
    }
    __syncthreads();
    if (t < BS) {
      const T* W = Wb + (long long)r0 * BS;  // W[i][j] at W[i * BS + j]
      T v = T(0);
      for (int j = 0; j <= t; ++j) v += W[t * BS + j] * sblk[j];
      if (r0 + t < m) zs[r0 + t] = v;
    }
    __syncthreads();
  }
  // backward L^T x = y
  T acc[kSolveCols];
#pragma unroll
  for (int q = 0; q < kSolveCols; ++q) acc[q] = T(0);
  for (int b = nb - 1; b >= 0; --b) {
    const int c0 = BS * b;
#pragma unroll
    for (int q = 0; q < kSolveCols; ++q) {
      const int a = t + kSolveThreads * q;
      if (a >= c0 && a < c0 + BS) sblk[a - c0] = ((a < m) ? zs[a] : T(0)) - acc[q];
    }
    __syncthreads();
    if (t < BS) {
      const T* W = Wb + (long long)c0 * BS;
      T v = T(0);  // x_i = sum_{j >= i} W[j][i] s_j
      for (int j = t; j < BS; ++j) v += W[j * BS + t] * sblk[j];
      zblk[t] = v;
      if (c0 + t < m) zs[c0 + t] = v;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kSolveCols; ++q) {
      const int a = t + kSolveThreads * q;
      if (a < c0) {
        const T* col = L + (long long)c0 * mp + a;
        T sacc = T(0);
#pragma unroll 8
        for (int r = 0; r < BS; ++r)
          if (c0 + r < m) sacc += col[r * mp] * zblk[r];
        acc[q] += sacc;
      }
    }
    __syncthreads();
  }
  // T += delta
  for (int k = t; k < m; k += blockDim.x) Tn[d.roff + k] += (double)zs[k];
  __syncthreads();
  // F(T)
  for (int i = t; i < d.N; i += blockDim.x) {
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

template <typename T>
cudaError_t launch_newton_solve(const T* K, const T* Kinv, const ChainDesc* cd, int n_chains, Phys ph,
                                const double* uhat, double* rhs, double* Tn, double* F, int* state,
                                int* iters, cudaStream_t s) {
  k_newton_solve<T, 32><<<n_chains, kSolveThreads, kSolveMaxM * sizeof(T), s>>>(K, Kinv, cd, ph, uhat, rhs,
                                                                                Tn, F, state, iters);
  return cudaGetLastError();
}

// Sets the while-node condition: 1 while any chain is ACTIVE or EXTRA and the
// loop has run fewer than max_loops times in this step (a chain still active
// then is failed by k_finalize; with the per-chain cap of max_newton updates
// the bound is never reached by a correct state machine).
// count: this instance ends a loop iteration (counted in *loops and in the
// step's iteration count); otherwise it only decides whether to enter.
__global__ void k_any_active(const int* __restrict__ state, int n_chains,
                             cudaGraphConditionalHandle h, unsigned long long* loops,
                             StepArgs* args, int max_loops, int count) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int c = threadIdx.x; c < n_chains; c += blockDim.x)
    if (state[c] == NS_ACTIVE || state[c] == NS_EXTRA) any = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    const int k = count ? ++args->loops_in_step : args->loops_in_step;
    cudaGraphSetConditional(h, (any && k < max_loops) ? 1u : 0u);
    if (count) *loops += 1;
  }
}

cudaError_t launch_newton_any_active(const int* state, int n_chains, cudaGraphConditionalHandle h,
                                     unsigned long long* loops, StepArgs* args, int max_loops,
                                     bool count, cudaStream_t s) {
  k_any_active<<<1, 256, 0, s>>>(state, n_chains, h, loops, args, max_loops, count ? 1 : 0);
  return cudaGetLastError();
}

// Commit r <- r(T) for chains that converged; failed chains keep r.
__global__ void k_finalize(const ChainDesc* __restrict__ cd, const double* __restrict__ rT,
                           double* __restrict__ r, const int* __restrict__ state,
                           int* __restrict__ status, StepArgs* args) {
  const int c = blockIdx.y;
  const ChainDesc d = cd[c];
  const int st = state[c];
  if (blockIdx.x == 0 && threadIdx.x == 0 && st != NS_DONE && st != NS_FAILED)
    atomicCAS(status + c, BD_OK, BD_ERR_CONSTRAINT);  // loop ended early (not expected)
  if (st == NS_DONE) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d.n; e += gridDim.x * blockDim.x)
      r[3 * d.boff + e] = rT[3 * d.boff + e];
  }
  if (args && c == 0 && blockIdx.x == 0 && threadIdx.x == 0) {
    args->step += 1;
    args->loops_in_step = 0;
  }
}

cudaError_t launch_finalize(const ChainDesc* cd, int n_chains, long long total_beads,
                            const double* rT, double* r, const int* state, int* status,
                            StepArgs* args, cudaStream_t s) {
  (void)total_beads;
  k_finalize<<<dim3(4, n_chains), 256, 0, s>>>(cd, rT, r, state, status, args);
  return cudaGetLastError();
}

// ------------------------------------------------------------ observables
// Sec. 5 Eqs. (25)-(27) per chain (ensemble averages are the caller's).
__global__ void __launch_bounds__(256) k_observables(const double* __restrict__ r,
                                                     const ChainDesc* __restrict__ cd,
                                                     const int* __restrict__ iters,
                                                     const double* __restrict__ T,
                                                     double* __restrict__ obs) {
  __shared__ double red[32];
  const int c = blockIdx.x;
  const ChainDesc d = cd[c];
  const double* rc = r + 3 * d.boff;
  double s0 = 0, s1 = 0, s2 = 0;
  for (int i = threadIdx.x; i < d.N; i += blockDim.x) {
    s0 += rc[3 * i];
    s1 += rc[3 * i + 1];
    s2 += rc[3 * i + 2];
  }
  const double cx = block_sum(s0, red) / d.N, cy = block_sum(s1, red) / d.N,
               cz = block_sum(s2, red) / d.N;
  double g = 0.0, md = 0.0, txx = 0.0, tyy = 0.0, tzz = 0.0, txy = 0.0;
  for (int i = threadIdx.x; i < d.N; i += blockDim.x) {
    const double dx = rc[3 * i] - cx, dy = rc[3 * i + 1] - cy, dz = rc[3 * i + 2] - cz;
    g += dx * dx + dy * dy + dz * dz;
    if (i < d.m) {
      const double q0 = rc[3 * i + 3] - rc[3 * i], q1 = rc[3 * i + 4] - rc[3 * i + 1],
                   q2 = rc[3 * i + 5] - rc[3 * i + 2];
      md = fmax(md, fabs(sqrt(q0 * q0 + q1 * q1 + q2 * q2) - 1.0));
      const double t = T[d.roff + i];  // Eq. (28) with the rod force T_k Q_k
      txx += t * q0 * q0;
      tyy += t * q1 * q1;
      tzz += t * q2 * q2;
      txy += t * q0 * q1;
    }
  }
  const double rg2 = block_sum(g, red) / d.N;
  md = block_max(md, red);
  txx = block_sum(txx, red);
  tyy = block_sum(tyy, red);
  tzz = block_sum(tzz, red);
  txy = block_sum(txy, red);
  if (threadIdx.x == 0) {
    const double* e = rc + 3 * (d.N - 1);
    const double rx = e[0] - rc[0], ry = e[1] - rc[1], rz = e[2] - rc[2];
    const double R2 = rx * rx + ry * ry + rz * rz;
    double* o = obs + (long long)c * BD_OBS_STRIDE;
    o[0] = rx;
    o[1] = ry;
    o[2] = rz;
    o[3] = R2;
    o[4] = rg2;
    o[5] = sqrt(R2) / (d.N - 1);
    o[6] = md;
    o[7] = (double)iters[c];
    o[BD_OBS_TAU_XX] = txx;
    o[BD_OBS_TAU_YY] = tyy;
    o[BD_OBS_TAU_ZZ] = tzz;
    o[BD_OBS_TAU_XY] = txy;
  }
}

cudaError_t launch_observables(const double* r, const ChainDesc* cd, int n_chains,
                               const int* iters, const double* T, double* obs, cudaStream_t s) {
  k_observables<<<n_chains, 256, 0, s>>>(r, cd, iters, T, obs);
  return cudaGetLastError();
}

__global__ void k_set_args(StepArgs* args, const double* noise, long long stride, int n_steps) {
  args->noise = noise;
  args->stride = stride;
  args->step = 0;
  args->loops_in_step = 0;
  args->n_steps = n_steps;
}

cudaError_t launch_set_args(StepArgs* args, const double* noise, long long stride, int n_steps,
                            cudaStream_t s) {
  k_set_args<<<1, 1, 0, s>>>(args, noise, stride, n_steps);
  return cudaGetLastError();
}

// The step graph's outer WHILE condition, after the step's commit has
// advanced args->step.
__global__ void k_step_loop(const StepArgs* args, cudaGraphConditionalHandle h) {
  cudaGraphSetConditional(h, args->step < args->n_steps ? 1u : 0u);
}

cudaError_t launch_step_loop(const StepArgs* args, cudaGraphConditionalHandle h, cudaStream_t s) {
  k_step_loop<<<1, 1, 0, s>>>(args, h);
  return cudaGetLastError();
}

template cudaError_t launch_newton_solve<double>(const double*, const double*, const ChainDesc*, int,
                                                 Phys, const double*, double*, double*, double*,
                                                 int*, int*, cudaStream_t);

const void* rod_dirs_kernel() { return (const void*)k_rod_dirs; }

cudaError_t tension_configure() {
  cudaError_t e = cudaFuncSetAttribute(k_newton_solve<double, 32>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(kSolveMaxM * sizeof(double)));
  return e;
}

}  // namespace bd
