// k_fraenkel.cu -- the paper's own constraint mode: Fraenkel springs with the
// semi-implicit link update of Sec. 3.
//
// Spring k joins beads k and k+1 with force F_k = K* (|Q_k| - 1) Q_k / |Q_k|
// (Sec. 3 Eq. (3)) on bead k and -F_k on bead k+1.  One step:
//   1-3. D, its factor and the Brownian displacement y = sqrt(2 dt) B xi as
//        for rigid rods;
//   k_fraenkel_forces : bead forces Fb_i = F_i - F_{i-1} at the current
//        positions;  u = D Fb  (the mobility product of the rigid path);
//   k_fraenkel_update : explicit bead step dr_i = dt (kappa.r_i + u_i) + y_i
//        (Eq. (6)); per link Y_k = Q_k + dr_{k+1} - dr_k + 2 dt F_k (eqQ2: the
//        2 dt F_k cancels the self term D_kk = D_k+1,k+1 = I of the explicit
//        change), |Q_k'| = (2 dt K* + |Y_k|) / (2 dt K* + 1) (Eq. (25)),
//        Q_k' = Y_k |Q_k'| / |Y_k| (Eq. (23)); positions: the centre of mass
//        moves with the explicit step and the new links are summed around it.
// No tension solve, no rod-coupling matrix.
#include "bd_internal.h"
#include "block_dev.h"

namespace bd {

__device__ __forceinline__ void spring_force(const double* rc, int k, double kspring, double f[3]) {
  double q[3], qn = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    q[c] = rc[3 * (k + 1) + c] - rc[3 * k + c];
    qn += q[c] * q[c];
  }
  qn = sqrt(qn);
  const double s = kspring * (qn - 1.0) / qn;
#pragma unroll
  for (int c = 0; c < 3; ++c) f[c] = s * q[c];
}

__global__ void k_fraenkel_forces(const double* __restrict__ r, const ChainDesc* __restrict__ cd,
                                  double kspring, double* __restrict__ F) {
  const ChainDesc d = cd[blockIdx.y];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.N) return;
  const double* rc = r + 3 * d.boff;
  double f[3] = {0.0, 0.0, 0.0}, s[3];
  if (i < d.N - 1) {
    spring_force(rc, i, kspring, s);
#pragma unroll
    for (int c = 0; c < 3; ++c) f[c] += s[c];
  }
  if (i > 0) {
    spring_force(rc, i - 1, kspring, s);
#pragma unroll
    for (int c = 0; c < 3; ++c) f[c] -= s[c];
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) F[3 * (d.boff + i) + c] = f[c];
}

constexpr int kFrThreads = 1024;
constexpr int kFrPer = 4;  // beads (and links) per thread: N <= 4096

__global__ void __launch_bounds__(kFrThreads) k_fraenkel_update(double* __restrict__ r,
                                                                const double* __restrict__ y,
                                                                const double* __restrict__ u,
                                                                const ChainDesc* __restrict__ cd, Phys ph,
                                                                double* __restrict__ T,
                                                                const int* __restrict__ status,
                                                                int* __restrict__ iters) {
  __shared__ double red[32][3];
  const int c = blockIdx.x;
  if (status[c] != BD_OK) return;  // a failed chain keeps its positions
  const ChainDesc d = cd[c];
  const int N = d.N, m = N - 1;
  double* rc = r + 3 * d.boff;
  const double* yc = y + 3 * d.boff;
  const double* uc = u + 3 * d.boff;
  const int t = threadIdx.x, i0 = kFrPer * t;
  const double dt = ph.dt, K = ph.kspring, tk = 2.0 * dt * K;
  auto bead_dr = [&](int i, double dr[3]) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const double kr = ph.kappa[3 * q] * rc[3 * i] + ph.kappa[3 * q + 1] * rc[3 * i + 1] +
                        ph.kappa[3 * q + 2] * rc[3 * i + 2];
      dr[q] = dt * (kr + uc[3 * i + q]) + yc[3 * i + q];
    }
  };
  // own beads i0 .. i0 + 3: old positions, explicit displacements; own links
  double sr[3] = {0.0, 0.0, 0.0}, sdr[3] = {0.0, 0.0, 0.0}, qn[kFrPer][3];
  double drn[3];
  if (i0 < N) bead_dr(i0, drn);
#pragma unroll
  for (int j = 0; j < kFrPer; ++j) {
    const int i = i0 + j;
#pragma unroll
    for (int q = 0; q < 3; ++q) qn[j][q] = 0.0;
    if (i >= N) continue;
    double dr[3] = {drn[0], drn[1], drn[2]};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      sr[q] += rc[3 * i + q];
      sdr[q] += dr[q];
    }
    if (i < m) {  // link i
      bead_dr(i + 1, drn);
      double fs[3], Y[3], yn = 0.0;
      spring_force(rc, i, K, fs);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        Y[q] = (rc[3 * (i + 1) + q] - rc[3 * i + q]) + (drn[q] - dr[q]) + 2.0 * dt * fs[q];
        yn += Y[q] * Y[q];
      }
      yn = sqrt(yn);
      const double ql = (tk + yn) / (tk + 1.0);
#pragma unroll
      for (int q = 0; q < 3; ++q) qn[j][q] = Y[q] * (ql / yn);
      T[d.roff + i] = K * (ql - 1.0) / ql;
    }
  }
  block_sum3(sr, red);   // N x old centre of mass
  block_sum3(sdr, red);  // N x mean explicit displacement
  // positions of the new links relative to bead 0: exclusive scan of the
  // per-thread link sums, then the running sum inside the thread
  double off[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int j = 0; j < kFrPer; ++j)
#pragma unroll
    for (int q = 0; q < 3; ++q) off[q] += qn[j][q];
  block_exscan3(off, red);
  double rp[kFrPer][3], srp[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int j = 0; j < kFrPer; ++j)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      rp[j][q] = off[q];
      off[q] += qn[j][q];
      if (i0 + j < N) srp[q] += rp[j][q];
    }
  block_sum3(srp, red);  // the block sums end with a barrier: every read of rc is done
  const double invN = 1.0 / (double)N;
#pragma unroll
  for (int j = 0; j < kFrPer; ++j) {
    const int i = i0 + j;
    if (i >= N) continue;
#pragma unroll
    for (int q = 0; q < 3; ++q) rc[3 * i + q] = rp[j][q] - srp[q] * invN + sr[q] * invN + sdr[q] * invN;
  }
  if (t == 0) iters[c] = 0;
}

// End of a step: advance the replay index that selects the step's noise.
__global__ void k_step_done(StepArgs* args) {
  args->step += 1;
  args->loops_in_step = 0;
}

cudaError_t launch_step_done(StepArgs* args, cudaStream_t s) {
  k_step_done<<<1, 1, 0, s>>>(args);
  return cudaGetLastError();
}

cudaError_t launch_fraenkel_forces(const double* r, const ChainDesc* cd, int n_chains, int max_N,
                                   double kspring, double* F, cudaStream_t s) {
  k_fraenkel_forces<<<dim3(ceil_div(max_N, 256), n_chains), 256, 0, s>>>(r, cd, kspring, F);
  return cudaGetLastError();
}

cudaError_t launch_fraenkel_update(double* r, const double* y, const double* u, const ChainDesc* cd,
                                   int n_chains, Phys ph, double* T, const int* status, int* iters,
                                   cudaStream_t s) {
  k_fraenkel_update<<<n_chains, kFrThreads, 0, s>>>(r, y, u, cd, ph, T, status, iters);
  return cudaGetLastError();
}

}  // namespace bd
