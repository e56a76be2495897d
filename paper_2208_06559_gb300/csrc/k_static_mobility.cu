// k_static_mobility.cu -- an allocation-free mobility product u = D(r) f for
// one chain, for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not allowed or not safe --
// inside a host framework that owns every device allocation (a plugin, a
// custom allocator arena), on a thread that must not synchronise the device
// (cudaMalloc/cudaFree can), or in a pipeline that forbids allocation after
// start-up.  Such callers cannot create a bd_ctx (bd_create allocates its
// workspace), so this entry point takes the positions and the force vector
// directly and keeps its only scratch in a fixed file-scope device array.
//
// The kernels are the same deterministic two-phase SYMV as the context's
// mobility product (tile partial sums, then a fixed-order reduction), with the
// RPY blocks evaluated on the fly from the positions (the coefficients of
// rpy_dev.h, shared with the assembly) instead of read from a matrix.
//
// Device.  The call works on the current CUDA device: its pointers must be
// memory of that device (checked), and the scratch array used is that
// device's copy.  The array's device address is looked up the first time the
// call runs on a device and then cached; a cudaDeviceReset of that device
// invalidates the cached address, so do not call this after resetting a
// device it has already run on.
//
// Scratch: g_static_scratch holds kStaticTiles x kStaticTiles x 32 x 3 FP64
// partial sums (786,432 bytes) for chains of at most BD_STATIC_MAX_BEADS =
// 1024 beads.  Every GPU that loads this library keeps that array until the
// process exits.  Each call writes every slot it later reads, so nothing has
// to be cleared between calls, but all calls share the one array: two calls
// whose kernels overlap on the GPU (different streams, or different host
// threads) race on it and give wrong results.  Serialise them.
#include <math.h>

#include <cmath>
#include <mutex>

#include "bd_internal.h"
#include "rpy_dev.h"

namespace {

constexpr int kTileBeads = 32;
constexpr int kStaticMaxBeads = BD_STATIC_MAX_BEADS;
constexpr int kStaticTiles = (kStaticMaxBeads + kTileBeads - 1) / kTileBeads;  // 32
constexpr long long kScratchElems = (long long)kStaticTiles * kStaticTiles * kTileBeads * 3;

// File-scope scratch.  In host code this name is only a stand-in for the
// device symbol; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) double g_static_scratch[kScratchElems];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

__device__ __forceinline__ void rpy_block64(const double* ri, const double* rj, double hstar,
                                            double a, double blk[9]) {
  const double R[3] = {ri[0] - rj[0], ri[1] - rj[1], ri[2] - rj[2]};
  double cI, cRR;
  bd::rpy_coeffs<double>(R[0] * R[0] + R[1] * R[1] + R[2] * R[2], hstar, a, cI, cRR);
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int l = 0; l < 3; ++l) blk[3 * k + l] = (k == l ? cI : 0.0) + cRR * R[k] * R[l];
}

// Phase 1: CTA per bead-tile pair (bi <= bj).  Thread t takes row bead
// i = t % 32 of tile bi and column beads 4 (t / 32) .. +3 of tile bj.
// P[t][b] (t, b tile indices, 32 x 3 values each) receives the contribution
// to the rows of tile b from the columns of tile t.
__global__ void __launch_bounds__(256) k_static_tiles(const double* __restrict__ r, int N,
                                                      double hstar, double a,
                                                      const double* __restrict__ f,
                                                      double* __restrict__ P) {
  __shared__ double rowp[8][kTileBeads][3];
  __shared__ double colp[kTileBeads][kTileBeads][3];
  const int TB = (N + kTileBeads - 1) / kTileBeads;
  const int p = blockIdx.x;
  if (p >= TB * (TB + 1) / 2) return;
  int bj = (int)((sqrt(8.0 * p + 1.0) - 1.0) * 0.5);
  while (bj * (bj + 1) / 2 > p) --bj;
  while ((bj + 1) * (bj + 2) / 2 <= p) ++bj;
  const int bi = p - bj * (bj + 1) / 2;  // bi <= bj
  const bool diag = (bi == bj);
  const int ti = threadIdx.x & 31, jg = threadIdx.x >> 5;
  const int i = bi * kTileBeads + ti;
  double rs[3] = {0.0, 0.0, 0.0};
  for (int q = 0; q < 4; ++q) {
    const int tj = jg * 4 + q;
    const int j = bj * kTileBeads + tj;
    double cs[3] = {0.0, 0.0, 0.0};
    const bool use = i < N && j < N && (!diag || ti <= tj);
    if (use) {
      const double* fi = f + 3 * i;
      const double* fj = f + 3 * j;
      if (i == j) {
#pragma unroll
        for (int k = 0; k < 3; ++k) rs[k] += fj[k];  // D_ii = I
      } else {
        double blk[9];
        rpy_block64(r + 3 * i, r + 3 * j, hstar, a, blk);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          rs[k] += blk[3 * k] * fj[0] + blk[3 * k + 1] * fj[1] + blk[3 * k + 2] * fj[2];
          cs[k] = blk[3 * k] * fi[0] + blk[3 * k + 1] * fi[1] + blk[3 * k + 2] * fi[2];
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) colp[ti][tj][k] = cs[k];
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) rowp[jg][ti][k] = rs[k];
  __syncthreads();
  if (threadIdx.x < 3 * kTileBeads) {
    const int b = threadIdx.x / 3, k = threadIdx.x % 3;
    double row = 0.0, col = 0.0;
#pragma unroll
    for (int g = 0; g < 8; ++g) row += rowp[g][b][k];
    for (int q = 0; q < kTileBeads; ++q) col += colp[q][b][k];
    const long long ld = (long long)TB * kTileBeads * 3;
    if (diag) {
      P[bi * ld + 3 * (bi * kTileBeads) + threadIdx.x] = row + col;
    } else {
      P[bj * ld + 3 * (bi * kTileBeads) + threadIdx.x] = row;  // rows of bi from columns of bj
      P[bi * ld + 3 * (bj * kTileBeads) + threadIdx.x] = col;  // rows of bj from columns of bi
    }
  }
}

// Phase 2: u[e] = sum_t P[t][e], fixed order.
__global__ void k_static_reduce(int N, const double* __restrict__ P, double* __restrict__ u) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 3 * N) return;
  const int TB = (N + kTileBeads - 1) / kTileBeads;
  const long long ld = (long long)TB * kTileBeads * 3;
  double s = 0.0;
  for (int t = 0; t < TB; ++t) s += P[t * ld + e];
  u[e] = s;
}

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and cached.
int static_scratch(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BD_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    double* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return BD_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return BD_OK;
}

// True when p is memory of the current device (device or managed memory).
bool on_current_device(const void* p) {
  int dev = 0;
  cudaPointerAttributes at;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" int bd_mobility_apply_static(const double* r_dev, int n_beads, double h_star,
                                        double a, const double* f_dev, double* u_dev,
                                        void* stream) {
  if (!r_dev || !f_dev || !u_dev || n_beads < 1) return BD_ERR_ARG;
  if (!std::isfinite(h_star) || !(h_star >= 0.0) || !std::isfinite(a)) return BD_ERR_ARG;
  if (n_beads > kStaticMaxBeads) return BD_ERR_ARG;  // beyond the fixed scratch
  const double aa = a > 0.0 ? a : h_star;
  if (h_star > 0.0 && aa < h_star) return BD_ERR_ARG;
  if (!on_current_device(r_dev) || !on_current_device(f_dev) || !on_current_device(u_dev)) return BD_ERR_ARG;
  double* P = nullptr;
  const int rc = static_scratch(&P);
  if (rc != BD_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int TB = (n_beads + kTileBeads - 1) / kTileBeads;
  k_static_tiles<<<TB * (TB + 1) / 2, 256, 0, s>>>(r_dev, n_beads, h_star, aa > 0.0 ? aa : 1.0,
                                                   f_dev, P);
  k_static_reduce<<<(3 * n_beads + 255) / 256, 256, 0, s>>>(n_beads, P, u_dev);
  return cudaGetLastError() == cudaSuccess ? BD_OK : BD_ERR_CUDA;
}
