// bd_runtime.cu -- the C ABI of libbd (declared in include/bd.h): context
// creation and workspace layout, the captured step graph, and the stage
// entry points.
//
// One bd_step replays a CUDA graph once per time step.  The graph holds the
// whole step for the whole batch: assembly, blocked Cholesky (one group of
// launches per block column), Brownian displacement, flow predictor, the
// rod-coupling matrix K and its factor, then a conditional WHILE node whose
// body (mobility product, residual, solve, condition update) repeats until
// every chain has converged or failed, and the commit of the new positions.
// The noise pointer and the step index live in device memory (StepArgs), so
// the same graph serves every call.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>
#include <mutex>
#include <new>
#include <vector>

#include "bd_internal.h"

using namespace bd;

struct bd_ctx;
using lanes_t = std::vector<bd_ctx*>;
constexpr int kMaxLanes = 8;

struct bd_ctx {
  int device = 0;
  bd_params p{};
  std::vector<int> Nc;
  int n_chains = 0;
  long long total_beads = 0, total_rods = 0;
  int max_N = 0, max_n = 0, max_np = 0, max_m = 0, max_mp = 0;
  bool mixed = false;
  int tileM = kSimtTile;
  Phys ph{};
  std::vector<ChainDesc> h_cd;
  ChainDesc* d_cd = nullptr;
  void* M = nullptr;
  size_t M_elems = 0;
  void* K = nullptr;
  size_t K_elems = 0;
  size_t elem = 8;
  double *r = nullptr, *rstar = nullptr, *rT = nullptr, *y = nullptr, *u = nullptr, *F = nullptr;
  double *uhat = nullptr, *T = nullptr, *rhs = nullptr, *scratch = nullptr, *obs = nullptr;
  float* Winv = nullptr;           // mixed: inverses of the diagonal tiles, [sum np][128]
  float2* fsplit = nullptr;        // mixed: (hi, lo) split of a mobility product's input, [sum np]
  double* dT = nullptr;            // mixed: change of the tensions in the last tension update
  float* G = nullptr;              // mixed: rod-space mobility C D C^T U, [3][mp][mp] per chain
  float* Vsb = nullptr;            // mixed: inverses of the 256-wide diagonal super-blocks of K's factor
  void* Minv = nullptr;            // FP64 path: 32 x 32 diagonal-block inverses of L, [sum np][32]
  void* Kinv = nullptr;            // 32 x 32 diagonal-block inverses of K's factor, [sum mp][32]
  CUtensorMap* tmaps = nullptr;    // mixed: TMA maps (one per chain matrix, Winv, one per chain FP16 copy)
  CUtensorMap* kmaps = nullptr;    // mixed: TMA maps of every chain's K
  __half* M16 = nullptr;           // mixed: FP16 copies of the off-diagonal L tiles, layout of M
  double* stage = nullptr;  // staging for host-memory noise / observables
  size_t stage_elems = 0;
  int *status = nullptr, *state = nullptr, *iters = nullptr;
  int* accurate = nullptr;  // mixed: per chain, mode of the tension iteration's mobility product (MobMode)
  StepArgs* args = nullptr;
  unsigned long long* loops = nullptr;  // Newton loop-body executions (device counter)
  unsigned long long steps_launched = 0;
  size_t graph_kernels = 0, body_kernels = 0;
  cudaStream_t cs = nullptr, cs2 = nullptr;
  int pr_high = 0, pr_low = 0;  // highest (numerically lowest) and lowest stream priorities
  // mixed factorisation: chain groups on their own streams, so that one
  // group's latency-bound diagonal-tile step overlaps another's products
  static constexpr int kMaxGroups = 16;
  int n_groups = 1;
  int panel = 4;                     // super-panel width of the mixed factorisation (tiles)
  std::vector<int> group_start;      // chain index of each group's first chain (+ end)
  std::vector<int> group_tiles;      // max 128-tiles of each group
  cudaStream_t gs[kMaxGroups] = {};
  cudaEvent_t gev[kMaxGroups + 1] = {};
  // concurrent branches of the step: the K chain, the refinement's solve
  cudaStream_t aux[3] = {};  // [0] K chain (low priority), [1] refinement solve, [2] midpoint K chain
  cudaEvent_t aev[7] = {};  // [0,1] K-chain fork/join, [2,3] refinement fork/join, [4,5] caller-stream fence,
                            // [6] mixed: rod directions and G formed
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // forward-mode tangent workspace (allocated by the first bd_adjoint call)
  double *Md = nullptr, *rdot = nullptr, *ydot = nullptr, *rsdot = nullptr, *Gt = nullptr;
  double *abase = nullptr, *zt = nullptr, *DdF = nullptr, *DG = nullptr, *vt = nullptr;
  double *Tdot = nullptr, *Fdot = nullptr, *rscale = nullptr, *kdot = nullptr;
  // midpoint step: y at r, s z, the midpoint's tangent, Phi(X)^T xi, z's tangent
  double *yB = nullptr, *zsv = nullptr, *rmdot = nullptr, *v2 = nullptr, *zdot = nullptr;
  bool have_state = false;
  int direct_iters = 0;  // > 0: launch the step's kernels directly (profiling), no graph
  int graph_unroll = 0;  // tension iterations captured as plain graph nodes before the WHILE node
  bool small = false;    // FP64 rigid rods, every chain <= kSmallMaxN beads: the fused step (k_small.cu)
  unsigned long long small_launches = 0;
  int while_cap = 1;     // WHILE-node iterations allowed per step
  cudaEvent_t* prof = nullptr;  // bd_profile_step: stage-boundary events
  bool fraenkel = false;        // BD_FRAENKEL: semi-implicit spring update instead of the tension solve
  bool midpoint = false;        // rigid rods, BD_SCHEME_MIDPOINT: mobility and rod directions at r_m
  double* rmid = nullptr;       // midpoint positions r_m, [sum N][3]
  double* umid = nullptr;       // unit rod directions of r_m, [sum (N-1)][3]
  void* M2 = nullptr;           // FP64 midpoint path: D(r_m), full symmetric, layout of M
  // lanes: a mixed-precision context of many chains holds sub-contexts over
  // contiguous chain ranges whose steps run concurrently on their own
  // streams; the parent holds no device workspace but the noise staging
  lanes_t lanes;
  std::vector<int> lane_c0;             // first chain of each lane (+ n_chains)
  std::vector<long long> lane_b0;       // first bead of each lane
  std::vector<long long> lane_r0;       // first rod of each lane
  cudaEvent_t fork = nullptr;           // caller-stream event every lane's steps wait for
  std::mutex mu;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

#define CK(call)                                                                  \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      fprintf(stderr, "libbd: %s failed: %s (%s:%d)\n", #call, cudaGetErrorString(e_), \
              __FILE__, __LINE__);                                                \
      return BD_ERR_CUDA;                                                         \
    }                                                                             \
  } while (0)

int enqueue_factor(bd_ctx* c, cudaStream_t s) {
  if (c->mixed) {
    const CUtensorMap* wmap = c->tmaps + c->n_chains;
    const CUtensorMap* maps16 = c->tmaps + c->n_chains + 1;
    if (c->n_groups <= 1) {
      CK(launch_chol_tc((float*)c->M, c->Winv, c->tmaps, wmap, maps16, c->d_cd, c->n_chains,
                        c->max_np / kMixedTile, c->panel, c->status, s));
      return BD_OK;
    }
    // fork
    CK(cudaEventRecord(c->gev[c->kMaxGroups], s));
    for (int g = 0; g < c->n_groups; ++g) {
      CK(cudaStreamWaitEvent(c->gs[g], c->gev[c->kMaxGroups], 0));
      const int c0 = c->group_start[g], c1 = c->group_start[g + 1];
      CK(launch_chol_tc((float*)c->M, c->Winv, c->tmaps + c0, wmap, maps16 + c0, c->d_cd + c0, c1 - c0,
                        c->group_tiles[g], c->panel, c->status + c0, c->gs[g]));
      CK(cudaEventRecord(c->gev[g], c->gs[g]));
    }
    // join
    for (int g = 0; g < c->n_groups; ++g) CK(cudaStreamWaitEvent(s, c->gev[g], 0));
    return BD_OK;
  }
    CK(launch_chol_simt<double>((double*)c->M, (double*)c->Minv, c->d_cd, c->n_chains,
                                c->max_np / kSimtTile, false, c->status, s));
  return BD_OK;
}

int enqueue_assemble(bd_ctx* c, cudaStream_t s) {
  const double a = c->ph.a;
  if (c->mixed)
    CK(launch_assemble<float>(c->r, (float*)c->M, c->d_cd, c->n_chains, c->max_N, c->max_np, c->ph.hstar,
                              a, c->fsplit, s));
  else
    CK(launch_assemble<double>(c->r, (double*)c->M, c->d_cd, c->n_chains, c->max_N, c->max_np,
                               c->ph.hstar, a, nullptr, s));
  return BD_OK;
}


// y = sqrt(2 dt) B xi; xi from `x` or, when args != NULL, from the step's
// slice of the noise array.
int enqueue_brownian(bd_ctx* c, const double* x, const StepArgs* args, double* y, cudaStream_t s) {
  const double sc = c->ph.sq2dt;
  if (c->mixed)  // buffers rT, F, u are free at this point of the step
    CK(launch_brownian_f32((const float*)c->M, c->Winv, c->d_cd, c->n_chains, c->max_np, x, args, sc,
                           c->p.refine != 0, y, c->rT, c->F, c->u, c->scratch, c->fsplit, s,
                           c->aux[1], c->aev + 2));
  else
    CK(launch_trmv<double>((const double*)c->M, c->d_cd, c->n_chains, c->max_n, x, args, sc, y, s));
  return BD_OK;
}

// u = D f with the matrix `Mat` (the context's M, or the midpoint matrix M2).
int enqueue_symv(bd_ctx* c, const void* Mat, const double* f, double* u, const int* state, cudaStream_t s) {
  if (c->mixed)
    CK(launch_symv_f32((const float*)Mat, c->d_cd, c->n_chains, c->max_np, f, c->fsplit, c->scratch, u,
                       state, s));
  else
    CK(launch_symv<double>((const double*)Mat, c->d_cd, c->n_chains, c->max_np, f, c->scratch, u,
                           state, s));
  return BD_OK;
}

// Stage-boundary event for bd_profile_step (no-op otherwise).
void prof_mark(bd_ctx* c, int i, cudaStream_t s) {
  if (c->prof) cudaEventRecord(c->prof[i], s);
}

// Midpoint step, FP64 path: D and its factor at r, y = s L xi and
// z = s L^{-T} xi (in F, free until the predictor), r_m and its rod
// directions, D(r_m) assembled into M2; then the K chain (K of D(r_m) and
// the directions of r_m, its factor) beside the product y = D(r_m) z.
int enqueue_pre_newton_mid_fp64(bd_ctx* c, cudaStream_t s) {
  int rc;
  cudaStream_t sk = c->aux[2];
  if ((rc = enqueue_assemble(c, s))) return rc;
  prof_mark(c, 1, s);
  if ((rc = enqueue_factor(c, s))) return rc;
  prof_mark(c, 2, s);
  CK(launch_trmv<double>((const double*)c->M, c->d_cd, c->n_chains, c->max_n, nullptr, c->args, c->ph.sq2dt,
                         c->y, s));
  CK(launch_trsv_t_f64((const double*)c->M, (const double*)c->Minv, c->d_cd, c->n_chains, c->max_n, nullptr,
                       c->args, c->ph.sq2dt, c->F, s));
  CK(launch_tangent_midpoint(c->r, c->y, nullptr, 1.0, c->d_cd, c->n_chains, c->status, c->rmid, c->umid, s));
  CK(launch_assemble<double>(c->rmid, (double*)c->M2, c->d_cd, c->n_chains, c->max_N, c->max_np, c->ph.hstar,
                             c->ph.a, nullptr, s));
  CK(cudaEventRecord(c->aev[0], s));
  CK(cudaStreamWaitEvent(sk, c->aev[0], 0));
  CK(launch_form_k<double>((const double*)c->M2, (double*)c->K, c->d_cd, c->n_chains, c->max_m, c->umid, sk));
  CK(launch_chol_simt<double>((double*)c->K, (double*)c->Kinv, c->d_cd, c->n_chains, c->max_mp / kSimtTile,
                              true, c->status, sk));
  prof_mark(c, 7, sk);
  CK(cudaEventRecord(c->aev[1], sk));
  if ((rc = enqueue_symv(c, c->M2, c->F, c->y, nullptr, s))) return rc;
  prof_mark(c, 3, s);
  CK(cudaStreamWaitEvent(s, c->aev[1], 0));
  CK(launch_predictor(c->r, c->y, c->d_cd, c->n_chains, c->max_N, c->ph, c->rstar, c->umid, c->T, c->F,
                      c->state, c->status, c->iters, nullptr, s));
  prof_mark(c, 4, s);
  return BD_OK;
}

// Midpoint step, mixed path.  D and its tensor-core factor at r; the product
// Lt xi (the raw displacement s Lt xi places the midpoint: its correlation
// with z = Lt^{-T} xi is exactly s^2 I) while the solve for z runs beside it;
// r_m and its rod directions; then the K chain (K and G of r_m, K's factor
// and super-block inverses) on its own high-priority stream, beside the
// refinement's product D z, y += s (D(r_m) - D(r)) z from the positions and
// the predictor.  The first tension product waits for G, the first solve for
// the end of the K chain.
int enqueue_pre_newton_mid_mixed(bd_ctx* c, cudaStream_t s) {
  int rc;
  cudaStream_t sk = c->aux[2];
  const bool refine = c->p.refine != 0;
  if ((rc = enqueue_assemble(c, s))) return rc;
  prof_mark(c, 1, s);
  if ((rc = enqueue_factor(c, s))) return rc;
  prof_mark(c, 2, s);
  CK(launch_brownian_f32_begin((const float*)c->M, c->Winv, c->d_cd, c->n_chains, c->max_np, nullptr, c->args,
                               c->ph.sq2dt, refine, c->y, c->rT, c->F, c->scratch, s, c->aux[1], c->aev + 2, true));
  CK(launch_tangent_midpoint(c->r, refine ? c->rT : c->y, nullptr, refine ? c->ph.sq2dt : 1.0, c->d_cd,
                             c->n_chains, c->status, c->rmid, c->umid, s));
  CK(cudaEventRecord(c->aev[0], s));
  CK(cudaStreamWaitEvent(sk, c->aev[0], 0));
  CK(launch_form_k_pos(c->rmid, (float*)c->K, c->G, c->d_cd, c->n_chains, c->max_m, c->umid, c->ph.hstar,
                       c->ph.a, sk));
  CK(cudaEventRecord(c->aev[6], sk));
  CK(launch_chol_k64((float*)c->K, (float*)c->Kinv, c->kmaps, c->d_cd, c->n_chains, c->max_mp / 64, c->status, sk));
  CK(launch_sb_inverse((const float*)c->K, (const float*)c->Kinv, c->Vsb, c->d_cd, c->n_chains, c->max_mp, sk));
  prof_mark(c, 7, sk);
  CK(cudaEventRecord(c->aev[1], sk));
  CK(launch_brownian_f32_end((const float*)c->M, c->d_cd, c->n_chains, c->max_np, c->ph.sq2dt, refine, c->y,
                             c->rT, c->F, c->u, c->scratch, c->fsplit, s, c->aev + 2, true));
  CK(launch_mob_delta_f32(c->r, c->rmid, c->F, c->d_cd, c->n_chains, c->max_N, c->status, c->ph.hstar, c->ph.a,
                          c->ph.sq2dt, c->y, s));
  prof_mark(c, 3, s);
  CK(launch_predictor(c->r, c->y, c->d_cd, c->n_chains, c->max_N, c->ph, c->rstar, c->umid, c->T, c->F,
                      c->state, c->status, c->iters, c->accurate, s));
  CK(cudaStreamWaitEvent(s, c->aev[6], 0));  // G of r_m, for the first product
  prof_mark(c, 4, s);
  return BD_OK;
}

// Before the tension solve.  The K chain (rod directions, K, its factor)
// needs only the old positions and the upper-triangle D, so it runs on its
// own stream while D is factored and the Brownian displacement is formed.
int enqueue_pre_newton(bd_ctx* c, cudaStream_t s) {
  if (c->midpoint) return c->mixed ? enqueue_pre_newton_mid_mixed(c, s) : enqueue_pre_newton_mid_fp64(c, s);
  int rc;
  cudaStream_t sk = c->aux[0];
  if (c->mixed) {
    // K from the positions: the chain forks before the assembly
    CK(cudaEventRecord(c->aev[0], s));
    CK(cudaStreamWaitEvent(sk, c->aev[0], 0));
  }
  if ((rc = enqueue_assemble(c, s))) return rc;
  prof_mark(c, 1, s);
  if (!c->mixed) {
    CK(cudaEventRecord(c->aev[0], s));
    CK(cudaStreamWaitEvent(sk, c->aev[0], 0));
  }
  CK(launch_rod_dirs(c->r, c->d_cd, c->n_chains, c->max_N, c->uhat, sk));
  if (c->mixed) {
    CK(launch_form_k_pos(c->r, (float*)c->K, c->G, c->d_cd, c->n_chains, c->max_m, c->uhat, c->ph.hstar,
                         c->ph.a, sk));
    CK(cudaEventRecord(c->aev[6], sk));  // the predictor and the first product need only these
    CK(launch_chol_k64((float*)c->K, (float*)c->Kinv, c->kmaps, c->d_cd, c->n_chains, c->max_mp / 64,
                       c->status, sk));
    CK(launch_sb_inverse((const float*)c->K, (const float*)c->Kinv, c->Vsb, c->d_cd, c->n_chains, c->max_mp, sk));
  } else {
    CK(launch_form_k<double>((const double*)c->M, (double*)c->K, c->d_cd, c->n_chains, c->max_m,
                             c->uhat, sk));
    CK(launch_chol_simt<double>((double*)c->K, (double*)c->Kinv, c->d_cd, c->n_chains,
                                c->max_mp / kSimtTile, true, c->status, sk));
  }
  prof_mark(c, 7, sk);
  CK(cudaEventRecord(c->aev[1], sk));
  if ((rc = enqueue_factor(c, s))) return rc;
  prof_mark(c, 2, s);
  if ((rc = enqueue_brownian(c, nullptr, c->args, c->y, s))) return rc;
  prof_mark(c, 3, s);
  // mixed path: K's factor is awaited only before the first solve
  CK(cudaStreamWaitEvent(s, c->aev[c->mixed ? 6 : 1], 0));
  CK(launch_predictor(c->r, c->y, c->d_cd, c->n_chains, c->max_N, c->ph, c->rstar, c->uhat, c->T,
                      c->F, c->state, c->status, c->iters, c->mixed ? c->accurate : nullptr, s));
  prof_mark(c, 4, s);
  return BD_OK;
}

// One tension iteration.  FP64 path: the bead-space mobility product D F,
// the residual from r(T) = r* + dt D F, the solve.  Mixed path: the rod-space
// product w = G T (plain FP32 sums while a chain's residual is large,
// compensated after, increments G dT once accurate), the residual from
// Q(T) = Q* - dt w, the solve (which also records dT).  `first`: the step's
// first iteration, whose solve waits for the end of the K chain (K's factor
// and its super-block inverses) -- the product and residual run beside it.
int enqueue_newton_iter(bd_ctx* c, cudaStream_t s, bool first = false) {
  const double* udir = c->midpoint ? c->umid : c->uhat;
  if (c->mixed) {
    CK(launch_tension_products_g(c->G, c->d_cd, c->n_chains, c->max_mp, c->T, c->dT, c->u, c->state,
                                 c->accurate, s));
    CK(launch_newton_residual_g(c->rstar, c->u, c->d_cd, c->n_chains, c->ph, c->rhs, c->state, c->status,
                                c->iters, c->accurate, s));
    if (first) CK(cudaStreamWaitEvent(s, c->aev[1], 0));
    CK(launch_newton_solve_sb((const float*)c->K, c->Vsb, c->d_cd, c->n_chains, c->ph, udir, c->rhs, c->T,
                              c->F, c->state, c->iters, c->dT, s));
    return BD_OK;
  }
  int rc;
  if ((rc = enqueue_symv(c, c->midpoint ? c->M2 : c->M, c->F, c->u, c->state, s))) return rc;
  CK(launch_newton_residual(c->rstar, c->u, c->d_cd, c->n_chains, c->ph, c->rT, c->rhs, c->state,
                            c->status, c->iters, s));
  CK(launch_newton_solve<double>((const double*)c->K, (const double*)c->Kinv, c->d_cd, c->n_chains, c->ph,
                                 udir, c->rhs, c->T, c->F, c->state, c->iters, s));
  return BD_OK;
}

// Commit the step: r <- r(T) for converged chains (mixed path: rebuilt from
// the rods), step index advanced.
int enqueue_finalize(bd_ctx* c, cudaStream_t s) {
  if (c->mixed)
    CK(launch_finalize_g(c->d_cd, c->n_chains, c->ph, c->midpoint ? c->rmid : c->r, c->rstar, c->u, c->F, c->r,
                         c->state, c->status, c->args, s));
  else
    CK(launch_finalize(c->d_cd, c->n_chains, c->total_beads, c->rT, c->r, c->state, c->status, c->args,
                       s));
  return BD_OK;
}

// Body of the WHILE node: one iteration, then the loop condition.
int enqueue_newton_body(bd_ctx* c, cudaGraphConditionalHandle h, cudaStream_t s) {
  int rc;
  if ((rc = enqueue_newton_iter(c, s))) return rc;
  CK(launch_newton_any_active(c->state, c->n_chains, h, c->loops, c->args, c->while_cap, true, s));
  return BD_OK;
}

size_t count_kernel_nodes(cudaGraph_t g) {
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return 0;
  std::vector<cudaGraphNode_t> nodes(n);
  if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return 0;
  size_t k = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

// Kernel nodes of a captured graph keep no stream priority: the K chain's
// nodes get the lowest priority, every other kernel the highest (mixed path;
// the FP64 path shares its tile kernels between both chains and keeps them
// all high).
void set_graph_priorities(bd_ctx* c, cudaGraph_t g) {
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess || n == 0) return;
  std::vector<cudaGraphNode_t> nodes(n);
  if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
    cudaKernelNodeParams kp;
    if (cudaGraphKernelNodeGetParams(nd, &kp) != cudaSuccess) continue;
    // (the midpoint step's K chain is on the critical path: high priority)
    const bool kchain = c->mixed && !c->midpoint && (kp.func == rod_dirs_kernel() ||
                                     is_k64_kernel(kp.func) || is_kchain_form_kernel(kp.func) ||
                                     is_sb_inverse_kernel(kp.func));
    cudaLaunchAttributeValue v;
    memset(&v, 0, sizeof(v));
    v.priority = kchain ? c->pr_low : c->pr_high;
    cudaGraphKernelNodeSetAttribute(nd, cudaLaunchAttributePriority, &v);
  }
  cudaGetLastError();
}

// Fraenkel-spring step (Sec. 3): D, its factor and the Brownian displacement
// as for rigid rods, the bead forces of the springs, one mobility product,
// then the per-link semi-implicit update, which also commits the positions.
int enqueue_step_fraenkel(bd_ctx* c, cudaStream_t s) {
  int rc;
  prof_mark(c, 0, s);
  if ((rc = enqueue_assemble(c, s))) return rc;
  prof_mark(c, 1, s);
  prof_mark(c, 7, s);  // no K chain in this mode
  if ((rc = enqueue_factor(c, s))) return rc;
  prof_mark(c, 2, s);
  if ((rc = enqueue_brownian(c, nullptr, c->args, c->y, s))) return rc;
  prof_mark(c, 3, s);
  CK(launch_fraenkel_forces(c->r, c->d_cd, c->n_chains, c->max_N, c->ph.kspring, c->F, s));
  if ((rc = enqueue_symv(c, c->M, c->F, c->u, nullptr, s))) return rc;
  prof_mark(c, 4, s);
  CK(launch_fraenkel_update(c->r, c->y, c->u, c->d_cd, c->n_chains, c->ph, c->T, c->status, c->iters, s));
  prof_mark(c, 5, s);
  CK(launch_step_done(c->args, s));
  prof_mark(c, 6, s);
  return BD_OK;
}

// Captures one step into `step` (the body of the graph's outer WHILE node):
// the pre-solve stages, the first graph_unroll tension iterations as plain
// nodes (chains that have converged skip them on the device), an inner WHILE
// node for the rest, the commit, and the outer loop's condition.  *inner
// receives the inner WHILE node's body (null in Fraenkel mode).
static int capture_step(bd_ctx* c, cudaGraph_t step, cudaGraphConditionalHandle hs, cudaGraph_t* inner) {
  *inner = nullptr;
  cudaStream_t s = c->cs;
  CK(cudaStreamBeginCaptureToGraph(s, step, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  auto end_capture = [&](int rc) {
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &g);  // `step` is owned by its WHILE node
    return rc ? rc : (e == cudaSuccess ? BD_OK : BD_ERR_CUDA);
  };
  if (c->fraenkel) {
    int rc = enqueue_step_fraenkel(c, s);
    if (rc == BD_OK && launch_step_loop(c->args, hs, s) != cudaSuccess) rc = BD_ERR_CUDA;
    return end_capture(rc);
  }
  int rc = enqueue_pre_newton(c, s);
  for (int i = 0; rc == BD_OK && i < c->graph_unroll; ++i) rc = enqueue_newton_iter(c, s, i == 0);
  if (rc == BD_OK && c->graph_unroll == 0 && c->mixed && cudaStreamWaitEvent(s, c->aev[1], 0) != cudaSuccess)
    rc = BD_ERR_CUDA;
  c->while_cap = c->ph.max_newton + 3 - c->graph_unroll;
  if (c->while_cap < 1) c->while_cap = 1;
  if (rc) return end_capture(rc);
  cudaStreamCaptureStatus cst;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaGraph_t cg = nullptr;
  cudaGraphConditionalHandle h;
  // The inner loop's condition is set by a kernel in every step (enter only
  // if a chain is still iterating), not left to the handle's default.
  if (cudaStreamGetCaptureInfo(s, &cst, nullptr, &cg, &deps, nullptr, &ndeps) != cudaSuccess ||
      cudaGraphConditionalHandleCreate(&h, cg, 0, cudaGraphCondAssignDefault) != cudaSuccess ||
      launch_newton_any_active(c->state, c->n_chains, h, c->loops, c->args, c->while_cap, false, s) !=
          cudaSuccess ||
      cudaStreamGetCaptureInfo(s, &cst, nullptr, &cg, &deps, nullptr, &ndeps) != cudaSuccess)
    return end_capture(BD_ERR_CUDA);
  // cudaGraphNodeParams holds a union without a default constructor
  alignas(cudaGraphNodeParams) unsigned char cp_buf[sizeof(cudaGraphNodeParams)];
  memset(cp_buf, 0, sizeof(cp_buf));
  cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_buf);
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  if (cudaGraphAddNode(&node, cg, deps, nullptr, ndeps, &cp) != cudaSuccess ||
      cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies) !=
          cudaSuccess)
    return end_capture(BD_ERR_CUDA);
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if (cudaStreamBeginCaptureToGraph(c->cs2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
      cudaSuccess)
    return end_capture(BD_ERR_CUDA);
  rc = enqueue_newton_body(c, h, c->cs2);
  cudaGraph_t body_out = nullptr;
  if (cudaStreamEndCapture(c->cs2, &body_out) != cudaSuccess && rc == BD_OK) rc = BD_ERR_CUDA;
  if (rc == BD_OK) rc = enqueue_finalize(c, s);
  if (rc == BD_OK && launch_step_loop(c->args, hs, s) != cudaSuccess) rc = BD_ERR_CUDA;
  *inner = body;
  return end_capture(rc);
}

// The step graph: one WHILE node whose body is one step (capture_step); the
// commit advances the step index and the body's last kernel continues the
// loop while steps of the bd_step call remain, so one launch of the graph
// advances every chain of the batch, however uneven, by all the steps of the
// call.  The condition's default is 1: every launch runs at least one step.
int build_step_graph(bd_ctx* c) {
  if (c->exec) return BD_OK;
  cudaGraph_t top = nullptr;
  CK(cudaGraphCreate(&top, 0));
  cudaGraphConditionalHandle hs;
  alignas(cudaGraphNodeParams) unsigned char cp_buf[sizeof(cudaGraphNodeParams)];
  memset(cp_buf, 0, sizeof(cp_buf));
  cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_buf);
  cudaGraphNode_t node;
  cudaGraph_t inner = nullptr;
  int rc = BD_OK;
  if (cudaGraphConditionalHandleCreate(&hs, top, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
    rc = BD_ERR_CUDA;
  } else {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hs;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if (cudaGraphAddNode(&node, top, nullptr, nullptr, 0, &cp) != cudaSuccess) rc = BD_ERR_CUDA;
  }
  cudaGraph_t step = rc == BD_OK ? cp.conditional.phGraph_out[0] : nullptr;
  if (rc == BD_OK) rc = capture_step(c, step, hs, &inner);
  if (rc) {
    cudaGraphDestroy(top);
    return rc;
  }
  set_graph_priorities(c, step);
  if (inner) set_graph_priorities(c, inner);
  c->graph = top;
  c->graph_kernels = count_kernel_nodes(step);  // per step
  c->body_kernels = inner ? count_kernel_nodes(inner) : 0;
  CK(cudaGraphInstantiate(&c->exec, top, cudaGraphInstantiateFlagUseNodePriority));
  return BD_OK;
}

// Direct (graph-free) step for kernel-level profilers that cannot see into a
// graph's conditional node: the same kernels, with the tension-solve body
// enqueued a fixed number of times (converged chains skip it on the device).
int enqueue_step_direct(bd_ctx* c, cudaStream_t s) {
  if (c->fraenkel) return enqueue_step_fraenkel(c, s);
  int rc;
  prof_mark(c, 0, s);
  if ((rc = enqueue_pre_newton(c, s))) return rc;
  for (int it = 0; it < c->direct_iters; ++it)
    if ((rc = enqueue_newton_iter(c, s, it == 0))) return rc;
  prof_mark(c, 5, s);
  if ((rc = enqueue_finalize(c, s))) return rc;
  prof_mark(c, 6, s);
  return BD_OK;
}

// Split the chains into G groups (each factored on its own stream).
void set_groups(bd_ctx* c, int G) {
  if (G < 1) G = 1;
  if (G > bd_ctx::kMaxGroups) G = bd_ctx::kMaxGroups;
  if (G > c->n_chains) G = c->n_chains;
  c->n_groups = G;
  c->group_start.assign(G + 1, 0);
  c->group_tiles.assign(G, 0);
  for (int g = 0; g <= G; ++g) c->group_start[g] = (int)((long long)c->n_chains * g / G);
  for (int g = 0; g < G; ++g)
    for (int i = c->group_start[g]; i < c->group_start[g + 1]; ++i)
      if (c->h_cd[i].np / kMixedTile > c->group_tiles[g]) c->group_tiles[g] = c->h_cd[i].np / kMixedTile;
}

void drop_graph(bd_ctx* c) {
  if (c->exec) cudaGraphExecDestroy(c->exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->exec = nullptr;
  c->graph = nullptr;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int ensure_stage(bd_ctx* c, size_t elems) {
  if (c->stage_elems >= elems) return BD_OK;
  if (c->stage) cudaFree(c->stage);
  c->stage = nullptr;
  c->stage_elems = 0;
  if (cudaMalloc(&c->stage, elems * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return BD_ERR_OOM;
  }
  c->stage_elems = elems;
  return BD_OK;
}

int worst(const int* st, int n) {
  int w = BD_OK;
  for (int i = 0; i < n; ++i)
    if (st[i] != BD_OK && (w == BD_OK || st[i] < w)) w = st[i];
  return w;
}

template <typename T>
__global__ void k_residual_fro(const T* M, const ChainDesc* cd, int chain, double* acc) {
  const ChainDesc d = cd[chain];
  const T* base = M + d.moff;
  const long long np = d.np;
  double num = 0.0, den = 0.0;
  const long long total = (long long)d.n * (d.n + 1) / 2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)((sqrt(8.0 * (double)e + 1.0) - 1.0) * 0.5);
    while ((long long)i * (i + 1) / 2 > e) --i;
    while ((long long)(i + 1) * (i + 2) / 2 <= e) ++i;
    const int j = (int)(e - (long long)i * (i + 1) / 2);  // j <= i
    double s = 0.0;
    for (int k = 0; k <= j; ++k) s += (double)base[i * np + k] * (double)base[j * np + k];
    const double dij = (i == j) ? 1.0 : (double)base[(long long)j * np + i];
    const double w = (i == j) ? 1.0 : 2.0;
    num += w * (s - dij) * (s - dij);
    den += w * dij * dij;
  }
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, o);
    den += __shfl_xor_sync(0xffffffffu, den, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(acc, num);
    atomicAdd(acc + 1, den);
  }
}

}  // namespace

extern "C" {

void bd_params_default(bd_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->n_chains = 1;
  p->n_beads = nullptr;
  p->h_star = 0.25;
  p->a = 0.0;
  p->dt = 1e-4;
  p->flow = BD_FLOW_NONE;
  p->Wi = 0.0;
  p->lambda = 1.0;
  p->precision = BD_FP64;
  p->constraint = BD_RIGID;
  p->tol = 1e-13;
  p->max_newton = 50;
  p->refine = 1;
  p->k_spring = 1e4;
}

const char* bd_strerror(int code) {
  switch (code) {
    case BD_OK: return "ok";
    case BD_ERR_ARG: return "invalid argument";
    case BD_ERR_CUDA: return "CUDA runtime error";
    case BD_ERR_OOM: return "device allocation failed";
    case BD_ERR_NOT_PD: return "diffusion tensor not positive definite (Cholesky pivot <= 0 or NaN)";
    case BD_ERR_CONSTRAINT: return "rod-tension Newton did not converge";
    case BD_ERR_TIMEOUT: return "bounded device wait expired";
    case BD_ERR_STATE: return "no state loaded (call bd_set_state first)";
    default: return "unknown error";
  }
}

static void ctx_destroy(bd_ctx* c) {
  if (!c) return;
  DeviceGuard g(c->device);
  if (c->exec) cudaGraphExecDestroy(c->exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  void* bufs[] = {c->d_cd, c->M,     c->K,       c->r,   c->rstar, c->rT,     c->y,
                  c->u,    c->F,     c->uhat,    c->T,   c->rhs,   c->scratch, c->obs,
                  c->stage, c->status, c->state, c->iters, c->accurate, c->args, c->loops, c->Winv, c->fsplit, c->dT, c->G, c->Vsb, c->M16, c->tmaps, c->kmaps,
                  c->Minv, c->Kinv, c->Md, c->rdot, c->ydot, c->rsdot, c->Gt, c->abase,
                  c->zt, c->DdF, c->DG, c->vt, c->Tdot, c->Fdot, c->rscale, c->kdot, c->rmid, c->umid, c->M2, c->yB, c->zsv, c->rmdot, c->v2, c->zdot};
  for (void* b : bufs)
    if (b) cudaFree(b);
  for (int g = 0; g < bd_ctx::kMaxGroups; ++g)
    if (c->gs[g]) cudaStreamDestroy(c->gs[g]);
  for (int g = 0; g <= bd_ctx::kMaxGroups; ++g)
    if (c->gev[g]) cudaEventDestroy(c->gev[g]);
  for (int g = 0; g < 3; ++g)
    if (c->aux[g]) cudaStreamDestroy(c->aux[g]);
  for (int g = 0; g < 7; ++g)
    if (c->aev[g]) cudaEventDestroy(c->aev[g]);
  if (c->cs) cudaStreamDestroy(c->cs);
  if (c->cs2) cudaStreamDestroy(c->cs2);
  delete c;
}

// Checks every field of *p; no device call.
static int validate_params(const bd_params* p) {
  if (!p || p->n_chains < 1 || !p->n_beads) return BD_ERR_ARG;
  if (p->lanes < 0 || p->lanes > kMaxLanes) return BD_ERR_ARG;
  if (!(p->dt > 0.0) || !(p->h_star >= 0.0)) return BD_ERR_ARG;
  if (!std::isfinite(p->dt) || !std::isfinite(p->h_star) || !std::isfinite(p->Wi) ||
      !std::isfinite(p->lambda) || !std::isfinite(p->tol))
    return BD_ERR_ARG;
  const double a = p->a > 0.0 ? p->a : p->h_star;
  if (p->h_star > 0.0 && a < p->h_star) return BD_ERR_ARG;  // D may not be positive definite
  if (p->flow < BD_FLOW_NONE || p->flow > BD_FLOW_UNIAXIAL) return BD_ERR_ARG;
  // BD_MIXED_BF16 names a factorisation with BF16 operands, which is not built
  if (p->precision != BD_FP64 && p->precision != BD_MIXED_TF32) return BD_ERR_ARG;
  if (p->constraint != BD_RIGID && p->constraint != BD_FRAENKEL) return BD_ERR_ARG;
  if (p->constraint == BD_FRAENKEL && !(p->k_spring > 0.0 && p->k_spring < 1e300)) return BD_ERR_ARG;
  if (p->scheme != BD_SCHEME_MIDPOINT && p->scheme != BD_SCHEME_EULER) return BD_ERR_ARG;
  // limits of the per-chain kernels: FP64 path, N <= 4096 (the tension solve
  // holds N - 1 unknowns in shared memory, the back substitution owns 12
  // columns per thread); mixed path, N <= 8192 (the super-block tension solve
  // holds N - 1 unknowns in shared memory, the refinement's triangular solve
  // spreads 3N <= 24576 columns over a cluster of four CTAs)
  const int max_beads = (p->precision == BD_FP64) ? 4096 : 8192;
  for (int i = 0; i < p->n_chains; ++i)
    if (p->n_beads[i] < 2 || p->n_beads[i] > max_beads) return BD_ERR_ARG;
  return BD_OK;
}

// One context over all of p's chains (no lanes).
static int ctx_create(const bd_params* p, bd_ctx** out) {
  if (!out) return BD_ERR_ARG;
  *out = nullptr;
  if (int rc = validate_params(p)) return rc;
  const double a = p->a > 0.0 ? p->a : p->h_star;

  bd_ctx* c = new (std::nothrow) bd_ctx();
  if (!c) return BD_ERR_OOM;
  cudaGetDevice(&c->device);
  c->p = *p;
  c->Nc.assign(p->n_beads, p->n_beads + p->n_chains);
  c->p.n_beads = c->Nc.data();
  c->n_chains = p->n_chains;
  c->mixed = p->precision != BD_FP64;
  c->tileM = c->mixed ? kMixedTile : kSimtTile;
  c->elem = c->mixed ? sizeof(float) : sizeof(double);

  Phys& ph = c->ph;
  ph.hstar = p->h_star;
  ph.a = a > 0.0 ? a : 1.0;
  ph.dt = p->dt;
  ph.sq2dt = sqrt(2.0 * p->dt);
  const double rate = p->Wi / (p->lambda > 0.0 ? p->lambda : 1.0);
  for (int q = 0; q < 9; ++q) ph.kappa[q] = 0.0;
  if (p->flow == BD_FLOW_UNIAXIAL) {
    ph.kappa[0] = rate;
    ph.kappa[4] = -0.5 * rate;
    ph.kappa[8] = -0.5 * rate;
  } else if (p->flow == BD_FLOW_SHEAR) {
    ph.kappa[1] = rate;
  }
  ph.tol = p->tol > 0.0 ? p->tol : 1e-13;
  ph.max_newton = p->max_newton > 0 ? p->max_newton : 50;
  ph.n_chains = c->n_chains;
  ph.kspring = p->constraint == BD_FRAENKEL ? p->k_spring : 0.0;
  c->fraenkel = p->constraint == BD_FRAENKEL;
  c->midpoint = !c->fraenkel && p->scheme == BD_SCHEME_MIDPOINT;
  if (const char* e = getenv("BD_STEP_DIRECT")) {
    const int v = atoi(e);
    c->direct_iters = v > 0 ? (v == 1 ? ph.max_newton + 2 : v) : 0;
  }
  // typical steps need 7-10 tension iterations: the first 8 are plain graph
  // nodes, the WHILE node runs the rest
  c->graph_unroll = ph.max_newton + 2 < 8 ? ph.max_newton + 2 : 8;
  if (const char* e = getenv("BD_GRAPH_UNROLL")) {
    const int v = atoi(e);
    c->graph_unroll = v < 0 ? 0 : (v > ph.max_newton + 2 ? ph.max_newton + 2 : v);
  }

  long long boff = 0, roff = 0, moff = 0, koff = 0, soff = 0, wrow = 0, swrow = 0, kwrow = 0;
  c->h_cd.resize(c->n_chains);
  for (int i = 0; i < c->n_chains; ++i) {
    ChainDesc& d = c->h_cd[i];
    memset(&d, 0, sizeof(d));
    d.N = c->Nc[i];
    d.n = 3 * d.N;
    d.np = (int)round_up(d.n, c->tileM);
    d.m = d.N - 1;
    d.mp = (int)round_up(d.m, 2 * kSimtTile);
    d.boff = boff;
    d.roff = roff;
    d.moff = moff;
    d.koff = koff;
    d.soff = soff;
    d.wrow = (int)wrow;
    d.swrow = swrow;
    d.kwrow = kwrow;
    const long long tsn = ceil_div(d.n, kSymvTile), tsn2 = ceil_div(d.n, 2 * kSymvTile);
    const long long sneed = tsn * tsn * kSymvTile > tsn2 * tsn2 * 2 * kSymvTile
                                ? tsn * tsn * kSymvTile
                                : tsn2 * tsn2 * 2 * kSymvTile;
    boff += d.N;
    roff += d.m;
    moff += (long long)d.np * d.np;
    koff += (long long)d.mp * d.mp;
    soff += sneed;
    wrow += d.np;
    swrow += d.np;
    kwrow += d.mp;
    c->max_N = d.N > c->max_N ? d.N : c->max_N;
    c->max_n = d.n > c->max_n ? d.n : c->max_n;
    c->max_np = d.np > c->max_np ? d.np : c->max_np;
    c->max_m = d.m > c->max_m ? d.m : c->max_m;
    c->max_mp = d.mp > c->max_mp ? d.mp : c->max_mp;
  }
  c->total_beads = boff;
  c->total_rods = roff;
  c->M_elems = (size_t)moff;
  c->K_elems = (size_t)koff;

  auto alloc = [&](void** ptr, size_t bytes) -> bool {
    if (cudaMalloc(ptr, bytes < 16 ? 16 : bytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  };
  const size_t b3 = (size_t)boff * 3 * sizeof(double);
  const size_t rr = (size_t)(roff > 0 ? roff : 1) * sizeof(double);
  bool ok = alloc((void**)&c->d_cd, sizeof(ChainDesc) * c->n_chains) &&
            alloc(&c->M, c->M_elems * c->elem) && alloc(&c->K, c->K_elems * c->elem) &&
            alloc((void**)&c->r, b3) && alloc((void**)&c->rstar, b3) && alloc((void**)&c->rT, b3) &&
            alloc((void**)&c->y, b3) && alloc((void**)&c->u, b3) && alloc((void**)&c->F, b3) &&
            alloc((void**)&c->uhat, 3 * rr) && alloc((void**)&c->T, rr) && alloc((void**)&c->rhs, rr) &&
            alloc((void**)&c->scratch, (size_t)(soff > 0 ? soff : 1) * sizeof(double)) &&
            alloc((void**)&c->obs, (size_t)c->n_chains * BD_OBS_STRIDE * sizeof(double)) &&
            alloc((void**)&c->status, sizeof(int) * c->n_chains) &&
            alloc((void**)&c->state, sizeof(int) * c->n_chains) &&
            alloc((void**)&c->iters, sizeof(int) * c->n_chains) &&
            alloc((void**)&c->accurate, sizeof(int) * c->n_chains) &&
            alloc((void**)&c->args, sizeof(StepArgs)) &&
            alloc((void**)&c->loops, sizeof(unsigned long long));
  ok = ok && alloc(&c->Kinv, (size_t)kwrow * 64 * c->elem) &&
       (c->mixed || alloc(&c->Minv, (size_t)swrow * kSimtTile * c->elem));
  if (ok && c->mixed)
    ok = alloc((void**)&c->Winv, (size_t)wrow * kMixedTile * sizeof(float)) &&
         alloc((void**)&c->fsplit, (size_t)swrow * sizeof(float2)) &&
         alloc((void**)&c->dT, rr) && alloc((void**)&c->G, 3 * c->K_elems * sizeof(float)) &&
         alloc((void**)&c->Vsb, (size_t)kwrow * 256 * sizeof(float)) &&
         alloc((void**)&c->M16, c->M_elems * sizeof(__half)) &&
         alloc((void**)&c->tmaps, sizeof(CUtensorMap) * (2 * c->n_chains + 1)) &&
         alloc((void**)&c->kmaps, sizeof(CUtensorMap) * c->n_chains);
  if (ok && c->midpoint)
    ok = alloc((void**)&c->rmid, b3) && alloc((void**)&c->umid, 3 * rr) &&
         (c->mixed || alloc(&c->M2, c->M_elems * sizeof(double)));
  if (!ok) {
    ctx_destroy(c);
    return BD_ERR_OOM;
  }
  auto fail = [&](int code) {
    ctx_destroy(c);
    return code;
  };
  // Stream priorities: the factorisation's latency-bound chain (main and
  // chain-group streams) and the refinement's triangular solve go first; the
  // rod-coupling matrix K, needed only after the Brownian displacement, is
  // built at the lowest priority so that its bulk kernels fill idle SMs
  // instead of delaying the diagonal tiles.
  int pr_low = 0, pr_high = 0;
  if (cudaDeviceGetStreamPriorityRange(&pr_low, &pr_high) != cudaSuccess) pr_low = pr_high = 0;
  c->pr_high = pr_high;
  c->pr_low = pr_low;
  if (cudaStreamCreateWithPriority(&c->cs, cudaStreamNonBlocking, pr_high) != cudaSuccess ||
      cudaStreamCreateWithPriority(&c->cs2, cudaStreamNonBlocking, pr_high) != cudaSuccess ||
      cudaStreamCreateWithPriority(&c->aux[0], cudaStreamNonBlocking, pr_low) != cudaSuccess ||
      cudaStreamCreateWithPriority(&c->aux[1], cudaStreamNonBlocking, pr_high) != cudaSuccess ||
      cudaStreamCreateWithPriority(&c->aux[2], cudaStreamNonBlocking, pr_high) != cudaSuccess)
    return fail(BD_ERR_CUDA);
  for (int g = 0; g < 7; ++g)
    if (cudaEventCreateWithFlags(&c->aev[g], cudaEventDisableTiming) != cudaSuccess)
      return fail(BD_ERR_CUDA);
  cudaStream_t s = c->cs;
  if (c->mixed) {
    set_groups(c, c->n_chains / 16);
    for (int g = 0; g < bd_ctx::kMaxGroups; ++g)
      if (cudaStreamCreateWithPriority(&c->gs[g], cudaStreamNonBlocking, c->pr_high) != cudaSuccess)
        return fail(BD_ERR_CUDA);
    for (int g = 0; g <= bd_ctx::kMaxGroups; ++g)
      if (cudaEventCreateWithFlags(&c->gev[g], cudaEventDisableTiming) != cudaSuccess)
        return fail(BD_ERR_CUDA);
    std::vector<CUtensorMap> hm(2 * c->n_chains + 1);
    if (!make_tc_maps(hm.data(), (float*)c->M, c->Winv, c->M16, c->h_cd.data(), c->n_chains))
      return fail(BD_ERR_CUDA);
    if (cudaMemcpy(c->tmaps, hm.data(), sizeof(CUtensorMap) * hm.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        tc_configure() != cudaSuccess)
      return fail(BD_ERR_CUDA);
    std::vector<CUtensorMap> km(c->n_chains);
    if (!make_k_maps(km.data(), (float*)c->K, c->h_cd.data(), c->n_chains) ||
        cudaMemcpy(c->kmaps, km.data(), sizeof(CUtensorMap) * km.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(BD_ERR_CUDA);
  }
  // The fused step takes FP64 rigid-rod batches of short chains (BD_SMALL_STEP=0
  // keeps them on the multi-kernel step, for comparisons).
  c->small = !c->mixed && !c->fraenkel && c->max_N <= kSmallMaxN;
  if (const char* e = getenv("BD_SMALL_STEP"))
    if (atoi(e) == 0) c->small = false;
  if (c->small && small_configure(c->max_N) != cudaSuccess) return fail(BD_ERR_CUDA);
  if (matvec_configure() != cudaSuccess || tension_configure() != cudaSuccess ||
      assemble_configure() != cudaSuccess || refine_configure() != cudaSuccess ||
      k64_configure() != cudaSuccess || gmode_configure() != cudaSuccess ||
      solve_sb_configure() != cudaSuccess || midpoint_configure() != cudaSuccess ||
      tangent_configure() != cudaSuccess)
    return fail(BD_ERR_CUDA);
  if (cudaMemcpyAsync(c->d_cd, c->h_cd.data(), sizeof(ChainDesc) * c->n_chains,
                      cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(c->M, 0, c->M_elems * c->elem, s) != cudaSuccess ||
      cudaMemsetAsync(c->K, 0, c->K_elems * c->elem, s) != cudaSuccess ||
      cudaMemsetAsync(c->status, 0, sizeof(int) * c->n_chains, s) != cudaSuccess ||
      cudaMemsetAsync(c->iters, 0, sizeof(int) * c->n_chains, s) != cudaSuccess ||
      cudaMemsetAsync(c->T, 0, rr, s) != cudaSuccess ||
      cudaMemsetAsync(c->args, 0, sizeof(StepArgs), s) != cudaSuccess ||
      cudaMemsetAsync(c->loops, 0, sizeof(unsigned long long), s) != cudaSuccess)
    return fail(BD_ERR_CUDA);
  cudaError_t e1, e2;
  if (c->mixed) {
    e1 = launch_fill_identity_border<float>((float*)c->M, c->d_cd, c->n_chains, c->max_np, false, s);
    e2 = launch_fill_identity_border<float>((float*)c->K, c->d_cd, c->n_chains, c->max_mp, true, s);
    if (e1 == cudaSuccess) e1 = cudaMemsetAsync(c->G, 0, 3 * c->K_elems * sizeof(float), s);
    if (e1 == cudaSuccess) e1 = cudaMemsetAsync(c->Vsb, 0, (size_t)kwrow * 256 * sizeof(float), s);
  } else {
    e1 = launch_fill_identity_border<double>((double*)c->M, c->d_cd, c->n_chains, c->max_np, false, s);
    e2 = launch_fill_identity_border<double>((double*)c->K, c->d_cd, c->n_chains, c->max_mp, true, s);
    if (c->M2 && e1 == cudaSuccess) e1 = cudaMemsetAsync(c->M2, 0, c->M_elems * sizeof(double), s);
    if (c->M2 && e1 == cudaSuccess)
      e1 = launch_fill_identity_border<double>((double*)c->M2, c->d_cd, c->n_chains, c->max_np, false, s);
  }
  if (e1 != cudaSuccess || e2 != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
    return fail(BD_ERR_CUDA);
  *out = c;
  return BD_OK;
}

static int ctx_set_state(bd_ctx* c, const double* r_dev, void* stream) {
  if (!c || !r_dev) return BD_ERR_ARG;
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(c->r, r_dev, (size_t)c->total_beads * 3 * sizeof(double),
                     cudaMemcpyDefault, s));
  CK(cudaMemsetAsync(c->status, 0, sizeof(int) * c->n_chains, s));
  CK(cudaMemsetAsync(c->iters, 0, sizeof(int) * c->n_chains, s));
  CK(cudaMemsetAsync(c->T, 0, (size_t)(c->total_rods > 0 ? c->total_rods : 1) * sizeof(double), s));
  c->have_state = true;
  return BD_OK;
}

static int ctx_get_state(bd_ctx* c, double* r_dev, void* stream) {
  if (!c || !r_dev) return BD_ERR_ARG;
  if (!c->have_state) return BD_ERR_STATE;
  DeviceGuard g(c->device);
  CK(cudaMemcpyAsync(r_dev, c->r, (size_t)c->total_beads * 3 * sizeof(double), cudaMemcpyDefault,
                     (cudaStream_t)stream));
  return BD_OK;
}

// Runs n_steps on the context's stream c->cs once `start` has completed and
// records c->aev[5] at their end; nz: the noise of the context's first bead
// in step 0, step k at nz + k stride.  The caller holds c->mu.
static int launch_steps_locked(bd_ctx* c, int n_steps, const double* nz, long long stride, cudaEvent_t start) {
  int rc = (c->direct_iters > 0 || c->small) ? BD_OK : build_step_graph(c);
  if (rc) return rc;
  cudaStream_t cs = c->cs;
  CK(cudaStreamWaitEvent(cs, start, 0));
  if (c->small && c->direct_iters == 0) {
    // short FP64 chains: the fused step, all n_steps in one launch
    CK(launch_step_small(c->r, c->T, c->status, c->iters, c->state, c->d_cd, c->n_chains, c->max_N, c->ph, nz,
                         stride, n_steps, c->midpoint, cs));
    c->small_launches += 1;
    c->steps_launched += (unsigned long long)n_steps;
  } else {
    CK(launch_set_args(c->args, nz, stride, n_steps, cs));
    if (c->direct_iters > 0) {
      for (int i = 0; i < n_steps; ++i)
        if ((rc = enqueue_step_direct(c, cs))) return rc;
    } else {
      CK(cudaGraphLaunch(c->exec, cs));  // all n_steps steps in one launch
      c->steps_launched += (unsigned long long)n_steps;
    }
  }
  CK(cudaEventRecord(c->aev[5], cs));
  return BD_OK;
}

// Copies host-memory noise of n_steps steps to the context's staging buffer
// on stream s; *nz receives the device address to read.
static int stage_noise(bd_ctx* c, int n_steps, const double* noise, cudaStream_t s, const double** nz) {
  const long long stride = c->total_beads * 3;
  *nz = noise;
  if (is_device_ptr(noise)) return BD_OK;
  if (int rc = ensure_stage(c, (size_t)stride * n_steps)) return rc;
  CK(cudaMemcpyAsync(c->stage, noise, (size_t)stride * n_steps * sizeof(double), cudaMemcpyHostToDevice, s));
  *nz = c->stage;
  return BD_OK;
}

static int ctx_step(bd_ctx* c, int n_steps, const double* noise, void* stream) {
  if (!c || n_steps < 1 || !noise) return BD_ERR_ARG;
  if (!c->have_state) return BD_ERR_STATE;
  DeviceGuard g(c->device);
  std::lock_guard<std::mutex> lk(c->mu);
  cudaStream_t s = (cudaStream_t)stream;
  const double* nz = nullptr;
  if (int rc = stage_noise(c, n_steps, noise, s, &nz)) return rc;
  // The steps run on the context's highest-priority stream, ordered after the
  // caller's work on `stream` and before the caller's later work on it (a
  // default-priority caller stream would share the lowest priority with the
  // K chain and lose the factorisation's precedence over it).
  CK(cudaEventRecord(c->aev[4], s));
  if (int rc = launch_steps_locked(c, n_steps, nz, c->total_beads * 3, c->aev[4])) return rc;
  CK(cudaStreamWaitEvent(s, c->aev[5], 0));
  return BD_OK;
}

static int ctx_profile_step(bd_ctx* c, const double* noise, int newton_iters, double* ms_out) {
  if (!c || !noise || !ms_out || !is_device_ptr(noise)) return BD_ERR_ARG;
  if (!c->have_state) return BD_ERR_STATE;
  DeviceGuard g(c->device);
  std::lock_guard<std::mutex> lk(c->mu);
  cudaStream_t s = c->cs;
  cudaEvent_t ev[8];
  int made = 0;
  for (; made < 8; ++made)
    if (cudaEventCreate(&ev[made]) != cudaSuccess) break;
  int rc = BD_OK;
  const int saved = c->direct_iters;
  if (made < 8) {
    rc = BD_ERR_CUDA;
  } else {
    c->prof = ev;
    c->direct_iters = newton_iters > 0 ? newton_iters : c->ph.max_newton + 2;
    const long long stride = c->total_beads * 3;
    if (launch_set_args(c->args, noise, stride, 1, s) != cudaSuccess) rc = BD_ERR_CUDA;
    if (rc == BD_OK) rc = enqueue_step_direct(c, s);
    if (rc == BD_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = BD_ERR_CUDA;
    c->prof = nullptr;
    c->direct_iters = saved;
    if (rc == BD_OK) {
      float t;
      const int seg[7][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 4}, {4, 5}, {5, 6}, {0, 6}};
      for (int k = 0; k < 7; ++k) {
        if (cudaEventElapsedTime(&t, ev[seg[k][0]], ev[seg[k][1]]) != cudaSuccess) rc = BD_ERR_CUDA;
        ms_out[k] = t;
      }
      if (cudaEventElapsedTime(&t, ev[0], ev[7]) != cudaSuccess) rc = BD_ERR_CUDA;
      ms_out[7] = t;
    }
  }
  for (int k = 0; k < made; ++k) cudaEventDestroy(ev[k]);
  return rc;
}

static int ctx_kernel_launches(bd_ctx* c, unsigned long long* out, void* stream) {
  if (!c || !out) return BD_ERR_ARG;
  DeviceGuard g(c->device);
  unsigned long long loops = 0;
  CK(cudaMemcpyAsync(&loops, c->loops, sizeof(loops), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  // set_args launches once per bd_step call; it is not counted here
  *out = c->small ? c->small_launches
                  : c->steps_launched * (unsigned long long)c->graph_kernels +
                        loops * (unsigned long long)c->body_kernels;
  return BD_OK;
}

static int ctx_observables(bd_ctx* c, double* obs, int* status_host, void* stream) {
  if (!c) return BD_ERR_ARG;
  if (!c->have_state) return BD_ERR_STATE;
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  CK(launch_observables(c->r, c->d_cd, c->n_chains, c->iters, c->T, c->obs, s));
  if (obs)
    CK(cudaMemcpyAsync(obs, c->obs, (size_t)c->n_chains * BD_OBS_STRIDE * sizeof(double),
                       cudaMemcpyDefault, s));
  if (status_host) {
    CK(cudaMemcpyAsync(status_host, c->status, sizeof(int) * c->n_chains, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return worst(status_host, c->n_chains);
  }
  return BD_OK;
}

static int ctx_chain_status(bd_ctx* c, int* status_host, int* newton_host, void* stream) {
  if (!c) return BD_ERR_ARG;
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int> st(c->n_chains);
  CK(cudaMemcpyAsync(st.data(), c->status, sizeof(int) * c->n_chains, cudaMemcpyDeviceToHost, s));
  if (newton_host)
    CK(cudaMemcpyAsync(newton_host, c->iters, sizeof(int) * c->n_chains, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (status_host) memcpy(status_host, st.data(), sizeof(int) * c->n_chains);
  return worst(st.data(), c->n_chains);
}

static int ctx_assemble(bd_ctx* c, void* stream) {
  if (!c) return BD_ERR_ARG;
  if (!c->have_state) return BD_ERR_STATE;
  DeviceGuard g(c->device);
  return enqueue_assemble(c, (cudaStream_t)stream);
}

static int ctx_factor(bd_ctx* c, void* stream) {
  if (!c) return BD_ERR_ARG;
  DeviceGuard g(c->device);
  return enqueue_factor(c, (cudaStream_t)stream);
}

static int ctx_brownian(bd_ctx* c, const double* xi_dev, double* y_dev, void* stream) {
  if (!c || !xi_dev || !y_dev) return BD_ERR_ARG;
  DeviceGuard g(c->device);
  return enqueue_brownian(c, xi_dev, nullptr, y_dev, (cudaStream_t)stream);
}

static int ctx_mobility_apply(bd_ctx* c, const double* f_dev, double* u_dev, void* stream) {
  if (!c || !f_dev || !u_dev) return BD_ERR_ARG;
  DeviceGuard g(c->device);
  return enqueue_symv(c, c->M, f_dev, u_dev, nullptr, (cudaStream_t)stream);
}

static int ctx_get_tensions(bd_ctx* c, double* T_dev, void* stream) {
  if (!c || !T_dev) return BD_ERR_ARG;
  DeviceGuard g(c->device);
  if (c->total_rods > 0)
    CK(cudaMemcpyAsync(T_dev, c->T, (size_t)c->total_rods * sizeof(double), cudaMemcpyDefault,
                       (cudaStream_t)stream));
  return BD_OK;
}

static int ctx_midpoint(bd_ctx* c, const double* xi_dev, double* rmid_dev, double* y_dev, void* stream) {
  if (!c || !xi_dev || !rmid_dev || !y_dev || !c->midpoint) return BD_ERR_ARG;
  if (!c->have_state) return BD_ERR_STATE;
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (c->mixed) {
    const bool refine = c->p.refine != 0;
    CK(launch_brownian_f32_begin((const float*)c->M, c->Winv, c->d_cd, c->n_chains, c->max_np, xi_dev, nullptr,
                                 c->ph.sq2dt, refine, c->y, c->rT, c->F, c->scratch, s, c->aux[1], c->aev + 2,
                                 true));
    CK(launch_tangent_midpoint(c->r, refine ? c->rT : c->y, nullptr, refine ? c->ph.sq2dt : 1.0, c->d_cd,
                               c->n_chains, c->status, c->rmid, c->umid, s));
    CK(launch_brownian_f32_end((const float*)c->M, c->d_cd, c->n_chains, c->max_np, c->ph.sq2dt, refine, c->y,
                               c->rT, c->F, c->u, c->scratch, c->fsplit, s, c->aev + 2, true));
    CK(launch_mob_delta_f32(c->r, c->rmid, c->F, c->d_cd, c->n_chains, c->max_N, c->status, c->ph.hstar,
                            c->ph.a, c->ph.sq2dt, c->y, s));
  } else {
    CK(launch_trmv<double>((const double*)c->M, c->d_cd, c->n_chains, c->max_n, xi_dev, nullptr, c->ph.sq2dt,
                           c->y, s));
    CK(launch_trsv_t_f64((const double*)c->M, (const double*)c->Minv, c->d_cd, c->n_chains, c->max_n, xi_dev,
                         nullptr, c->ph.sq2dt, c->F, s));
    CK(launch_tangent_midpoint(c->r, c->y, nullptr, 1.0, c->d_cd, c->n_chains, c->status, c->rmid, c->umid, s));
    CK(launch_assemble<double>(c->rmid, (double*)c->M2, c->d_cd, c->n_chains, c->max_N, c->max_np,
                               c->ph.hstar, c->ph.a, nullptr, s));
    int rc = enqueue_symv(c, c->M2, c->F, c->y, nullptr, s);
    if (rc) return rc;
  }
  const size_t b3 = (size_t)c->total_beads * 3 * sizeof(double);
  CK(cudaMemcpyAsync(rmid_dev, c->rmid, b3, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(y_dev, c->y, b3, cudaMemcpyDeviceToDevice, s));
  return BD_OK;
}

// noise of step k at noise_dev + k noise_stride (the context's own 3 sum N,
// or a parent's when the context is a lane)
// Enqueues the n_steps primal steps and their tangents on `stream`
// (adjoint_finish forms the gradient).
static int adjoint_enqueue(bd_ctx* c, const double* r0_dev, int n_steps, const double* noise_dev,
                           long long noise_stride, void* stream) {
  if (!c || !r0_dev || !noise_dev || n_steps < 1) return BD_ERR_ARG;
  if (c->mixed || c->fraenkel || !(c->ph.hstar > 0.0)) return BD_ERR_ARG;
  DeviceGuard g(c->device);
  std::lock_guard<std::mutex> lk(c->mu);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t b3 = (size_t)c->total_beads * 3;
  const size_t nr = (size_t)(c->total_rods > 0 ? c->total_rods : 1);
  if (!c->Md) {
    auto al = [&](double** p, size_t n) {
      if (cudaMalloc(p, (n < 2 ? 2 : n) * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return false;
      }
      return true;
    };
    if (!(al(&c->Md, c->M_elems) && al(&c->rdot, 2 * b3) && al(&c->ydot, b3) && al(&c->rsdot, b3) &&
          al(&c->Gt, b3) && al(&c->abase, b3) && al(&c->zt, b3) && al(&c->DdF, b3) && al(&c->DG, b3) &&
          al(&c->vt, b3) && al(&c->Tdot, nr) && al(&c->Fdot, b3) && al(&c->rscale, c->n_chains) &&
          al(&c->kdot, 18)))
      return BD_ERR_OOM;
    if (c->midpoint && !(al(&c->yB, b3) && al(&c->zsv, b3) && al(&c->rmdot, b3) && al(&c->v2, b3) &&
                         al(&c->zdot, b3)))
      return BD_ERR_OOM;
    CK(cudaMemsetAsync(c->Md, 0, c->M_elems * sizeof(double), s));
  }
  // d kappa / d Wi = kappa at rate 1 / lambda; d kappa / d h* = 0
  double kd[18] = {0};
  const double lam = c->p.lambda > 0.0 ? c->p.lambda : 1.0;
  if (c->p.flow == BD_FLOW_UNIAXIAL) {
    kd[0] = 1.0 / lam;
    kd[4] = -0.5 / lam;
    kd[8] = -0.5 / lam;
  } else if (c->p.flow == BD_FLOW_SHEAR) {
    kd[1] = 1.0 / lam;
  }
  CK(cudaMemcpyAsync(c->kdot, kd, sizeof(kd), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->r, r0_dev, b3 * sizeof(double), cudaMemcpyDefault, s));
  CK(cudaMemsetAsync(c->status, 0, sizeof(int) * c->n_chains, s));
  CK(cudaMemsetAsync(c->rdot, 0, 2 * b3 * sizeof(double), s));
  c->have_state = true;
  const bool tied = !(c->p.a > 0.0);  // a = h*: a moves with h*
  const int tiles = c->max_np / kSimtTile;
  const int iters_max = c->ph.max_newton + 2;
  int rc;
  const bool mid = c->midpoint;
  // the mobility, rod directions and their positions the tension solve uses
  const void* Mt = mid ? c->M2 : c->M;
  const double* udir = mid ? c->umid : c->uhat;
  const size_t b3b = b3 * sizeof(double);
  for (int step = 0; step < n_steps; ++step) {
    const double* xi = noise_dev + (size_t)step * (size_t)noise_stride;
    // ---- primal step, intermediates kept (r still holds the old positions)
    if ((rc = enqueue_assemble(c, s))) return rc;
    if ((rc = enqueue_factor(c, s))) return rc;
    CK(launch_trmv<double>((const double*)c->M, c->d_cd, c->n_chains, c->max_n, xi, nullptr, c->ph.sq2dt,
                           c->y, s));
    if (mid) {
      CK(cudaMemcpyAsync(c->yB, c->y, b3b, cudaMemcpyDeviceToDevice, s));
      CK(launch_trsv_t_f64((const double*)c->M, (const double*)c->Minv, c->d_cd, c->n_chains, c->max_n, xi,
                           nullptr, c->ph.sq2dt, c->zsv, s));
      CK(launch_tangent_midpoint(c->r, c->yB, nullptr, 1.0, c->d_cd, c->n_chains, c->status, c->rmid, c->umid,
                                 s));
      CK(launch_assemble<double>(c->rmid, (double*)c->M2, c->d_cd, c->n_chains, c->max_N, c->max_np,
                                 c->ph.hstar, c->ph.a, nullptr, s));
      CK(launch_form_k<double>((const double*)c->M2, (double*)c->K, c->d_cd, c->n_chains, c->max_m, c->umid, s));
      if ((rc = enqueue_symv(c, c->M2, c->zsv, c->y, nullptr, s))) return rc;
    } else {
      CK(launch_rod_dirs(c->r, c->d_cd, c->n_chains, c->max_N, c->uhat, s));
      CK(launch_form_k<double>((const double*)c->M, (double*)c->K, c->d_cd, c->n_chains, c->max_m,
                               c->uhat, s));
    }
    CK(launch_chol_simt<double>((double*)c->K, (double*)c->Kinv, c->d_cd, c->n_chains,
                                c->max_mp / kSimtTile, true, c->status, s));
    CK(launch_predictor(c->r, c->y, c->d_cd, c->n_chains, c->max_N, c->ph, c->rstar, udir, c->T,
                        c->F, c->state, c->status, c->iters, nullptr, s));
    for (int it = 0; it < iters_max; ++it) {
      if ((rc = enqueue_symv(c, Mt, c->F, c->u, c->state, s))) return rc;
      CK(launch_newton_residual(c->rstar, c->u, c->d_cd, c->n_chains, c->ph, c->rT, c->rhs, c->state,
                                c->status, c->iters, s));
      CK(launch_newton_solve<double>((const double*)c->K, (const double*)c->Kinv, c->d_cd, c->n_chains,
                                     c->ph, udir, c->rhs, c->T, c->F, c->state, c->iters, s));
    }
    // ---- tangents for p = Wi (0) and p = h* (1)
    for (int p = 0; p < 2; ++p) {
      double* rd = c->rdot + (size_t)p * b3;
      const double hdot = (p == 1) ? 1.0 : 0.0, adot = (p == 1 && tied) ? 1.0 : 0.0;
      // X = L^{-1} D' L^{-T} in Md; y' = s L Phi(X) xi
      CK(launch_assemble_dot(c->r, rd, c->d_cd, c->n_chains, c->max_N, c->Md, c->ph.hstar, c->ph.a, hdot,
                             adot, s));
      if (!mid) CK(launch_gemv_dense(c->Md, c->d_cd, c->n_chains, c->max_n, c->F, c->DdF, s));
      CK(launch_trsm_rhs((const double*)c->M, (const double*)c->Minv, c->d_cd, c->n_chains, tiles, c->Md,
                         s));
      CK(launch_transpose(c->d_cd, c->n_chains, tiles, c->Md, s));
      CK(launch_trsm_rhs((const double*)c->M, (const double*)c->Minv, c->d_cd, c->n_chains, tiles, c->Md,
                         s));
      CK(launch_phi_matvec(c->Md, c->d_cd, c->n_chains, c->max_n, xi, c->vt, s));
      CK(launch_trmv<double>((const double*)c->M, c->d_cd, c->n_chains, c->max_n, c->vt, nullptr,
                             c->ph.sq2dt, c->ydot, s));
      const double* rq = c->r;
      const double* rqd = rd;
      if (mid) {
        // (s z)' = -s L^{-T} Phi(X)^T xi; r_m'; D_m' in Md; noise part s (D_m' z + D_m z')
        CK(launch_phi_upper_matvec(c->Md, c->d_cd, c->n_chains, c->max_n, xi, c->v2, s));
        CK(launch_trsv_t_f64((const double*)c->M, (const double*)c->Minv, c->d_cd, c->n_chains, c->max_n,
                             c->v2, nullptr, -c->ph.sq2dt, c->zdot, s));
        CK(launch_tangent_midpoint_dot(c->r, rd, c->yB, c->ydot, c->d_cd, c->n_chains, c->status, c->rmdot, s));
        CK(launch_assemble_dot(c->rmid, c->rmdot, c->d_cd, c->n_chains, c->max_N, c->Md, c->ph.hstar, c->ph.a,
                               hdot, adot, s));
        CK(launch_gemv_dense(c->Md, c->d_cd, c->n_chains, c->max_n, c->F, c->DdF, s));
        CK(launch_gemv_dense(c->Md, c->d_cd, c->n_chains, c->max_n, c->zsv, c->vt, s));
        if ((rc = enqueue_symv(c, c->M2, c->zdot, c->DG, nullptr, s))) return rc;
        CK(launch_vec_add(c->d_cd, c->n_chains, c->max_n, c->vt, c->DG, c->ydot, s));
        rq = c->rmid;
        rqd = c->rmdot;
      }
      CK(launch_tangent_predictor(c->r, rd, rq, rqd, c->ydot, udir, c->T, c->d_cd, c->n_chains, c->max_N, c->ph,
                                  c->kdot + 9 * p, c->rsdot, c->Gt, s));
      if ((rc = enqueue_symv(c, Mt, c->Gt, c->DG, nullptr, s))) return rc;
      CK(launch_tangent_base(c->d_cd, c->n_chains, c->max_n, c->ph, c->rsdot, c->DdF, c->DG, c->abase, s));
      CK(launch_tangent_init(c->d_cd, c->n_chains, c->max_n, c->status, c->state, c->iters, c->Tdot,
                             c->Fdot, s));
      for (int it = 0; it < iters_max; ++it) {
        if ((rc = enqueue_symv(c, Mt, c->Fdot, c->u, c->state, s))) return rc;
        CK(launch_tangent_residual(c->abase, c->u, c->rT, c->d_cd, c->n_chains, c->ph, 1e-12, c->rscale,
                                   c->zt, c->rhs, c->state, c->status, c->iters, s));
        CK(launch_newton_solve<double>((const double*)c->K, (const double*)c->Kinv, c->d_cd, c->n_chains,
                                       c->ph, udir, c->rhs, c->Tdot, c->Fdot, c->state, c->iters, s));
      }
      CK(cudaMemcpyAsync(rd, c->zt, b3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    // ---- commit the primal step
    CK(launch_finalize(c->d_cd, c->n_chains, c->total_beads, c->rT, c->r, c->state, c->status, nullptr,
                       s));
  }
  return BD_OK;
}

// grad_host[p] = dJ/dr_final . r'_p for the context's chains, after
// adjoint_enqueue on the same stream; synchronises it and returns the most
// severe chain status.
static int adjoint_finish(bd_ctx* c, const double* dJdr_final_dev, double grad_host[2], void* stream) {
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t b3 = (size_t)c->total_beads * 3;
  std::vector<double> J(b3), rd(2 * b3);
  CK(cudaMemcpyAsync(J.data(), dJdr_final_dev, b3 * sizeof(double), cudaMemcpyDefault, s));
  CK(cudaMemcpyAsync(rd.data(), c->rdot, 2 * b3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  std::vector<int> st(c->n_chains);
  CK(cudaMemcpyAsync(st.data(), c->status, sizeof(int) * c->n_chains, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int p = 0; p < 2; ++p) {
    long double acc = 0.0L;
    for (size_t e = 0; e < b3; ++e) acc += (long double)J[e] * (long double)rd[(size_t)p * b3 + e];
    grad_host[p] = (double)acc;
  }
  return worst(st.data(), c->n_chains);
}

static int ctx_adjoint(bd_ctx* c, const double* r0_dev, int n_steps, const double* noise_dev, int ckpt_every,
                       const double* dJdr_final_dev, double grad_host[2], void* stream) {
  (void)ckpt_every;  // forward-mode tangents carry O(1) state: no checkpoints are needed
  if (!c || !dJdr_final_dev || !grad_host) return BD_ERR_ARG;
  if (int rc = adjoint_enqueue(c, r0_dev, n_steps, noise_dev, c->total_beads * 3, stream)) return rc;
  return adjoint_finish(c, dJdr_final_dev, grad_host, stream);
}

static int ctx_set_factor_config(bd_ctx* c, int panel, int groups) {
  if (!c || !c->mixed || panel < 1 || panel > 96 || groups < 1 || groups > bd_ctx::kMaxGroups)
    return BD_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  c->panel = panel;
  set_groups(c, groups);
  drop_graph(c);
  return BD_OK;
}

// Shapes bd_tune_factor tries: super-panel widths and chain-group counts.
static const int kTunePanels[7] = {2, 4, 6, 8, 12, 16, 24};
static const int kTuneGroups[6] = {1, 2, 4, 8, 12, 16};

static int ctx_tune_factor(bd_ctx* c, int* panel_out, int* groups_out, double* ms_out, void* stream) {
  if (!c || !c->mixed) return BD_ERR_ARG;
  if (!c->have_state) return BD_ERR_STATE;
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int* panels = kTunePanels;
  const int* groups = kTuneGroups;
  double best = 1e30;
  int bp = c->panel, bg = c->n_groups;
  int rc = BD_OK;
  for (int gi = 0; gi < 6 && rc == BD_OK; ++gi) {
    if (groups[gi] > c->n_chains) continue;
    for (int pi = 0; pi < 7 && rc == BD_OK; ++pi) {
      c->panel = panels[pi];
      set_groups(c, groups[gi]);
      float tot = 0.f;
      for (int rep = 0; rep < 3 && rc == BD_OK; ++rep) {  // first repetition warms up
        if ((rc = enqueue_assemble(c, s))) break;
        if (cudaEventRecord(e0, s) != cudaSuccess) rc = BD_ERR_CUDA;
        if (!rc) rc = enqueue_factor(c, s);
        if (!rc && cudaEventRecord(e1, s) != cudaSuccess) rc = BD_ERR_CUDA;
        if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = BD_ERR_CUDA;
        float ms = 0.f;
        if (!rc && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = BD_ERR_CUDA;
        if (rep > 0) tot += ms;
      }
      if (!rc && tot / 2 < best) {
        best = tot / 2;
        bp = panels[pi];
        bg = groups[gi];
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->panel = bp;
  set_groups(c, bg);
  drop_graph(c);
  if (rc) return rc;
  if (panel_out) *panel_out = bp;
  if (groups_out) *groups_out = bg;
  if (ms_out) *ms_out = best;
  return BD_OK;
}

static int ctx_read_matrix(bd_ctx* c, int chain, int which, double* out_host) {
  if (!c || !out_host || chain < 0 || chain >= c->n_chains || (which != 0 && which != 1))
    return BD_ERR_ARG;
  DeviceGuard g(c->device);
  const int n = c->h_cd[chain].n;
  double* tmp = nullptr;
  if (cudaMalloc(&tmp, (size_t)n * n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return BD_ERR_OOM;
  }
  cudaError_t e = c->mixed ? launch_extract<float>((const float*)c->M, c->d_cd, chain, which, tmp, 0)
                           : launch_extract<double>((const double*)c->M, c->d_cd, chain, which, tmp, 0);
  if (e == cudaSuccess) e = cudaMemcpy(out_host, tmp, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(tmp);
  return e == cudaSuccess ? BD_OK : BD_ERR_CUDA;
}

static int ctx_factor_residual(bd_ctx* c, int chain, double* rel_fro) {
  if (!c || !rel_fro || chain < 0 || chain >= c->n_chains) return BD_ERR_ARG;
  DeviceGuard g(c->device);
  double* acc = nullptr;
  if (cudaMalloc(&acc, 2 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return BD_ERR_OOM;
  }
  cudaMemset(acc, 0, 2 * sizeof(double));
  if (c->mixed)
    k_residual_fro<float><<<1024, 256>>>((const float*)c->M, c->d_cd, chain, acc);
  else
    k_residual_fro<double><<<1024, 256>>>((const double*)c->M, c->d_cd, chain, acc);
  double h[2] = {0, 0};
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(h, acc, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(acc);
  if (e != cudaSuccess) return BD_ERR_CUDA;
  *rel_fro = sqrt(h[0] / h[1]);
  return BD_OK;
}

// ------------------------------------------------------------ public entry points
// A context without lanes forwards every call to its ctx_ function.  A context
// with lanes forwards to each lane with the arrays offset to the lane's first
// chain, bead or rod; bd_step and the stage calls (assembly, factorisation,
// Brownian displacement, mobility product, midpoint) fork every lane from one
// event on the caller's stream and join them back onto it.

// Lane count: p->lanes if given.  Otherwise, mixed precision: 2 for at
// least 32 chains, or at least 4 chains one of which has 2000 beads or more
// (two concurrent half-batches overlap one half's latency-bound
// factorisation and per-chain solves with the other half's streaming
// products; measured faster at 64 and 32 chains of 1000 beads and 4 of 4000,
// slower at 16 of 1000, and slower with 3 or 4 lanes at 64), else 1.  FP64:
// one lane per 16 chains, at most 8 (measured faster with 4 lanes at 64
// chains of 1000 beads and with 8 at 128 uneven chains of 50-500 and at 256
// of 100), and 1 for rigid-rod batches of chains of at most kSmallMaxN beads,
// which one fused kernel steps.  Never more lanes than chains.
static int lane_count(const bd_params* p) {
  int max_N = 0;
  for (int i = 0; i < p->n_chains; ++i) max_N = p->n_beads[i] > max_N ? p->n_beads[i] : max_N;
  int L = p->lanes;
  if (L <= 0) {
    if (p->precision == BD_FP64)
      L = (p->constraint == BD_RIGID && max_N <= kSmallMaxN) ? 1 : p->n_chains / 16;
    else
      L = (p->n_chains >= 32 || (p->n_chains >= 4 && max_N >= 2000)) ? 2 : 1;
  }
  L = L < kMaxLanes ? L : kMaxLanes;
  L = L < p->n_chains ? L : p->n_chains;
  return L > 1 ? L : 1;
}

// First chain of each lane: contiguous ranges of about equal factorisation
// work (3 N)^3, each of at least one chain.
static std::vector<int> lane_split(const bd_params* p, int L) {
  std::vector<double> cum(p->n_chains + 1, 0.0);
  for (int i = 0; i < p->n_chains; ++i) {
    const double n = 3.0 * p->n_beads[i];
    cum[i + 1] = cum[i] + n * n * n;
  }
  std::vector<int> c0(L + 1, 0);
  c0[L] = p->n_chains;
  for (int l = 1; l < L; ++l) {
    const double target = cum[p->n_chains] * l / L;
    int i = c0[l - 1] + 1;
    while (i < p->n_chains - (L - l) && cum[i] < target) ++i;
    c0[l] = i;
  }
  return c0;
}

int bd_create(const bd_params* p, bd_ctx** out) {
  if (!out) return BD_ERR_ARG;
  *out = nullptr;
  if (int rc = validate_params(p)) return rc;
  const int L = lane_count(p);
  if (L <= 1) return ctx_create(p, out);
  bd_ctx* c = new (std::nothrow) bd_ctx();
  if (!c) return BD_ERR_OOM;
  cudaGetDevice(&c->device);
  c->p = *p;
  c->Nc.assign(p->n_beads, p->n_beads + p->n_chains);
  c->p.n_beads = c->Nc.data();
  c->n_chains = p->n_chains;
  c->mixed = p->precision != BD_FP64;
  c->lane_c0 = lane_split(p, L);
  long long b = 0, r = 0;
  for (int l = 0; l < L; ++l) {
    c->lane_b0.push_back(b);
    c->lane_r0.push_back(r);
    bd_params q = *p;
    q.n_chains = c->lane_c0[l + 1] - c->lane_c0[l];
    q.n_beads = c->Nc.data() + c->lane_c0[l];
    q.lanes = 1;
    bd_ctx* sub = nullptr;
    const int rc = ctx_create(&q, &sub);
    if (rc) {
      bd_destroy(c);
      return rc;
    }
    c->lanes.push_back(sub);
    for (int i = 0; i < q.n_chains; ++i) {
      b += q.n_beads[i];
      r += q.n_beads[i] - 1;
    }
  }
  c->total_beads = b;
  c->total_rods = r;
  if (cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    bd_destroy(c);
    return BD_ERR_CUDA;
  }
  *out = c;
  return BD_OK;
}

void bd_destroy(bd_ctx* c) {
  if (!c) return;
  if (c->lanes.empty()) return ctx_destroy(c);
  DeviceGuard g(c->device);
  for (bd_ctx* l : c->lanes) ctx_destroy(l);
  if (c->stage) cudaFree(c->stage);
  if (c->fork) cudaEventDestroy(c->fork);
  delete c;
}

// Lane holding chain `chain` (the chain's index within it in *local).
static bd_ctx* lane_of(bd_ctx* c, int chain, int* local) {
  int l = 0;
  while (l + 1 < (int)c->lanes.size() && chain >= c->lane_c0[l + 1]) ++l;
  *local = chain - c->lane_c0[l];
  return c->lanes[l];
}

static int more_severe(int w, int r) { return (r != BD_OK && (w == BD_OK || r < w)) ? r : w; }

}  // extern "C"

// Runs fn(lane, index, lane stream) for every lane concurrently: each lane's
// stream waits for the caller's earlier work on `stream`, and the caller's
// later work waits for every lane that was started.
template <typename F>
static int on_lanes(bd_ctx* c, void* stream, F&& fn) {
  DeviceGuard g(c->device);
  std::lock_guard<std::mutex> lk(c->mu);
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaEventRecord(c->fork, s));
  int rc = BD_OK;
  size_t started = 0;
  for (; started < c->lanes.size(); ++started) {
    bd_ctx* ln = c->lanes[started];
    if (cudaStreamWaitEvent(ln->cs, c->fork, 0) != cudaSuccess) {
      rc = BD_ERR_CUDA;
      break;
    }
    rc = fn(ln, started, (void*)ln->cs);
    if (cudaEventRecord(ln->aev[5], ln->cs) != cudaSuccess && rc == BD_OK) rc = BD_ERR_CUDA;
    if (rc) {
      ++started;
      break;
    }
  }
  for (size_t l = 0; l < started; ++l)
    if (cudaStreamWaitEvent(s, c->lanes[l]->aev[5], 0) != cudaSuccess && rc == BD_OK) rc = BD_ERR_CUDA;
  return rc;
}

extern "C" {

int bd_set_state(bd_ctx* c, const double* r_dev, void* stream) {
  if (!c || c->lanes.empty()) return ctx_set_state(c, r_dev, stream);
  if (!r_dev) return BD_ERR_ARG;
  for (size_t l = 0; l < c->lanes.size(); ++l)
    if (int rc = ctx_set_state(c->lanes[l], r_dev + 3 * c->lane_b0[l], stream)) return rc;
  c->have_state = true;
  return BD_OK;
}

int bd_get_state(bd_ctx* c, double* r_dev, void* stream) {
  if (!c || c->lanes.empty()) return ctx_get_state(c, r_dev, stream);
  if (!r_dev) return BD_ERR_ARG;
  for (size_t l = 0; l < c->lanes.size(); ++l)
    if (int rc = ctx_get_state(c->lanes[l], r_dev + 3 * c->lane_b0[l], stream)) return rc;
  return BD_OK;
}

int bd_step(bd_ctx* c, int n_steps, const double* noise, void* stream) {
  if (!c || c->lanes.empty()) return ctx_step(c, n_steps, noise, stream);
  if (n_steps < 1 || !noise) return BD_ERR_ARG;
  if (!c->have_state) return BD_ERR_STATE;
  DeviceGuard g(c->device);
  std::lock_guard<std::mutex> lk(c->mu);
  cudaStream_t s = (cudaStream_t)stream;
  const double* nz = nullptr;
  if (int rc = stage_noise(c, n_steps, noise, s, &nz)) return rc;
  CK(cudaEventRecord(c->fork, s));
  for (size_t l = 0; l < c->lanes.size(); ++l) {
    bd_ctx* ln = c->lanes[l];
    std::lock_guard<std::mutex> ll(ln->mu);
    if (int rc = launch_steps_locked(ln, n_steps, nz + 3 * c->lane_b0[l], c->total_beads * 3, c->fork)) return rc;
  }
  for (bd_ctx* ln : c->lanes) CK(cudaStreamWaitEvent(s, ln->aev[5], 0));
  return BD_OK;
}

int bd_profile_step(bd_ctx* c, const double* noise, int newton_iters, double* ms_out) {
  if (!c || c->lanes.empty()) return ctx_profile_step(c, noise, newton_iters, ms_out);
  if (!noise || !ms_out) return BD_ERR_ARG;
  for (int k = 0; k < 8; ++k) ms_out[k] = 0.0;
  for (size_t l = 0; l < c->lanes.size(); ++l) {  // lane after lane
    double ms[8];
    if (int rc = ctx_profile_step(c->lanes[l], noise + 3 * c->lane_b0[l], newton_iters, ms)) return rc;
    for (int k = 0; k < 8; ++k) ms_out[k] += ms[k];
  }
  return BD_OK;
}

int bd_kernel_launches(bd_ctx* c, unsigned long long* out, void* stream) {
  if (!c || c->lanes.empty()) return ctx_kernel_launches(c, out, stream);
  if (!out) return BD_ERR_ARG;
  unsigned long long tot = 0;
  for (bd_ctx* l : c->lanes) {
    unsigned long long v = 0;
    if (int rc = ctx_kernel_launches(l, &v, stream)) return rc;
    tot += v;
  }
  *out = tot;
  return BD_OK;
}

int bd_selftest_bounded_wait(int arrive, int* status_host) {
  if (!status_host) return BD_ERR_ARG;
  int* d = nullptr;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return BD_ERR_OOM;
  }
  cudaError_t e = cudaMemset(d, 0xff, sizeof(int));
  if (e == cudaSuccess) e = launch_wait_selftest(arrive != 0, d, 0);
  if (e == cudaSuccess) e = cudaMemcpy(status_host, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e == cudaSuccess ? BD_OK : BD_ERR_CUDA;
}

int bd_lanes(bd_ctx* c, int* out) {
  if (!c || !out) return BD_ERR_ARG;
  *out = c->lanes.empty() ? 1 : (int)c->lanes.size();
  return BD_OK;
}

int bd_observables(bd_ctx* c, double* obs, int* status_host, void* stream) {
  if (!c || c->lanes.empty()) return ctx_observables(c, obs, status_host, stream);
  if (!status_host)  // asynchronous: every lane's kernel and copy on its own stream
    return on_lanes(c, stream, [&](bd_ctx* l, size_t k, void* ls) {
      return ctx_observables(l, obs ? obs + (size_t)c->lane_c0[k] * BD_OBS_STRIDE : nullptr, nullptr, ls);
    });
  int w = BD_OK;
  for (size_t l = 0; l < c->lanes.size(); ++l) {
    const int c0 = c->lane_c0[l];
    w = more_severe(w, ctx_observables(c->lanes[l], obs ? obs + (size_t)c0 * BD_OBS_STRIDE : nullptr,
                                       status_host ? status_host + c0 : nullptr, stream));
  }
  return w;
}

int bd_chain_status(bd_ctx* c, int* status_host, int* newton_host, void* stream) {
  if (!c || c->lanes.empty()) return ctx_chain_status(c, status_host, newton_host, stream);
  int w = BD_OK;
  for (size_t l = 0; l < c->lanes.size(); ++l) {
    const int c0 = c->lane_c0[l];
    w = more_severe(w, ctx_chain_status(c->lanes[l], status_host ? status_host + c0 : nullptr,
                                        newton_host ? newton_host + c0 : nullptr, stream));
  }
  return w;
}

int bd_factor_residual(bd_ctx* c, int chain, double* rel_fro) {
  if (!c || c->lanes.empty()) return ctx_factor_residual(c, chain, rel_fro);
  if (chain < 0 || chain >= c->n_chains) return BD_ERR_ARG;
  int local = 0;
  bd_ctx* l = lane_of(c, chain, &local);
  return ctx_factor_residual(l, local, rel_fro);
}

int bd_read_matrix(bd_ctx* c, int chain, int which, double* out_host) {
  if (!c || c->lanes.empty()) return ctx_read_matrix(c, chain, which, out_host);
  if (chain < 0 || chain >= c->n_chains) return BD_ERR_ARG;
  int local = 0;
  bd_ctx* l = lane_of(c, chain, &local);
  return ctx_read_matrix(l, local, which, out_host);
}

int bd_assemble(bd_ctx* c, void* stream) {
  if (!c || c->lanes.empty()) return ctx_assemble(c, stream);
  return on_lanes(c, stream, [&](bd_ctx* l, size_t, void* ls) { return ctx_assemble(l, ls); });
}

int bd_factor(bd_ctx* c, void* stream) {
  if (!c || c->lanes.empty()) return ctx_factor(c, stream);
  return on_lanes(c, stream, [&](bd_ctx* l, size_t, void* ls) { return ctx_factor(l, ls); });
}

int bd_brownian(bd_ctx* c, const double* xi_dev, double* y_dev, void* stream) {
  if (!c || c->lanes.empty()) return ctx_brownian(c, xi_dev, y_dev, stream);
  if (!xi_dev || !y_dev) return BD_ERR_ARG;
  return on_lanes(c, stream, [&](bd_ctx* l, size_t k, void* ls) {
    const long long o = 3 * c->lane_b0[k];
    return ctx_brownian(l, xi_dev + o, y_dev + o, ls);
  });
}

int bd_mobility_apply(bd_ctx* c, const double* f_dev, double* u_dev, void* stream) {
  if (!c || c->lanes.empty()) return ctx_mobility_apply(c, f_dev, u_dev, stream);
  if (!f_dev || !u_dev) return BD_ERR_ARG;
  return on_lanes(c, stream, [&](bd_ctx* l, size_t k, void* ls) {
    const long long o = 3 * c->lane_b0[k];
    return ctx_mobility_apply(l, f_dev + o, u_dev + o, ls);
  });
}

int bd_get_tensions(bd_ctx* c, double* T_dev, void* stream) {
  if (!c || c->lanes.empty()) return ctx_get_tensions(c, T_dev, stream);
  if (!T_dev) return BD_ERR_ARG;
  for (size_t l = 0; l < c->lanes.size(); ++l)
    if (int rc = ctx_get_tensions(c->lanes[l], T_dev + c->lane_r0[l], stream)) return rc;
  return BD_OK;
}

int bd_midpoint(bd_ctx* c, const double* xi_dev, double* rmid_dev, double* y_dev, void* stream) {
  if (!c || c->lanes.empty()) return ctx_midpoint(c, xi_dev, rmid_dev, y_dev, stream);
  if (!xi_dev || !rmid_dev || !y_dev) return BD_ERR_ARG;
  return on_lanes(c, stream, [&](bd_ctx* l, size_t k, void* ls) {
    const long long o = 3 * c->lane_b0[k];
    return ctx_midpoint(l, xi_dev + o, rmid_dev + o, y_dev + o, ls);
  });
}

int bd_adjoint(bd_ctx* c, const double* r0_dev, int n_steps, const double* noise_dev, int ckpt_every,
               const double* dJdr_final_dev, double grad_host[2], void* stream) {
  if (!c || c->lanes.empty())
    return ctx_adjoint(c, r0_dev, n_steps, noise_dev, ckpt_every, dJdr_final_dev, grad_host, stream);
  if (!r0_dev || !noise_dev || !dJdr_final_dev || !grad_host || n_steps < 1) return BD_ERR_ARG;
  // J's gradient is a sum over chains: every lane contributes its chains'
  // part; the lanes' steps and tangents run concurrently on their streams,
  // each reading its beads of the caller's arrays
  DeviceGuard dg(c->device);
  std::lock_guard<std::mutex> lk(c->mu);
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaEventRecord(c->fork, s));
  for (size_t l = 0; l < c->lanes.size(); ++l) {
    bd_ctx* ln = c->lanes[l];
    const long long o = 3 * c->lane_b0[l];
    CK(cudaStreamWaitEvent(ln->cs, c->fork, 0));
    if (int rc = adjoint_enqueue(ln, r0_dev + o, n_steps, noise_dev + o, c->total_beads * 3, (void*)ln->cs)) {
      for (size_t k = 0; k <= l; ++k) cudaStreamSynchronize(c->lanes[k]->cs);
      return rc;
    }
  }
  int w = BD_OK;
  double g[2] = {0.0, 0.0};
  for (size_t l = 0; l < c->lanes.size(); ++l) {
    double gl[2] = {0.0, 0.0};
    const int rc = adjoint_finish(c->lanes[l], dJdr_final_dev + 3 * c->lane_b0[l], gl, (void*)c->lanes[l]->cs);
    if (rc == BD_ERR_CUDA) return rc;
    w = more_severe(w, rc);
    g[0] += gl[0];
    g[1] += gl[1];
  }
  grad_host[0] = g[0];
  grad_host[1] = g[1];
  c->have_state = true;
  return w;
}

int bd_set_factor_config(bd_ctx* c, int panel, int groups) {
  if (!c || c->lanes.empty()) return ctx_set_factor_config(c, panel, groups);
  for (bd_ctx* l : c->lanes)
    if (int rc = ctx_set_factor_config(l, panel, groups)) return rc;
  return BD_OK;
}

int bd_tune_factor(bd_ctx* c, int* panel_out, int* groups_out, double* ms_out, void* stream) {
  if (!c || c->lanes.empty()) return ctx_tune_factor(c, panel_out, groups_out, ms_out, stream);
  if (!c->have_state) return BD_ERR_STATE;
  // every shape is timed with all lanes factoring concurrently, as in the
  // step (measured a little faster than tuning each lane alone)
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  int min_chains = c->n_chains;
  for (bd_ctx* l : c->lanes) min_chains = l->n_chains < min_chains ? l->n_chains : min_chains;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return BD_ERR_CUDA;
  }
  double best = 1e30;
  int bp = 0, bg = 0;
  int rc = BD_OK;
  for (int gi = 0; gi < 6 && rc == BD_OK; ++gi) {
    if (kTuneGroups[gi] > min_chains) continue;
    for (int pi = 0; pi < 7 && rc == BD_OK; ++pi) {
      for (bd_ctx* l : c->lanes)
        if (!rc) rc = ctx_set_factor_config(l, kTunePanels[pi], kTuneGroups[gi]);
      float tot = 0.f;
      for (int rep = 0; rep < 3 && rc == BD_OK; ++rep) {  // first repetition warms up
        if ((rc = bd_assemble(c, stream))) break;
        if (cudaEventRecord(e0, s) != cudaSuccess) rc = BD_ERR_CUDA;
        if (!rc) rc = bd_factor(c, stream);
        if (!rc && cudaEventRecord(e1, s) != cudaSuccess) rc = BD_ERR_CUDA;
        if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = BD_ERR_CUDA;
        float ms = 0.f;
        if (!rc && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = BD_ERR_CUDA;
        if (rep > 0) tot += ms;
      }
      if (!rc && tot / 2 < best) {
        best = tot / 2;
        bp = kTunePanels[pi];
        bg = kTuneGroups[gi];
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  for (bd_ctx* l : c->lanes)
    if ((rc = ctx_set_factor_config(l, bp, bg))) return rc;
  if (panel_out) *panel_out = bp;
  if (groups_out) *groups_out = bg;
  if (ms_out) *ms_out = best;
  return BD_OK;
}

}  // extern "C"

