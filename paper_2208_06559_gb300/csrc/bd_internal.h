// bd_internal.h -- shared definitions of libbd's kernels and runtime.
//
// Data layout in HBM (one context = one batch of chains):
//   * positions r, noise, forces: packed FP64 [sum N][3];
//   * per chain c one square row-major matrix of order np_c (3 N_c rounded up
//     to the Cholesky tile) holding, after a step's factorisation, the factor
//     B = L in the lower triangle (diagonal included) and the diffusion tensor
//     D in the strict upper triangle.  D's diagonal is 1 (Sec. 3 Eq. (7)) and
//     is not stored.  Rows and columns past 3 N_c are an identity border, so
//     the padded matrix factors to diag(L, I);
//   * per chain a second square matrix of order mp_c (N_c - 1 rounded up to
//     64) for the rod-coupling matrix K = U^T C^T D C U and its factor;
//   * FP64 (BD_FP64) or FP32 (mixed) element type for both matrices.
#pragma once
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bd.h"

namespace bd {

// Per-chain descriptor (device resident, one per chain).
struct ChainDesc {
  int N;           // beads
  int n;           // 3N
  int np;          // padded order of the D/L matrix
  int m;           // rods N-1
  int mp;          // padded order of K
  int wrow;        // mixed: first row of this chain's diagonal-tile inverses in Winv
  long long boff;  // first bead in packed [sum N][3] arrays
  long long roff;  // first rod in packed [sum (N-1)] arrays
  long long moff;  // first element of the D/L matrix
  long long koff;  // first element of K
  long long soff;  // first element of the SYMV partial-sum scratch
  long long swrow; // FP64 path: first row of this chain's 32 x 32 diagonal-block inverses of L
  long long kwrow; // first row of this chain's 32 x 32 diagonal-block inverses of K's factor
};

enum NewtonState : int { NS_ACTIVE = 0, NS_EXTRA = 1, NS_DONE = 2, NS_FAILED = 3 };

// Physical parameters read by the kernels (passed by value).
struct Phys {
  double hstar, a, dt, sq2dt;
  double kappa[9];
  double tol;
  int max_newton;
  int n_chains;
  double kspring;  // Fraenkel spring constant K* (Fraenkel mode)
};

// Device-side step arguments (read by the captured step graph each replay).
struct StepArgs {
  const double* noise;  // [n_steps][sum N][3]
  long long stride;     // sum N * 3
  int step;             // step index within the current bd_step call
  int loops_in_step;    // tension-solve loop iterations in the current step
  int n_steps;          // steps of the current bd_step call
};

constexpr int kSimtTile = 32;     // SIMT Cholesky tile (FP64, FP32) and K tile
constexpr int kMixedTile = 128;   // tensor-core Cholesky tile (mixed precision)
constexpr int kSymvTile = 64;     // SYMV tile

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }
inline long long round_up(long long a, long long b) { return (a + b - 1) / b * b; }

// ---- kernel launchers (each enqueues on `s`; return cudaGetLastError) ----
template <typename T>
cudaError_t launch_fill_identity_border(T* M, const ChainDesc* cd, int n_chains,
                                        int max_np, bool k_matrix, cudaStream_t s);
// rsplit: [sum np] float2 scratch for the FP32 path's (hi, lo) positions
// (unused by the FP64 path).
template <typename T>
cudaError_t launch_assemble(const double* r, T* M, const ChainDesc* cd, int n_chains,
                            int max_N, int max_np, double hstar, double a, float2* rsplit,
                            cudaStream_t s);
// v (FP64, per chain 3N values at 3 boff) -> (hi, lo) float pairs at swrow, zero-padded to np.
cudaError_t launch_split_f2(const ChainDesc* cd, int n_chains, int max_np, const double* v,
                            float2* out, const int* state, cudaStream_t s);
template <typename T>
cudaError_t launch_chol_simt(T* M, T* Winv, const ChainDesc* cd, int n_chains, int max_tiles,
                             bool k_matrix, int* status, cudaStream_t s);
template <typename T>
cudaError_t launch_trmv(const T* M, const ChainDesc* cd, int n_chains, int max_n,
                        const double* x, const StepArgs* args, double scale, double* y,
                        cudaStream_t s);
template <typename T>
cudaError_t launch_symv(const T* M, const ChainDesc* cd, int n_chains, int max_np,
                        const double* f, double* scratch, double* u, const int* state,
                        cudaStream_t s);
// Per-chain mode of the mixed path's rod-space product inside the tension
// iteration (k_gmode.cu): the full product w = G T or the increment
// w += G dT, in plain FP32 or in compensated (double-float) FP32.
enum MobMode : int { MOB_FULL_F32 = 0, MOB_FULL_DF = 1, MOB_INC_DF = 2, MOB_INC_F32 = 3 };
// FP32-storage mobility product u = D f with FP32 arithmetic: groups of four
// products summed in FP32, the group sums added with a two-sum (relative
// error a few FP32 round-offs, independent of the length of the sum).
// fsplit: [sum np] float2; scratch: the two-phase partials.
cudaError_t launch_symv_f32(const float* M, const ChainDesc* cd, int n_chains, int max_np,
                            const double* f, float2* fsplit, double* scratch, double* u,
                            const int* state, cudaStream_t s);
// Mixed path: K (FP32) and G = C D C^T U (three planes [3][mp][mp] per chain
// at 3 koff) from the positions, without D (k_matvec.cu); either output may
// be NULL.
cudaError_t launch_form_k_pos(const double* r, float* K, float* G, const ChainDesc* cd, int n_chains,
                              int max_m, const double* u, double hstar, double a, cudaStream_t s);
template <typename T>
cudaError_t launch_form_k(const T* M, T* K, const ChainDesc* cd, int n_chains, int max_m,
                          const double* u, cudaStream_t s);

cudaError_t launch_rod_dirs(const double* r, const ChainDesc* cd, int n_chains, int max_N,
                            double* uhat, cudaStream_t s);
cudaError_t launch_predictor(const double* r, const double* y, const ChainDesc* cd,
                             int n_chains, int max_N, Phys ph, double* rstar,
                             const double* uhat, double* T, double* F, int* state,
                             const int* status, int* iters, int* accurate, cudaStream_t s);
cudaError_t launch_newton_residual(const double* rstar, const double* u, const ChainDesc* cd,
                                   int n_chains, Phys ph, double* rT, double* rhs,
                                   int* state, int* status, const int* iters, cudaStream_t s);
// FP64 path (32-wide blocks of K's factor and their inverses).
template <typename T>
cudaError_t launch_newton_solve(const T* K, const T* Kinv, const ChainDesc* cd, int n_chains, Phys ph,
                                const double* uhat, double* rhs, double* Tn, double* F,
                                int* state, int* iters, cudaStream_t s);
// Mixed path, tension solve with 256-wide super-blocks (k_solve_sb.cu): the
// inverses of the diagonal super-blocks of K's factor, V ([sum mp][256] FP32,
// chain offset kwrow * 256, zero above the diagonal), once per step; then the
// solve itself, T += delta, dT = delta (optional), F(T).
cudaError_t launch_sb_inverse(const float* K, const float* Kinv, float* V, const ChainDesc* cd, int n_chains,
                              int max_mp, cudaStream_t s);
cudaError_t launch_newton_solve_sb(const float* K, const float* V, const ChainDesc* cd, int n_chains, Phys ph,
                                   const double* uhat, const double* rhs, double* Tn, double* F, int* state,
                                   int* iters, double* dT, cudaStream_t s);
bool is_sb_inverse_kernel(const void* f);
cudaError_t solve_sb_configure();
// Rod-space tension iteration of the mixed path (k_gmode.cu).
cudaError_t launch_tension_products_g(const float* G, const ChainDesc* cd, int n_chains, int max_mp,
                                      const double* T, const double* dT, double* w, const int* state,
                                      const int* mode, cudaStream_t s);
cudaError_t launch_newton_residual_g(const double* rstar, const double* w, const ChainDesc* cd,
                                     int n_chains, Phys ph, double* rhs, int* state, int* status,
                                     const int* iters, int* mode, cudaStream_t s);
// rpos: the positions whose mobility moves bead 0 ((D F)_0 is evaluated from
// them in FP64): the start of the step, or the midpoint of the corrected step.
cudaError_t launch_finalize_g(const ChainDesc* cd, int n_chains, Phys ph, const double* rpos, const double* rstar,
                              const double* w, const double* F, double* r, const int* state, int* status,
                              StepArgs* args, cudaStream_t s);
cudaError_t gmode_configure();
cudaError_t launch_newton_any_active(const int* state, int n_chains,
                                     cudaGraphConditionalHandle h, unsigned long long* loops,
                                     StepArgs* args, int max_loops, bool count, cudaStream_t s);
cudaError_t launch_finalize(const ChainDesc* cd, int n_chains, long long total_beads,
                            const double* rT, double* r, const int* state, int* status,
                            StepArgs* args, cudaStream_t s);
cudaError_t launch_observables(const double* r, const ChainDesc* cd, int n_chains,
                               const int* iters, const double* T, double* obs, cudaStream_t s);
cudaError_t launch_set_args(StepArgs* args, const double* noise, long long stride, int n_steps,
                            cudaStream_t s);
// Ends one step of the step graph's WHILE loop: continue while steps remain.
cudaError_t launch_step_loop(const StepArgs* args, cudaGraphConditionalHandle h, cudaStream_t s);
// FP32 Cholesky of the rod-coupling matrix with 64-wide tiles (k_chol_k64.cu);
// mp must be a multiple of 64; the 64 x 64 diagonal-tile inverses go to Kinv.
cudaError_t k64_configure();
cudaError_t launch_chol_k64(float* K, float* Kinv, const CUtensorMap* kmaps, const ChainDesc* cd, int n_chains,
                            int max_tiles, int* status, cudaStream_t s);

// Opt-in shared-memory sizes of the matvec kernels (once per device).
cudaError_t matvec_configure();
cudaError_t assemble_configure();
cudaError_t tension_configure();
// Fraenkel-spring mode (k_fraenkel.cu).
cudaError_t launch_fraenkel_forces(const double* r, const ChainDesc* cd, int n_chains, int max_N,
                                   double kspring, double* F, cudaStream_t s);
cudaError_t launch_fraenkel_update(double* r, const double* y, const double* u, const ChainDesc* cd,
                                   int n_chains, Phys ph, double* T, const int* status, int* iters,
                                   cudaStream_t s);
cudaError_t launch_step_done(StepArgs* args, cudaStream_t s);
// Kernels of the rod-coupling-matrix chain (K formation and factorisation),
// for per-node priorities in the captured step graph.
bool is_kchain_form_kernel(const void* f);  // K (with or without G) from the positions
bool is_k64_kernel(const void* f);
const void* rod_dirs_kernel();
cudaError_t refine_configure();

// Mixed-precision Brownian displacement with one refinement step (k_refine.cu):
// y = s/2 (B xi + D B^{-T} xi); with refine == 0, y = s B xi.
// The triangular solve of the refinement runs on `s2` (forked from and joined
// back into `s` with events ev[0], ev[1]) concurrently with the product.
// need_z: leave z = B^{-T} xi (unscaled) in `z` also when refine == 0.
cudaError_t launch_brownian_f32(const float* M, const float* Winv, const ChainDesc* cd, int n_chains,
                                int max_np, const double* x, const StepArgs* args, double scale,
                                bool refine, double* y, double* y1, double* z, double* w,
                                double* scratch, float2* fsplit, cudaStream_t s, cudaStream_t s2,
                                cudaEvent_t* ev, bool need_z = false);
// The same in two parts.  begin: the noise split, the triangular solve forked
// to s2 (z = B^{-T} xi, unscaled, when refine or need_z), and the product
// B xi on s -- into y1 unscaled when refine, else into y scaled; end: the
// join, then (refine) the product D z and y = s/2 (y1 + D z).
cudaError_t launch_brownian_f32_begin(const float* M, const float* Winv, const ChainDesc* cd, int n_chains,
                                      int max_np, const double* x, const StepArgs* args, double scale,
                                      bool refine, double* y, double* y1, double* z, double* scratch,
                                      cudaStream_t s, cudaStream_t s2, cudaEvent_t* ev, bool need_z);
cudaError_t launch_brownian_f32_end(const float* M, const ChainDesc* cd, int n_chains, int max_np, double scale,
                                    bool refine, double* y, const double* y1, const double* z, double* w,
                                    double* scratch, float2* fsplit, cudaStream_t s, cudaEvent_t* ev,
                                    bool need_z);

// Midpoint corrector of the rigid-rod step (k_midpoint.cu).
// r_m = r + P y / 2 (P: orthogonal projection onto the tangent space of the
// rod constraints at r) into rmid, the unit rod directions of r_m into umid;
// y = yscale * y (or yscale * the step's noise when args != NULL).
cudaError_t launch_tangent_midpoint(const double* r, const double* y, const StepArgs* args, double yscale,
                                    const ChainDesc* cd, int n_chains, const int* status, double* rmid,
                                    double* umid, cudaStream_t s);
// z = scale L^{-T} xi for the FP64 factor (xi from x, or the step's noise when args != NULL).
cudaError_t launch_trsv_t_f64(const double* M, const double* Winv, const ChainDesc* cd, int n_chains,
                              int max_n, const double* x, const StepArgs* args, double scale, double* z,
                              cudaStream_t s);
// y += scale (D(rmid) - D(r)) z, from the positions in FP32 (mixed path).
cudaError_t launch_mob_delta_f32(const double* r, const double* rmid, const double* z, const ChainDesc* cd,
                                 int n_chains, int max_N, const int* status, double hstar, double a,
                                 double scale, double* y, cudaStream_t s);
cudaError_t midpoint_configure();

// The whole FP64 rigid-rod step of chains of at most kSmallMaxN beads, one
// CTA per chain with every matrix in shared memory, all n_steps steps in one
// launch (k_small.cu).
constexpr int kSmallMaxN = 32;
size_t small_smem_bytes(int max_N);
cudaError_t small_configure(int max_N);
cudaError_t launch_step_small(double* r, double* T, int* status, int* iters, int* state, const ChainDesc* cd,
                              int n_chains, int max_N, Phys ph, const double* noise, long long stride,
                              int n_steps, bool midpoint, cudaStream_t s);

// Mixed-precision tensor-core Cholesky (k_chol_tc.cu).
bool make_tc_maps(CUtensorMap* host_maps, float* M, float* Winv, __half* M16, const ChainDesc* h_cd,
                  int n_chains);
cudaError_t tc_configure();
// TMA maps of every chain's FP32 K, for the tensor-core update of K's factorisation.
bool make_k_maps(CUtensorMap* host_maps, float* K, const ChainDesc* h_cd, int n_chains);
// K_ij -= L_ik L_jk^T after K's 64-wide block column k, FP32-accurate on the
// tensor cores (split TF32 operands).
cudaError_t launch_kupdate_tc(const CUtensorMap* kmaps, const ChainDesc* cd, int n_chains, int max_mp, int k,
                              int* status, cudaStream_t s);
bool is_kupdate_tc_kernel(const void* f);
// One thread waits on an mbarrier that completes only if `arrive`; *out:
// BD_OK, or BD_ERR_TIMEOUT once the bounded wait gives up.
cudaError_t launch_wait_selftest(int arrive, int* out, cudaStream_t s);
// Factor chains [0, n_chains) of the given arrays (pointers may be offset to
// a chain subrange); wmap is the TMA map of Winv; maps16 map the FP16 copies
// of the off-diagonal L tiles (same layout as M), written by the panel
// solves and read by the trailing updates.
cudaError_t launch_chol_tc(float* M, float* Winv, const CUtensorMap* maps, const CUtensorMap* wmap,
                           const CUtensorMap* maps16, const ChainDesc* cd, int n_chains, int max_tiles,
                           int panel, int* status, cudaStream_t s);

// Forward-mode tangents of the FP64 step (k_tangent.cu).
cudaError_t launch_assemble_dot(const double* r, const double* rdot, const ChainDesc* cd, int n_chains,
                                int max_N, double* Md, double hstar, double a, double hdot,
                                double adot, cudaStream_t s);
cudaError_t launch_trsm_rhs(const double* M, const double* Winv, const ChainDesc* cd, int n_chains,
                            int max_tiles, double* B, cudaStream_t s);
cudaError_t launch_transpose(const ChainDesc* cd, int n_chains, int max_tiles, double* B,
                             cudaStream_t s);
cudaError_t launch_phi_matvec(const double* X, const ChainDesc* cd, int n_chains, int max_n,
                              const double* xi, double* v, cudaStream_t s);
cudaError_t launch_gemv_dense(const double* A, const ChainDesc* cd, int n_chains, int max_n,
                              const double* f, double* w, cudaStream_t s);
// r*' and G = C(T u'); the rod directions and their tangents from (rq, rqdot).
cudaError_t launch_tangent_predictor(const double* r, const double* rdot, const double* rq, const double* rqdot,
                                     const double* ydot, const double* uhat, const double* T, const ChainDesc* cd,
                                     int n_chains, int max_N, Phys ph, const double* kappa_dot,
                                     double* rsdot, double* G, cudaStream_t s);
// v = Phi(X)^T xi for symmetric X (strict upper triangle plus half the diagonal).
cudaError_t launch_phi_upper_matvec(const double* X, const ChainDesc* cd, int n_chains, int max_n,
                                    const double* xi, double* v, cudaStream_t s);
// r_m' = r' + (P y)' / 2, the tangent of the midpoint of the corrected step.
cudaError_t launch_tangent_midpoint_dot(const double* r, const double* rdot, const double* y, const double* ydot,
                                        const ChainDesc* cd, int n_chains, const int* status, double* rmdot,
                                        cudaStream_t s);
cudaError_t tangent_configure();
// out = a + b over every chain's 3N values.
cudaError_t launch_vec_add(const ChainDesc* cd, int n_chains, int max_n, const double* a, const double* b,
                           double* out, cudaStream_t s);
cudaError_t launch_tangent_base(const ChainDesc* cd, int n_chains, int max_n, Phys ph,
                                const double* rsdot, const double* DdF, const double* DG, double* a,
                                cudaStream_t s);
cudaError_t launch_tangent_residual(const double* a, const double* u, const double* rnew,
                                    const ChainDesc* cd, int n_chains, Phys ph, double rel_tol,
                                    double* rscale, double* z, double* rhs, int* state, int* status,
                                    const int* iters, cudaStream_t s);
cudaError_t launch_tangent_init(const ChainDesc* cd, int n_chains, int max_n, const int* status,
                                int* state, int* iters, double* Tdot, double* Fdot, cudaStream_t s);

template <typename T>
cudaError_t launch_extract(const T* M, const ChainDesc* cd, int chain, int which, double* out,
                           cudaStream_t s);

}  // namespace bd
