/*
 * bd.h -- C ABI of libbd, the GB300 (sm_103a) library for the per-timestep
 * hot path of Brownian dynamics of bead-rod polymer chains with hydrodynamic
 * interaction (HI), after Prakash et al., arXiv 2208.06559.
 *
 * One time step of every chain in a batch (Sec. 3; Sec. 4 flowchart):
 *   1. assemble the 3N x 3N Rotne-Prager-Yamakawa diffusion tensor D from the
 *      bead positions (Sec. 3 Eqs. (7)-(9));
 *   2. factor D = B B^T by Cholesky (Sec. 3 Eq. (10));
 *   3. form the Brownian displacement sqrt(2 dt) B xi (noise term of Eq. (6));
 *   4. add the flow drift dt kappa.r (Eq. (5)/(6)) and the tension drift
 *      dt D F(T) (constraint-force term of Eq. (6));
 *   5. solve for the rod tensions T that keep every rod at unit length (the
 *      rigid, K* -> infinity limit of the semi-implicit scheme of Eqs. (13)-(17)),
 *      or, with BD_FRAENKEL, the paper's own finite-K* semi-implicit update of
 *      Fraenkel springs (Sec. 3 Eq. (3), eqQ2, Eqs. (23)-(25)): steps 1-3, one
 *      mobility product with the spring forces at t, then a closed-form
 *      update per link.
 * Rigid rods with BD_SCHEME_MIDPOINT (the default) evaluate the mobility of
 * steps 3-5 and the rod directions of step 5 at the midpoint
 * r_m = r + P y / 2 (y = sqrt(2 dt) L xi, P the orthogonal projection onto
 * the tangent space of the rod constraints at r) and move by
 * sqrt(2 dt) D(r_m) L^{-T} xi: one Cholesky factor per step, and the mean
 * drift of rigid-rod diffusion with HI, whose statics HI leaves unchanged.
 * BD_SCHEME_EULER uses D and the rod directions of r throughout; with
 * h* > 0 it lacks part of that drift (the paper itself runs stiff springs,
 * which need no such term).
 *
 * Conventions.  A chain has N >= 2 beads and N-1 rods; rod k joins bead k to
 * bead k+1.  Rod length b = 1 and bead mobility kT/zeta = 1, so D_ii = I.
 * Positions, noise and forces are packed FP64 arrays [sum_c N_c][3]: the
 * beads of chain c start at bead offset sum_{c'<c} N_c'.
 *
 * Memory.  Every pointer argument named *_dev is a device pointer allocated by
 * the caller (cudaMalloc or a framework allocator); pointers named *_host are
 * host memory.  bd_step and bd_observables also accept host memory for their
 * data buffers (detected with cudaPointerGetAttributes) and then copy through
 * library-owned device staging.  The caller owns every buffer it passes; the
 * context owns its workspace (matrices, tensions, scratch) and frees it in
 * bd_destroy.
 *
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Device work is enqueued asynchronously on it; calls that return
 * host results (bd_observables with status_host, bd_factor_residual,
 * bd_read_matrix, bd_chain_status) synchronise that stream first.
 *
 * Errors.  Every int-returning call returns BD_OK (0) or a negative code.
 * Per-chain failures inside a step (a non-positive Cholesky pivot, a tension
 * solve that did not converge) do not fail the call: the chain is frozen at
 * its last good state, its status word records the first error, and the
 * status words are read with bd_observables or bd_chain_status.  No kernel
 * traps; every device wait is bounded.
 */
#ifndef BD_H
#define BD_H

#ifdef __cplusplus
extern "C" {
#endif

#define BD_OK 0
#define BD_ERR_ARG (-1)         /* invalid argument */
#define BD_ERR_CUDA (-2)        /* a CUDA runtime call failed */
#define BD_ERR_OOM (-3)         /* device allocation failed */
#define BD_ERR_NOT_PD (-4)      /* non-positive or NaN Cholesky pivot */
#define BD_ERR_CONSTRAINT (-5)  /* tension Newton did not converge */
#define BD_ERR_TIMEOUT (-6)     /* a bounded device wait expired */
#define BD_ERR_STATE (-7)       /* call made before bd_set_state */

typedef struct bd_ctx bd_ctx; /* opaque, library-owned */

typedef enum { BD_FLOW_NONE = 0, BD_FLOW_SHEAR = 1, BD_FLOW_UNIAXIAL = 2 } bd_flow;
/* BD_FP64: every stage in FP64.
 * BD_MIXED_TF32: D and its factor stored in FP32; FP32 diagonal tiles of the
 * factor; panel solves on the tensor cores with operands rounded to TF32
 * (round to nearest), the factor's tiles stored so rounded; trailing updates
 * on the tensor cores from FP16 copies of those tiles (the same 10-bit
 * mantissa; |L_ij| <= 1 since D has a unit diagonal), FP32 accumulation;
 * one refinement step on the Brownian displacement; the tension iteration
 * with FP64-level (double-float) products, so rods hold to the tolerance.
 * BD_MIXED_BF16: rejected by bd_create with BD_ERR_ARG (no factorisation
 * with BF16 operands is built).  The FP16 operands of BD_MIXED_TF32 already
 * run at the BF16 tensor rate with two more mantissa bits; BF16 operands
 * (8-bit mantissa) leave the refined factor's error at 4.6e-6 for N = 1000
 * in an FP64 emulation of the factorisation's roundings, above 1e-6. */
typedef enum { BD_FP64 = 0, BD_MIXED_TF32 = 1, BD_MIXED_BF16 = 2 } bd_precision;
typedef enum { BD_RIGID = 0, BD_FRAENKEL = 1 } bd_constraint;
typedef enum { BD_SCHEME_MIDPOINT = 0, BD_SCHEME_EULER = 1 } bd_scheme;

/* Observables written per chain by bd_observables (Sec. 5 Eqs. (25)-(29)). */
#define BD_OBS_STRIDE 12
#define BD_OBS_REE_X 0     /* r_{N-1} - r_0, three components */
#define BD_OBS_R2 3        /* |R_ee|^2 */
#define BD_OBS_RG2 4       /* radius of gyration squared */
#define BD_OBS_STRETCH 5   /* |R_ee| / (N-1) */
#define BD_OBS_MAXDEV 6    /* max_k | |Q_k| - 1 | */
#define BD_OBS_NEWTON 7    /* Newton updates in the last step */
/* Rod part of the Kramers stress, Eq. (28), with the rod force T_k Q_k (|Q_k|
 * = 1, T_k the tension of the last step) in place of the spring force:
 * sum_k T_k Q_k,a Q_k,b.  The isotropic N delta_ab and the ensemble average
 * are the caller's; N1 = tau_xx - tau_yy (Eq. (29)). */
#define BD_OBS_TAU_XX 8
#define BD_OBS_TAU_YY 9
#define BD_OBS_TAU_ZZ 10
#define BD_OBS_TAU_XY 11

typedef struct {
  int n_chains;          /* >= 1 */
  const int* n_beads;    /* host array [n_chains], each 2 <= N_c <= 4096 (BD_FP64) or 8192 (mixed); uneven allowed */
  double h_star;         /* HI parameter h* >= 0 (Eqs. (8)-(9)) */
  double a;              /* bead radius; <= 0 means a = h*; a < h* is rejected */
  double dt;             /* time step > 0 */
  int flow;              /* bd_flow */
  double Wi;             /* Weissenberg number; rate = Wi / lambda */
  double lambda;         /* relaxation time; <= 0 means 1 */
  int precision;         /* bd_precision: BD_FP64 or BD_MIXED_TF32 */
  int constraint;        /* bd_constraint: BD_RIGID (tension solve) or BD_FRAENKEL */
  double tol;            /* Newton tolerance on max_k | |Q_k|^2 - 1 |; <= 0 -> 1e-13 */
  int max_newton;        /* Newton update cap; <= 0 -> 50 */
  int refine;            /* mixed precision: 1 = one refinement step on B xi */
  double k_spring;       /* BD_FRAENKEL: spring constant K* > 0 (Eq. (3)); unused for BD_RIGID */
  int scheme;            /* bd_scheme of the rigid-rod step (BD_RIGID only) */
  int lanes;             /* concurrent sub-batches (lanes) the chains are split into, contiguous
                            ranges of about equal factorisation work, each stepped by its own graph
                            on its own streams; 1..8 (at most n_chains), or 0 = automatic: mixed
                            precision 2 from 32 chains, or from 4 chains when one has >= 2000 beads,
                            else 1; FP64 one per 16 chains up to 8, and 1 for rigid-rod batches of
                            chains of <= 32 beads (one fused kernel steps them).  A chain's result
                            depends on the lanes only through the shapes chosen for its per-chain
                            kernels (summation order).  Out of range: BD_ERR_ARG */
} bd_params;

/* Fill *p with defaults: 1 chain (n_beads NULL), h* = 0.25, a = h*, dt = 1e-4,
 * no flow, lambda = 1, BD_FP64, BD_RIGID, tol 1e-13, max_newton 50, refine 1,
 * k_spring 1e4, BD_SCHEME_MIDPOINT, lanes 0 (automatic). */
void bd_params_default(bd_params* p);

/* Create a context on the current CUDA device: validates *p, copies n_beads,
 * allocates all device workspace.  *out receives the handle (NULL on error).
 * Non-finite dt, h*, Wi, lambda or tol are rejected, as are the range errors
 * noted on the fields above.  Errors: BD_ERR_ARG, BD_ERR_OOM, BD_ERR_CUDA. */
int bd_create(const bd_params* p, bd_ctx** out);

/* Free every resource of the context (NULL is allowed). */
void bd_destroy(bd_ctx* ctx);

/* Load positions [sum N][3] FP64 (device pointer) into the context and reset
 * every chain's status word and tensions. */
int bd_set_state(bd_ctx* ctx, const double* r_dev, void* stream);

/* Copy the current positions [sum N][3] FP64 into r_dev (device pointer). */
int bd_get_state(bd_ctx* ctx, double* r_dev, void* stream);

/* Advance every chain by n_steps >= 1 time steps.  noise: [n_steps][sum N][3]
 * FP64 i.i.d. N(0,1) numbers, device or host memory, owned by the caller and
 * read during the call's stream work (host memory is copied before return of
 * the staged copies).  All n_steps run in one launch of the context's CUDA
 * graph, whose outer WHILE node loops over the steps on the device (the
 * first call captures and instantiates the graph); a context with lanes
 * launches every lane's graph on the lane's own stream, all waiting for the
 * caller's earlier work on `stream`, and the caller's later work on it waits
 * for all of them.  Asynchronous; returns
 * BD_OK unless the arguments or a CUDA call fail.  Errors: BD_ERR_ARG,
 * BD_ERR_STATE, BD_ERR_CUDA. */
int bd_step(bd_ctx* ctx, int n_steps, const double* noise, void* stream);

/* Per-chain observables [n_chains][BD_OBS_STRIDE] FP64 into obs (device or
 * host memory).  If status_host is not NULL it receives the n_chains status
 * words (BD_OK or the first per-chain error) after a stream synchronisation,
 * and the call returns the most severe of them. */
int bd_observables(bd_ctx* ctx, double* obs, int* status_host, void* stream);

/* Host copies of the per-chain status words and Newton update counts of the
 * last step (either pointer may be NULL).  Synchronises the stream and
 * returns the most severe status. */
int bd_chain_status(bd_ctx* ctx, int* status_host, int* newton_host, void* stream);

/* One time step launched kernel by kernel (no graph) with CUDA events at the
 * stage boundaries, for profiling.  noise: device pointer, [sum N][3] FP64,
 * the step's N(0,1) noise; newton_iters: tension-solve bodies enqueued
 * (<= 0: max_newton + 2; chains that have converged skip them on the
 * device).  ms_out[8] (host) receives milliseconds: assembly, Cholesky
 * factorisation, Brownian displacement, wait for the rod-coupling matrix K
 * (built on a second stream) plus the predictor, tension iterations,
 * commit, whole step, and the end of the K chain measured from the start of
 * the step.  The state advances by one step as with bd_step.  It runs on the
 * context's own stream, where bd_step runs too; work the caller enqueued on
 * other streams must be complete.  Synchronises the context's stream.  A
 * context with lanes profiles them one after another and reports the sums of
 * their times.  Errors: BD_ERR_ARG (NULL or host noise),
 * BD_ERR_STATE (no state), BD_ERR_CUDA. */
int bd_profile_step(bd_ctx* ctx, const double* noise, int newton_iters, double* ms_out);

/* Number of kernel launches executed by bd_step on this context since its
 * creation (the kernels of one step of the captured graph times the steps,
 * plus the kernels of every executed tension-solve iteration), summed over
 * the lanes.  Synchronises the stream. */
int bd_kernel_launches(bd_ctx* ctx, unsigned long long* out, void* stream);

/* Number of lanes (concurrent sub-batches, see bd_params.lanes) the context
 * steps its chains in.  Errors: BD_ERR_ARG (NULL). */
int bd_lanes(bd_ctx* ctx, int* out);

/* Diagnostic: ||B B^T - D||_F / ||D||_F for one chain, from the factor and
 * the D currently held by the context (after bd_factor or bd_step), in FP64
 * on the device.  Synchronises the legacy default stream. */
int bd_factor_residual(bd_ctx* ctx, int chain, double* rel_fro);

/* ---- stage entry points (one row of the step each; for tests and tools) ---- */

/* Stage 1: D from the current positions (Eqs. (7)-(9)). */
int bd_assemble(bd_ctx* ctx, void* stream);
/* Stage 2: Cholesky factor of the assembled D (Eq. (10)). */
int bd_factor(bd_ctx* ctx, void* stream);
/* Stage 3: y = sqrt(2 dt) B xi for xi [sum N][3] (device); with mixed
 * precision and refine = 1 the refined displacement of the library is
 * returned.  y_dev [sum N][3] FP64. */
int bd_brownian(bd_ctx* ctx, const double* xi_dev, double* y_dev, void* stream);
/* Stage 4: u = D f for f [sum N][3] (device), FP64 result. */
int bd_mobility_apply(bd_ctx* ctx, const double* f_dev, double* u_dev, void* stream);
/* Stage 5 input/outputs: tensions of the last step, [sum (N-1)] FP64. */
int bd_get_tensions(bd_ctx* ctx, double* T_dev, void* stream);
/* Stage 3' of the midpoint scheme (after bd_assemble and bd_factor; rigid
 * contexts with BD_SCHEME_MIDPOINT only): for xi [sum N][3] (device),
 * rmid_dev [sum N][3] receives r_m = r + P y / 2 (y = sqrt(2 dt) B xi, P the
 * orthogonal projection onto the tangent space of |Q_k| = 1 at r) and y_dev
 * [sum N][3] the step's Brownian displacement sqrt(2 dt) D(r_m) B^{-T} xi.
 * Mixed precision: y is the refined displacement of stage 3 plus
 * sqrt(2 dt) (D(r_m) - D(r)) B^{-T} xi with that difference evaluated from
 * the positions in FP32.  Errors: BD_ERR_ARG, BD_ERR_STATE, BD_ERR_CUDA. */
int bd_midpoint(bd_ctx* ctx, const double* xi_dev, double* rmid_dev, double* y_dev, void* stream);

/* Pathwise gradient of an objective J(r_final) with respect to the
 * Weissenberg number and h*, at fixed noise (the paper has no derivatives).
 * Runs n_steps FP64 steps from r0_dev [sum N][3] (device) with noise_dev
 * [n_steps][sum N][3] (device) and returns grad_host[0] = dJ/dWi,
 * grad_host[1] = dJ/dh* (a = h* when the context was created with a <= 0, so
 * a moves with h*), given dJdr_final_dev = dJ/dr at the final positions
 * [sum N][3] (device).  The derivative of the discrete step map is exact: it
 * is propagated forward (tangents of the RPY assembly, of the Cholesky factor
 * L' = L Phi(L^{-1} D' L^{-T}), of the Brownian and flow terms, and of the
 * tension solve by the implicit function theorem), which for two parameters
 * needs no checkpoints; ckpt_every is accepted and ignored.  The context is
 * left at the final state.  With BD_SCHEME_MIDPOINT the tangents also run
 * through the midpoint: z' = -L^{-T} Phi(X)^T xi, the derivative of the
 * tangent-space projection, and D(r_m)' from r_m'.  FP64 rigid-rod contexts
 * with h* > 0 only (else BD_ERR_ARG).  With lanes, the lanes' steps and
 * tangents run concurrently and their chains' contributions are summed.
 * Synchronises the stream; returns the most severe chain status. */
int bd_adjoint(bd_ctx* ctx, const double* r0_dev, int n_steps, const double* noise_dev,
               int ckpt_every, const double* dJdr_final_dev, double grad_host[2], void* stream);

/* ---- tile-shape tuning of the mixed-precision Cholesky ----
 * The tensor-core factorisation has two shape parameters: the super-panel
 * width (tile columns whose trailing update is applied together, K = 128 x
 * panel) and the number of chain groups factored concurrently on separate
 * streams.  A panel at least as wide as a chain's tile count makes the
 * factorisation left-looking (every column receives all earlier columns'
 * updates at once, no trailing update).  bd_tune_factor times every
 * combination of panel {2, 4, 6, 8, 12, 16, 24} and groups {1, 2, 4, 8, 12,
 * 16} (groups <= chains) on the context's current positions,
 * keeps the fastest and reports it (any output pointer may be NULL);
 * bd_set_factor_config applies a known choice (e.g. from a cache).  Both drop
 * the captured step graph, which is rebuilt by the next bd_step.  Mixed
 * contexts only (BD_ERR_ARG otherwise); bd_tune_factor needs bd_set_state
 * first and synchronises the stream.  With lanes, each shape is timed with
 * every lane factoring its chains concurrently and the winner is applied to
 * every lane; bd_set_factor_config also applies to every lane (groups are
 * per lane). */
int bd_tune_factor(bd_ctx* ctx, int* panel_out, int* groups_out, double* ms_out, void* stream);
int bd_set_factor_config(bd_ctx* ctx, int panel, int groups);  /* 1 <= panel <= 96 */

/* Copy chain `chain`'s dense n x n (n = 3 N_c) matrix `which` to host FP64
 * row-major: which = 0 -> D, 1 -> the Cholesky factor B (zeros above the
 * diagonal).  Synchronises the legacy default stream. */
int bd_read_matrix(bd_ctx* ctx, int chain, int which, double* out_host);

/* ---- self-test of the bounded device wait ----
 * Every wait of the library's kernels on an mbarrier (TMA arrivals, tensor-core
 * commits) is bounded: after 4e9 SM clock cycles (about two seconds) it gives up, the kernel
 * records BD_ERR_TIMEOUT in the chain's status word and unwinds, and the CUDA
 * context stays usable.  This call runs that wait in one thread on the current
 * device: with arrive = 0 nothing completes the barrier's phase and
 * *status_host receives BD_ERR_TIMEOUT after the limit (about two seconds);
 * with arrive != 0 the thread arrives first and it receives BD_OK.  Returns
 * BD_OK when the kernel ran (synchronising the legacy default stream);
 * errors: BD_ERR_ARG (NULL), BD_ERR_OOM, BD_ERR_CUDA. */
int bd_selftest_bounded_wait(int arrive, int* status_host);

/* ---- allocation-free entry point ----
 * The paper has no counterpart to this call; it exists for callers that cannot
 * allocate device memory (code inside a host framework that owns all device
 * allocations, or a thread that must not call cudaMalloc/cudaFree, which can
 * synchronise the device) and therefore cannot create a bd_ctx.
 *
 * u = D(r) f for ONE chain of n_beads <= BD_STATIC_MAX_BEADS beads, with D the
 * same RPY diffusion tensor the context assembles, evaluated on the fly from
 * the positions (finite h_star >= 0; finite a, a <= 0 meaning a = h_star;
 * a < h_star is rejected).
 * r_dev, f_dev, u_dev: FP64 [n_beads][3] in memory of the CURRENT CUDA device
 * (checked; other memory is rejected), owned by the caller.
 * It allocates nothing: its scratch is a fixed file-scope device array of
 * 786,432 bytes that every GPU loading the library holds until exit.  The
 * first call on each device looks up that array's device address (with the
 * device current) and caches it; make that first call before any stream
 * capture, and do not call it again on a device after cudaDeviceReset of that
 * device (the cached address is then stale).  Every call shares the array and
 * writes each slot before reading it, so calls whose work overlaps on the GPU
 * (other streams or host threads) race and must be serialised by the caller.
 * Asynchronous on `stream`.
 * Errors: BD_ERR_ARG (NULL pointer or memory of another device, n_beads < 1 or
 * > BD_STATIC_MAX_BEADS, bad h_star/a), BD_ERR_CUDA. */
#define BD_STATIC_MAX_BEADS 1024
int bd_mobility_apply_static(const double* r_dev, int n_beads, double h_star, double a,
                             const double* f_dev, double* u_dev, void* stream);

/* Human-readable text for an error code (static storage). */
const char* bd_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* BD_H */
