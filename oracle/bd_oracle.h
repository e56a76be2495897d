/*
 * bd_oracle.h -- plain FP64 CPU oracle for the per-timestep hot path of
 * bead-rod Brownian dynamics with hydrodynamic interaction (HI), following
 * Prakash et al., "Petascale Brownian dynamics simulations of highly resolved
 * polymer chains with hydrodynamic interactions using modern GPUs"
 * (arXiv 2208.06559), Sec. 3.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The GPU product path
 * never links, imports or calls it, and it shares no code with the GPU path.
 *
 * Conventions (one chain):
 *   N beads, N-1 rods, rod k joins bead k to bead k+1, Q_k = r_{k+1} - r_k.
 *   n = 3N.  Rod length b = 1 and bead mobility kT/zeta = 1, so D_ii = I.
 *   Dense matrices are row-major n x n; element (3i+k, 3j+l) is component
 *   (k,l) of the 3x3 block D_ij, the bead-major interleaved ordering of the
 *   two-bead example in Sec. 4 (Eqs. (18)-(20)).
 *   Positions r are [N][3]; noise xi is [N][3] of i.i.d. N(0,1) numbers.
 *
 * Status codes returned by the step functions:
 *   0 ok, -4 non-positive (or NaN) Cholesky pivot, -5 Newton did not converge.
 */
#ifndef BD_ORACLE_H
#define BD_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define OR_OK 0
#define OR_ERR_NOT_PD (-4)
#define OR_ERR_CONSTRAINT (-5)

#define OR_FLOW_NONE 0
#define OR_FLOW_SHEAR 1
#define OR_FLOW_UNIAXIAL 2

#define OR_RIGID 0    /* rigid rods: tension solve */
#define OR_FRAENKEL 1 /* Fraenkel springs of stiffness kspring, semi-implicit (Sec. 3) */

#define OR_SCHEME_MIDPOINT 0 /* rigid rods: midpoint corrector (the default) */
#define OR_SCHEME_EULER 1    /* rigid rods: one projection from the start of the step */

#define OR_OBS_STRIDE 12 /* Rx Ry Rz R2 Rg2 stretch max||Q|-1| newton_iters tau_xx tau_yy tau_zz tau_xy */

typedef struct {
  double hstar;    /* HI parameter h* (>= 0) */
  double a;        /* bead radius; <= 0 means a = h* */
  double dt;       /* time step */
  int flow;        /* OR_FLOW_* */
  double Wi;       /* Weissenberg number */
  double lambda;   /* relaxation time; rate = Wi / lambda; <= 0 means 1 */
  double tol;      /* Newton tolerance on max_k | |Q_k|^2 - 1 | */
  int max_newton;  /* Newton update cap */
  int constraint;  /* OR_RIGID or OR_FRAENKEL */
  double kspring;  /* Fraenkel spring constant K* (OR_FRAENKEL) */
  int scheme;      /* OR_SCHEME_* (rigid rods only) */
} or_params;

/* 3x3 RPY block for separation R = r_i - r_j, Sec. 3 Eqs. (8)-(9). */
void or_rpy_block(const double R[3], double hstar, double a, double out[9]);
/* Full n x n diffusion tensor, Sec. 3 Eqs. (7)-(9). */
void or_assemble(int N, const double* r, double hstar, double a, double* D);
/* Unblocked Cholesky D = L L^T, Sec. 3 Eq. (10); L lower, zeros above.
 * Returns 0 or OR_ERR_NOT_PD. */
int or_cholesky(int n, const double* D, double* L);
/* y = L x with L lower triangular (the sum over j <= i of Eq. (6)). */
void or_trmv_lower(int n, const double* L, const double* x, double* y);
/* z = L^{-T} x: back substitution with the transpose of lower-triangular L. */
void or_trsv_lower_t(int n, const double* L, const double* x, double* z);
/* out = y - A^T (A A^T)^{-1} A y: the orthogonal projection of a bead
 * displacement y ([N][3]) onto the tangent space of the rod constraints
 * |Q_k| = 1 at positions r.  Row k of A holds -u_k at bead k and +u_k at
 * bead k+1 (u_k = Q_k/|Q_k|). */
void or_tangent_project(int N, const double* r, const double* y, double* out);
/* y = A x, dense. */
void or_gemv(int n, const double* A, const double* x, double* y);
/* kappa for the flow type (Sec. 3, flow-force paragraph); row-major 3x3. */
void or_kappa(int flow, double rate, double kappa[9]);
/* ||L L^T - D||_F / ||D||_F with long-double accumulation. */
double or_factor_residual(int n, const double* D, const double* L);

/* Rigid-rod tension solve for one chain: find T with |Q_k(r(T))| = 1,
 * r(T) = rstar + dt D F(T), F_i = T_i u_i - T_{i-1} u_{i-1}.
 * Newton with the exact Jacobian and dense LU; T holds the result.
 * r_out receives r(T).  Returns 0 or OR_ERR_CONSTRAINT. */
int or_tension_solve(int N, const double* D, const double* rstar,
                     const double* u, double dt, double tol, int max_newton,
                     double* T, double* r_out, int* iters);

/* Semi-implicit Fraenkel-spring update of one chain (Sec. 3, Eq. (3) and
 * the link equations eqQ2, (23)-(25)): from the old positions r, the
 * scaled Brownian displacement y (= sqrt(2 dt) L xi), kappa and D, the new
 * positions r_new; T_out[k] = K* (|Q_k| - 1) / |Q_k| at the new links (the
 * spring force is T_out[k] Q_k).  The centre of mass moves with the
 * explicit step; the new links are summed around it. */
void or_fraenkel_update(int N, const double* D, const double* kappa, double dt, double kspring,
                        const double* r, const double* y, double* r_new, double* T_out);

/* One full time step for one chain (assembly, Cholesky, Brownian
 * displacement, flow predictor, tension solve or Fraenkel update).
 * Rigid rods, OR_SCHEME_MIDPOINT: with y = sqrt(2 dt) L xi and z = L^{-T} xi
 * (so that D z = L xi), the midpoint r_m = r + P y / 2 (P: or_tangent_project
 * at r), D_m = D(r_m) and the rod directions u_m of r_m; the predictor is
 * r* = r + dt kappa.r + sqrt(2 dt) D_m z and the tensions act along u_m
 * through D_m.  OR_SCHEME_EULER: D and u of r throughout.  r is updated in place
 * unless the step fails, in which case r is left unchanged.
 * T_out (N-1) may be NULL.  Returns 0 or an error code. */
int or_step(const or_params* p, int N, double* r, const double* xi,
            double* T_out, int* iters, double* maxdev);

/* n_steps steps for a batch of chains (OpenMP across chains).
 * r is packed [sum N][3]; noise is [n_steps][sum N][3].
 * status[c], iters[c] (Newton updates in the last step), maxdev[c]
 * (max | |Q|-1 | over all steps) per chain.  A failed chain stops. */
void or_run(const or_params* p, int n_chains, const int* Nc, double* r,
            int n_steps, const double* noise, double* T_out, int* status,
            int* iters, double* maxdev);

/* Per-chain observables, Sec. 5 Eqs. (25)-(29):
 * out[0..2] = r_{N-1} - r_0, out[3] = |R_ee|^2, out[4] = Rg^2,
 * out[5] = |R_ee| / (N-1), out[6] = max_k | |Q_k| - 1 |, out[7] = 0,
 * out[8..11] = sum_k T_k Q_k,a Q_k,b for ab = xx, yy, zz, xy: the rod part of
 * the Kramers stress of Eq. (28) with the rod force T_k Q_k / |Q_k| (|Q_k| = 1)
 * in place of the spring force; T may be NULL (zero tensions). */
void or_observables(int N, const double* r, const double* T, double* out);

int or_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
