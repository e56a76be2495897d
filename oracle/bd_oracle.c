/*
 * bd_oracle.c -- plain FP64 CPU oracle, bead-rod Brownian dynamics with HI
 * (arXiv 2208.06559, Sec. 3).  TEST INFRASTRUCTURE ONLY: see bd_oracle.h.
 *
 * Everything here is written for a reader checking it against the paper:
 * no blocking, no fusion, loops in the order of the definitions.
 * Readings of points where the paper is silent or garbled:
 *   - N beads (the paper counts N rods and N+1 beads).
 *   - Brownian displacement sqrt(2 dt) L xi with xi ~ N(0,1); this has the
 *     second moment of the paper's sqrt(6/dt) uniform[-1,1] force times dt
 *     (Sec. 3 Eq. (2)); the sum in Eq. (6) is read as lower triangular.
 *   - Rigid rods: the K* -> infinity limit of the Fraenkel scheme of
 *     Eqs. (13)-(17) gives |Q| = 1; tensions T_k are solved by Newton so that
 *     |Q_k| = 1 to the tolerance, with the self-only K* -> infinity limit of
 *     Eq. (17), T_k = (|Q*_k| - 1)/(2 dt), as the starting point.
 *   - a <= 0 means a = h*; R = 0 takes the limit of the overlap branch.
 */
#include "bd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Sec. 3 Eqs. (8) and (9).  R = r_i - r_j, i != j. */
void or_rpy_block(const double R[3], double hstar, double a, double out[9]) {
  double R2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
  double Rn = sqrt(R2);
  double cI, cRR; /* D = cI * I + cRR * (R R^T / R^2) */
  if (hstar == 0.0) {
    cI = 0.0;
    cRR = 0.0;
  } else if (Rn >= 2.0 * a) {
    /* Eq. (8): (3 hs / (4R)) [ (1 + 2a^2/(3R^2)) I + (1 - 2a^2/R^2) RR/R^2 ] */
    double pref = 3.0 * hstar / (4.0 * Rn);
    cI = pref * (1.0 + 2.0 * a * a / (3.0 * R2));
    cRR = pref * (1.0 - 2.0 * a * a / R2);
  } else {
    /* Eq. (9): (3 hs / (4R)) (R/(2a)) [ (8/3 - 3R/(4a)) I + (R/(4a)) RR/R^2 ] */
    double pref = 3.0 * hstar / (8.0 * a);
    cI = pref * (8.0 / 3.0 - 3.0 * Rn / (4.0 * a));
    cRR = pref * (Rn / (4.0 * a));
  }
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) {
      double rr = (Rn > 0.0) ? R[k] * R[l] / R2 : 0.0;
      out[3 * k + l] = (k == l ? cI : 0.0) + cRR * rr;
    }
}

/* Sec. 3 Eqs. (7)-(9) over all bead pairs. */
void or_assemble(int N, const double* r, double hstar, double a, double* D) {
  int n = 3 * N;
  if (a <= 0.0) a = hstar;
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      double blk[9];
      if (i == j) {
        for (int q = 0; q < 9; ++q) blk[q] = (q % 4 == 0) ? 1.0 : 0.0;
      } else {
        double R[3] = {r[3 * i] - r[3 * j], r[3 * i + 1] - r[3 * j + 1],
                       r[3 * i + 2] - r[3 * j + 2]};
        or_rpy_block(R, hstar, a, blk);
      }
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l)
          D[(size_t)(3 * i + k) * n + (3 * j + l)] = blk[3 * k + l];
    }
}

/* Sec. 3 Eq. (10): D = L L^T, L lower triangular, positive diagonal. */
int or_cholesky(int n, const double* D, double* L) {
  memset(L, 0, sizeof(double) * (size_t)n * n);
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = D[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) s -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      if (i == j) {
        if (!(s > 0.0)) return OR_ERR_NOT_PD;
        L[(size_t)i * n + i] = sqrt(s);
      } else {
        L[(size_t)i * n + j] = s / L[(size_t)j * n + j];
      }
    }
  }
  return OR_OK;
}

void or_trmv_lower(int n, const double* L, const double* x, double* y) {
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 0; j <= i; ++j) s += L[(size_t)i * n + j] * x[j];
    y[i] = s;
  }
}

void or_trsv_lower_t(int n, const double* L, const double* x, double* z) {
  for (int i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int j = i + 1; j < n; ++j) s -= L[(size_t)j * n + i] * z[j];
    z[i] = s / L[(size_t)i * n + i];
  }
}

static int lu_solve(int m, double* A, double* b);

void or_tangent_project(int N, const double* r, const double* y, double* out) {
  int m = N - 1;
  double* u = (double*)malloc(sizeof(double) * 3 * (m > 0 ? m : 1));
  double* H = (double*)calloc((size_t)(m > 0 ? m : 1) * (m > 0 ? m : 1), sizeof(double));
  double* c = (double*)malloc(sizeof(double) * (m > 0 ? m : 1));
  for (int k = 0; k < m; ++k) {
    double q[3], qn = 0.0;
    for (int e = 0; e < 3; ++e) {
      q[e] = r[3 * (k + 1) + e] - r[3 * k + e];
      qn += q[e] * q[e];
    }
    qn = sqrt(qn);
    for (int e = 0; e < 3; ++e) u[3 * k + e] = q[e] / qn;
  }
  /* H = A A^T and c = A y, row k of A being (-u_k at bead k, +u_k at bead k+1) */
  for (int k = 0; k < m; ++k) {
    c[k] = 0.0;
    for (int e = 0; e < 3; ++e) c[k] += u[3 * k + e] * (y[3 * (k + 1) + e] - y[3 * k + e]);
    for (int l = 0; l < m; ++l) {
      double s = 0.0;
      for (int i = 0; i < N; ++i)
        for (int e = 0; e < 3; ++e) {
          double ak = (i == k + 1 ? u[3 * k + e] : 0.0) - (i == k ? u[3 * k + e] : 0.0);
          double al = (i == l + 1 ? u[3 * l + e] : 0.0) - (i == l ? u[3 * l + e] : 0.0);
          s += ak * al;
        }
      H[(size_t)k * m + l] = s;
    }
  }
  if (m > 0) lu_solve(m, H, c); /* c <- (A A^T)^{-1} A y */
  for (int i = 0; i < N; ++i)
    for (int e = 0; e < 3; ++e) {
      double s = y[3 * i + e];
      if (i < m) s += c[i] * u[3 * i + e];             /* row i of A: -u_i at bead i */
      if (i > 0) s -= c[i - 1] * u[3 * (i - 1) + e];   /* row i-1: +u_{i-1} at bead i */
      out[3 * i + e] = s;
    }
  free(u);
  free(H);
  free(c);
}

void or_gemv(int n, const double* A, const double* x, double* y) {
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += A[(size_t)i * n + j] * x[j];
    y[i] = s;
  }
}

/* Sec. 3: uniaxial extension diag(e, -e/2, -e/2); shear kappa_xy = g. */
void or_kappa(int flow, double rate, double kappa[9]) {
  for (int q = 0; q < 9; ++q) kappa[q] = 0.0;
  if (flow == OR_FLOW_UNIAXIAL) {
    kappa[0] = rate;
    kappa[4] = -0.5 * rate;
    kappa[8] = -0.5 * rate;
  } else if (flow == OR_FLOW_SHEAR) {
    kappa[1] = rate;
  }
}

double or_factor_residual(int n, const double* D, const double* L) {
  long double num = 0.0L, den = 0.0L;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      int m = i < j ? i : j;
      long double s = 0.0L;
      for (int k = 0; k <= m; ++k)
        s += (long double)L[(size_t)i * n + k] * (long double)L[(size_t)j * n + k];
      long double d = (long double)D[(size_t)i * n + j];
      num += (s - d) * (s - d);
      den += d * d;
    }
  return (double)sqrtl(num / den);
}

/* Dense LU with partial pivoting, solves A x = b in place (b -> x).
 * A (m x m, row-major) is destroyed.  Returns 0 or -1 if singular. */
static int lu_solve(int m, double* A, double* b) {
  for (int c = 0; c < m; ++c) {
    int p = c;
    double best = fabs(A[(size_t)c * m + c]);
    for (int i = c + 1; i < m; ++i) {
      double v = fabs(A[(size_t)i * m + c]);
      if (v > best) { best = v; p = i; }
    }
    if (best == 0.0) return -1;
    if (p != c) {
      for (int j = 0; j < m; ++j) {
        double t = A[(size_t)c * m + j];
        A[(size_t)c * m + j] = A[(size_t)p * m + j];
        A[(size_t)p * m + j] = t;
      }
      double t = b[c]; b[c] = b[p]; b[p] = t;
    }
    double piv = A[(size_t)c * m + c];
    for (int i = c + 1; i < m; ++i) {
      double f = A[(size_t)i * m + c] / piv;
      if (f == 0.0) continue;
      A[(size_t)i * m + c] = f;
      for (int j = c + 1; j < m; ++j) A[(size_t)i * m + j] -= f * A[(size_t)c * m + j];
      b[i] -= f * b[c];
    }
  }
  for (int i = m - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < m; ++j) s -= A[(size_t)i * m + j] * b[j];
    b[i] = s / A[(size_t)i * m + i];
  }
  return 0;
}

/* r(T) = rstar + dt D F(T) with F_i = T_i u_i - T_{i-1} u_{i-1}. */
static void positions_of_tension(int N, const double* D, const double* rstar,
                                 const double* u, const double* T, double dt,
                                 double* F, double* r_out) {
  int n = 3 * N;
  for (int i = 0; i < N; ++i)
    for (int k = 0; k < 3; ++k) {
      double f = 0.0;
      if (i < N - 1) f += T[i] * u[3 * i + k];
      if (i > 0) f -= T[i - 1] * u[3 * (i - 1) + k];
      F[3 * i + k] = f;
    }
  for (int p = 0; p < n; ++p) {
    double s = 0.0;
    for (int q = 0; q < n; ++q) s += D[(size_t)p * n + q] * F[q];
    r_out[p] = rstar[p] + dt * s;
  }
}

int or_tension_solve(int N, const double* D, const double* rstar,
                     const double* u, double dt, double tol, int max_newton,
                     double* T, double* r_out, int* iters) {
  int n = 3 * N, m = N - 1;
  double* F = (double*)malloc(sizeof(double) * n);
  double* g = (double*)malloc(sizeof(double) * (m > 0 ? m : 1));
  double* J = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1) * (m > 0 ? m : 1));
  int status = OR_OK, it = 0, extra = 0;

  /* Starting point: K* -> infinity limit of Eq. (17), rod by rod. */
  for (int k = 0; k < m; ++k) {
    double q2 = 0.0;
    for (int c = 0; c < 3; ++c) {
      double d = rstar[3 * (k + 1) + c] - rstar[3 * k + c];
      q2 += d * d;
    }
    T[k] = (sqrt(q2) - 1.0) / (2.0 * dt);
  }
  for (;;) {
    positions_of_tension(N, D, rstar, u, T, dt, F, r_out);
    double maxg = 0.0;
    for (int k = 0; k < m; ++k) {
      double q2 = 0.0;
      for (int c = 0; c < 3; ++c) {
        double d = r_out[3 * (k + 1) + c] - r_out[3 * k + c];
        q2 += d * d;
      }
      g[k] = q2 - 1.0;
      if (fabs(g[k]) > maxg || g[k] != g[k]) maxg = (g[k] != g[k]) ? INFINITY : fabs(g[k]);
    }
    if (extra) break;
    if (maxg <= tol) extra = 1; /* one more update after convergence */
    else if (it >= max_newton) { status = OR_ERR_CONSTRAINT; break; }
    /* J_kl = 2 Q_k . dQ_k/dT_l,
     * dQ_k/dT_l = dt [ (D_{k+1,l} - D_{k,l}) - (D_{k+1,l+1} - D_{k,l+1}) ] u_l */
    for (int k = 0; k < m; ++k) {
      double Q[3];
      for (int c = 0; c < 3; ++c) Q[c] = r_out[3 * (k + 1) + c] - r_out[3 * k + c];
      for (int l = 0; l < m; ++l) {
        double dQ[3];
        for (int c = 0; c < 3; ++c) {
          double s = 0.0;
          for (int e = 0; e < 3; ++e) {
            double blk = D[(size_t)(3 * (k + 1) + c) * n + 3 * l + e]
                       - D[(size_t)(3 * k + c) * n + 3 * l + e]
                       - D[(size_t)(3 * (k + 1) + c) * n + 3 * (l + 1) + e]
                       + D[(size_t)(3 * k + c) * n + 3 * (l + 1) + e];
            s += blk * u[3 * l + e];
          }
          dQ[c] = dt * s;
        }
        J[(size_t)k * m + l] = 2.0 * (Q[0] * dQ[0] + Q[1] * dQ[1] + Q[2] * dQ[2]);
      }
      g[k] = -g[k];
    }
    if (lu_solve(m, J, g) != 0) { status = OR_ERR_CONSTRAINT; break; }
    for (int k = 0; k < m; ++k) T[k] += g[k];
    ++it;
  }
  if (iters) *iters = it;
  free(F);
  free(g);
  free(J);
  return status;
}

int or_step(const or_params* p, int N, double* r, const double* xi,
            double* T_out, int* iters, double* maxdev) {
  int n = 3 * N, m = N - 1;
  double a = p->a > 0.0 ? p->a : p->hstar;
  double rate = p->Wi / (p->lambda > 0.0 ? p->lambda : 1.0);
  double kap[9];
  or_kappa(p->flow, rate, kap);
  double* D = (double*)malloc(sizeof(double) * (size_t)n * n);
  double* L = (double*)malloc(sizeof(double) * (size_t)n * n);
  double* y = (double*)malloc(sizeof(double) * n);
  double* rs = (double*)malloc(sizeof(double) * n);
  double* rn = (double*)malloc(sizeof(double) * n);
  double* u = (double*)malloc(sizeof(double) * 3 * (m > 0 ? m : 1));
  double* T = (double*)malloc(sizeof(double) * (m > 0 ? m : 1));
  double* z = (double*)malloc(sizeof(double) * n);
  double* w = (double*)malloc(sizeof(double) * n);
  double* rm = (double*)malloc(sizeof(double) * n);
  double* Dm = (double*)malloc(sizeof(double) * (size_t)n * n);
  int status;

  /* 1. diffusion tensor at the current positions, Eqs. (7)-(9) */
  or_assemble(N, r, p->hstar, a, D);
  /* 2. its Cholesky factor, Eq. (10) */
  status = or_cholesky(n, D, L);
  if (status == OR_OK) {
    /* 3. Brownian displacement y = sqrt(2 dt) L xi (Eq. (6) noise term) */
    or_trmv_lower(n, L, xi, y);
    double s = sqrt(2.0 * p->dt);
    if (p->constraint == OR_FRAENKEL) {
      /* 4'. Fraenkel springs, semi-implicit link update (Sec. 3) */
      for (int e = 0; e < n; ++e) y[e] *= s;
      or_fraenkel_update(N, D, kap, p->dt, p->kspring, r, y, rn, T);
      memcpy(r, rn, sizeof(double) * n);
      if (T_out) memcpy(T_out, T, sizeof(double) * m);
      if (iters) *iters = 0;
      if (maxdev) {
        double md = 0.0;
        for (int k = 0; k < m; ++k) {
          double q2 = 0.0;
          for (int c = 0; c < 3; ++c) {
            double d = r[3 * (k + 1) + c] - r[3 * k + c];
            q2 += d * d;
          }
          double dv = fabs(sqrt(q2) - 1.0);
          if (dv > md) md = dv;
        }
        *maxdev = md;
      }
      free(D);
      free(L);
      free(y);
      free(rs);
      free(rn);
      free(u);
      free(T);
      free(z);
      free(w);
      free(rm);
      free(Dm);
      return OR_OK;
    }
    /* 4. The mobility and the rod directions the step uses.  Euler: those
     *    of r.  Midpoint (a reading: the paper runs stiff springs, whose
     *    statistics need no such term): they are taken at
     *    r_m = r + P y / 2, P the orthogonal projection onto the tangent
     *    space of the constraints at r, and the Brownian displacement
     *    becomes sqrt(2 dt) D_m z with z = L^{-T} xi (D z = L xi).  Through
     *    the correlation of r_m with z this adds the mean drift that the
     *    rigid-rod diffusion on the constraint surface needs with HI. */
    const double* Dstep = D;
    const double* rdir = r;
    if (p->scheme != OR_SCHEME_EULER) {
      or_trsv_lower_t(n, L, xi, z);
      or_tangent_project(N, r, y, w);
      for (int e = 0; e < n; ++e) rm[e] = r[e] + 0.5 * s * w[e];
      or_assemble(N, rm, p->hstar, a, Dm);
      or_gemv(n, Dm, z, y); /* y <- D_m z */
      Dstep = Dm;
      rdir = rm;
    }
    /* 5. predictor r* = r + dt kappa.r + sqrt(2 dt) y (Eq. (6) flow term)
     *    and the rod directions u_k = Q_k / |Q_k| along which tensions act */
    for (int i = 0; i < N; ++i)
      for (int k = 0; k < 3; ++k) {
        double kr = kap[3 * k] * r[3 * i] + kap[3 * k + 1] * r[3 * i + 1] +
                    kap[3 * k + 2] * r[3 * i + 2];
        rs[3 * i + k] = r[3 * i + k] + p->dt * kr + s * y[3 * i + k];
      }
    for (int k = 0; k < m; ++k) {
      double q[3], qn = 0.0;
      for (int c = 0; c < 3; ++c) {
        q[c] = rdir[3 * (k + 1) + c] - rdir[3 * k + c];
        qn += q[c] * q[c];
      }
      qn = sqrt(qn);
      for (int c = 0; c < 3; ++c) u[3 * k + c] = q[c] / qn;
    }
    /* 6. rod tensions with |Q_k| = 1; 7. r <- r(T) */
    int it = 0;
    status = or_tension_solve(N, Dstep, rs, u, p->dt, p->tol, p->max_newton, T, rn, &it);
    if (iters) *iters = it;
    if (status == OR_OK) {
      memcpy(r, rn, sizeof(double) * n);
      if (T_out) memcpy(T_out, T, sizeof(double) * m);
      if (maxdev) {
        double md = 0.0;
        for (int k = 0; k < m; ++k) {
          double q2 = 0.0;
          for (int c = 0; c < 3; ++c) {
            double d = r[3 * (k + 1) + c] - r[3 * k + c];
            q2 += d * d;
          }
          double dv = fabs(sqrt(q2) - 1.0);
          if (dv > md) md = dv;
        }
        *maxdev = md;
      }
    }
  }
  free(D);
  free(L);
  free(y);
  free(rs);
  free(rn);
  free(u);
  free(T);
  free(z);
  free(w);
  free(rm);
  free(Dm);
  return status;
}

/* Fraenkel springs, Sec. 3 Eq. (3): F_k = K* (|Q_k| - 1) Q_k / |Q_k|, the
 * force that spring k exerts on bead k (and minus it on bead k + 1).  The
 * semi-implicit scheme of Sec. 3 takes spring k's own contribution to link
 * k implicitly:
 *   eqQ2: Y_k = Q_k + [explicit change of link k with every spring force at
 *         time t] + 2 dt F_k(t)  (the 2 dt F_k cancels the self term that
 *         D_kk = D_k+1,k+1 = I gives to the explicit change);
 *   Eq. (25): |Q_k'| = (2 dt K* + |Y_k|) / (2 dt K* + 1);
 *   Eq. (23): Q_k' = Y_k |Q_k'| / |Y_k|  (Q_k' parallel to Y_k).
 * The explicit change of the bead positions is the Euler step of Eq. (6):
 * dr_i = dt (kappa . r_i + sum_j D_ij Fb_j) + y_i, with the bead forces
 * Fb_i = F_i - F_{i-1}. */
void or_fraenkel_update(int N, const double* D, const double* kappa, double dt, double kspring,
                        const double* r, const double* y, double* r_new, double* T_out) {
  int n = 3 * N, m = N - 1;
  double* Fs = (double*)calloc(3 * (size_t)(m > 0 ? m : 1), sizeof(double));
  double* Fb = (double*)calloc((size_t)n, sizeof(double));
  double* v = (double*)calloc((size_t)n, sizeof(double));
  double* dr = (double*)calloc((size_t)n, sizeof(double));
  double* rp = (double*)calloc((size_t)n, sizeof(double));
  /* spring forces at time t and the bead forces */
  for (int k = 0; k < m; ++k) {
    double q[3], qn = 0.0;
    for (int c = 0; c < 3; ++c) {
      q[c] = r[3 * (k + 1) + c] - r[3 * k + c];
      qn += q[c] * q[c];
    }
    qn = sqrt(qn);
    for (int c = 0; c < 3; ++c) Fs[3 * k + c] = kspring * (qn - 1.0) / qn * q[c];
  }
  for (int i = 0; i < N; ++i)
    for (int c = 0; c < 3; ++c) {
      double f = 0.0;
      if (i < m) f += Fs[3 * i + c];
      if (i > 0) f -= Fs[3 * (i - 1) + c];
      Fb[3 * i + c] = f;
    }
  /* explicit bead step */
  or_gemv(n, D, Fb, v);
  for (int i = 0; i < N; ++i)
    for (int c = 0; c < 3; ++c) {
      double kr = kappa[3 * c] * r[3 * i] + kappa[3 * c + 1] * r[3 * i + 1] + kappa[3 * c + 2] * r[3 * i + 2];
      dr[3 * i + c] = dt * (kr + v[3 * i + c]) + y[3 * i + c];
    }
  /* new links (eqQ2, Eqs. (25), (23)) summed from bead 0 */
  for (int c = 0; c < 3; ++c) rp[c] = 0.0;
  for (int k = 0; k < m; ++k) {
    double Y[3], yn = 0.0;
    for (int c = 0; c < 3; ++c) {
      Y[c] = (r[3 * (k + 1) + c] - r[3 * k + c]) + (dr[3 * (k + 1) + c] - dr[3 * k + c]) +
             2.0 * dt * Fs[3 * k + c];
      yn += Y[c] * Y[c];
    }
    yn = sqrt(yn);
    double qn = (2.0 * dt * kspring + yn) / (2.0 * dt * kspring + 1.0);
    for (int c = 0; c < 3; ++c) rp[3 * (k + 1) + c] = rp[3 * k + c] + Y[c] * (qn / yn);
    if (T_out) T_out[k] = kspring * (qn - 1.0) / qn;
  }
  /* centre of mass: old centre plus the mean explicit displacement */
  for (int c = 0; c < 3; ++c) {
    double cm_old = 0.0, mdr = 0.0, mrp = 0.0;
    for (int i = 0; i < N; ++i) {
      cm_old += r[3 * i + c];
      mdr += dr[3 * i + c];
      mrp += rp[3 * i + c];
    }
    cm_old /= N;
    mdr /= N;
    mrp /= N;
    for (int i = 0; i < N; ++i) r_new[3 * i + c] = rp[3 * i + c] - mrp + cm_old + mdr;
  }
  free(Fs);
  free(Fb);
  free(v);
  free(dr);
  free(rp);
}

void or_run(const or_params* p, int n_chains, const int* Nc, double* r,
            int n_steps, const double* noise, double* T_out, int* status,
            int* iters, double* maxdev) {
  long* boff = (long*)malloc(sizeof(long) * (n_chains + 1));
  long* toff = (long*)malloc(sizeof(long) * (n_chains + 1));
  boff[0] = 0;
  toff[0] = 0;
  for (int c = 0; c < n_chains; ++c) {
    boff[c + 1] = boff[c] + Nc[c];
    toff[c + 1] = toff[c] + (Nc[c] - 1);
  }
  long sumN = boff[n_chains];
#pragma omp parallel for schedule(dynamic, 1)
  for (int c = 0; c < n_chains; ++c) {
    double md_all = 0.0;
    int st = OR_OK, it = 0;
    for (int s = 0; s < n_steps && st == OR_OK; ++s) {
      double md = 0.0;
      st = or_step(p, Nc[c], r + 3 * boff[c],
                   noise + 3 * ((long)s * sumN + boff[c]),
                   T_out ? T_out + toff[c] : NULL, &it, &md);
      if (md > md_all) md_all = md;
    }
    if (status) status[c] = st;
    if (iters) iters[c] = it;
    if (maxdev) maxdev[c] = md_all;
  }
  free(boff);
  free(toff);
}

/* Sec. 5 Eqs. (25)-(29), per chain (the ensemble average is the caller's). */
void or_observables(int N, const double* r, const double* T, double* out) {
  double cm[3] = {0, 0, 0};
  for (int i = 0; i < N; ++i)
    for (int c = 0; c < 3; ++c) cm[c] += r[3 * i + c] / N;
  double rg2 = 0.0;
  for (int i = 0; i < N; ++i)
    for (int c = 0; c < 3; ++c) {
      double d = r[3 * i + c] - cm[c];
      rg2 += d * d;
    }
  rg2 /= N;
  double R2 = 0.0;
  for (int c = 0; c < 3; ++c) {
    out[c] = r[3 * (N - 1) + c] - r[c];
    R2 += out[c] * out[c];
  }
  double md = 0.0;
  for (int k = 0; k + 1 < N; ++k) {
    double q2 = 0.0;
    for (int c = 0; c < 3; ++c) {
      double d = r[3 * (k + 1) + c] - r[3 * k + c];
      q2 += d * d;
    }
    double dv = fabs(sqrt(q2) - 1.0);
    if (dv > md) md = dv;
  }
  out[3] = R2;
  out[4] = rg2;
  out[5] = N > 1 ? sqrt(R2) / (N - 1) : 0.0;
  out[6] = md;
  out[7] = 0.0;
  /* Eq. (28): sum over rods of (force in rod k) (link vector k), tension part */
  double txx = 0.0, tyy = 0.0, tzz = 0.0, txy = 0.0;
  for (int k = 0; T && k + 1 < N; ++k) {
    double q[3];
    for (int c = 0; c < 3; ++c) q[c] = r[3 * (k + 1) + c] - r[3 * k + c];
    txx += T[k] * q[0] * q[0];
    tyy += T[k] * q[1] * q[1];
    tzz += T[k] * q[2] * q[2];
    txy += T[k] * q[0] * q[1];
  }
  out[8] = txx;
  out[9] = tyy;
  out[10] = tzz;
  out[11] = txy;
}
