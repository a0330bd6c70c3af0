/*
 * FP64 CPU oracle for the direct-sum boundary-integral Poisson-Boltzmann
 * method (centroid collocation).  TEST INFRASTRUCTURE ONLY: the tests, the
 * smoke check and the timed CPU baseline of the benchmark call it; the
 * library never does.  It shares no code with the CUDA path.
 *
 * Every function is the plain definition, in double precision, one pair at a
 * time, with each row summed serially in ascending source index.  OpenMP only
 * splits rows (targets), so results are identical for any thread count.
 *
 * Notation (per pair, target x_i with unit normal n_i, source x_j with n_j):
 *   d = x_i - x_j, r = |d|, G0 = 1/(4 pi r), Gk = exp(-kappa r)/(4 pi r)
 *   (Eq. of the Coulomb / screened-Coulomb potentials, Sec. 2.2.1).
 * Normal derivatives (Sec. 2.2.1): d/dnu_y = n_j . grad_y,
 *   d/dnu_x = +n_i . grad_x and d2/dnu_x dnu_y = +sum n_im n_jn d_xm d_yn.
 *   The printed formulas carry a leading minus on the two x-derivatives; that
 *   sign contradicts the derivation of the second boundary equation from the
 *   two Green representations with the outward normal, and with it the Born
 *   test diverges, so the plus sign is used (tests pin it by finite
 *   differences of G0 and Gk).
 * Kernels (Eqs. for K1..K4): K1 = G0 - Gk, K2 = eps dGk/dnu_y - dG0/dnu_y,
 *   K3 = dG0/dnu_x - (1/eps) dGk/dnu_x, K4 = d2Gk/dnu_x dnu_y - d2G0/dnu_x dnu_y,
 *   eps = eps_out / eps_in.
 * Discrete system (Eqs. 5-6, centroid collocation, j = i omitted):
 *   1/2 (1+eps) phi_i   - sum_{j!=i} [K1_ij psi_j + K2_ij phi_j] ds_j = S1_i
 *   1/2 (1+1/eps) psi_i - sum_{j!=i} [K3_ij psi_j + K4_ij phi_j] ds_j = S2_i
 *   with psi = dphi/dnu on the inner side and unknown u = [phi ; psi].
 * Sources (Eq. for S1, S2): S1 = (1/eps_in) sum_k q_k G0(x_i, y_k),
 *   S2 = (1/eps_in) sum_k q_k dG0(x_i, y_k)/dnu_x.
 * Solvation energy (Eq. for E_sol), in the units of the unknowns:
 *   E = 1/2 sum_k q_k sum_j ds_j [K1(y_k, x_j) psi_j + K2(y_k, x_j) phi_j].
 * Potential at a point p off the surface (Sec. 2.2.1):
 *   p inside (Eq. eq_inside):  phi(p) = sum_j ds_j [K1(p, x_j) psi_j + K2(p, x_j) phi_j] + S1(p);
 *   p outside (Eq. eqbim_2):   phi(p) = sum_j ds_j [-Gk(p, x_j) dphi2/dnu_j + dGk(p, x_j)/dnu_y phi_j]
 *   with dphi2/dnu = (eps_in / eps_out) psi (flux continuity across the surface).
 * Coulomb energy of the charges in the solute dielectric (the Coulomb part of
 * E_free, Eq. free_energy, without the infinite self terms):
 *   E_coul = 1/2 (1/eps_in) sum_{k != l} q_k q_l G0(y_k, y_l).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* G0, Gk and their derivatives written out from their definitions. */
static double g0(double r) { return 1.0 / (4.0 * ORC_PI * r); }
static double gk(double r, double kappa) { return exp(-kappa * r) / (4.0 * ORC_PI * r); }

/* radial derivative dG/dr of G0 and Gk */
static double g0_r(double r) { return -1.0 / (4.0 * ORC_PI * r * r); }
static double gk_r(double r, double kappa) {
  return -exp(-kappa * r) * (1.0 + kappa * r) / (4.0 * ORC_PI * r * r);
}
/* second radial derivative d2G/dr2 */
static double g0_rr(double r) { return 2.0 / (4.0 * ORC_PI * r * r * r); }
static double gk_rr(double r, double kappa) {
  double kr = kappa * r;
  return exp(-kr) * (2.0 + 2.0 * kr + kr * kr) / (4.0 * ORC_PI * r * r * r);
}

/*
 * For G(x, y) = g(|x - y|), with d = x - y, r = |d|, dhat = d / r:
 *   grad_x G = g'(r) dhat,  grad_y G = -g'(r) dhat
 *   d_xm d_yn G = -[ g''(r) dhat_m dhat_n + g'(r) (delta_mn - dhat_m dhat_n) / r ]
 */
static void pair_derivs(const double* x, const double* nx, const double* y, const double* ny,
                        double kappa, double out[8]) {
  double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
  double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  double dh[3] = {d[0] / r, d[1] / r, d[2] / r};
  double cx = nx ? nx[0] * dh[0] + nx[1] * dh[1] + nx[2] * dh[2] : 0.0; /* n_x . dhat */
  double cy = ny ? ny[0] * dh[0] + ny[1] * dh[1] + ny[2] * dh[2] : 0.0; /* n_y . dhat */
  double cxy = (nx && ny) ? nx[0] * ny[0] + nx[1] * ny[1] + nx[2] * ny[2] : 0.0;
  double G0 = g0(r), Gk = gk(r, kappa);
  double G0r = g0_r(r), Gkr = gk_r(r, kappa);
  double G0rr = g0_rr(r), Gkrr = gk_rr(r, kappa);
  out[0] = G0;
  out[1] = Gk;
  out[2] = -G0r * cy;                                      /* dG0/dnu_y = n_y . grad_y G0 */
  out[3] = -Gkr * cy;                                      /* dGk/dnu_y */
  out[4] = G0r * cx;                                       /* dG0/dnu_x = n_x . grad_x G0 */
  out[5] = Gkr * cx;                                       /* dGk/dnu_x */
  out[6] = -(G0rr * cx * cy + G0r * (cxy - cx * cy) / r); /* d2G0/dnu_x dnu_y */
  out[7] = -(Gkrr * cx * cy + Gkr * (cxy - cx * cy) / r); /* d2Gk/dnu_x dnu_y */
}

/* Green's functions and normal derivatives at one pair (for tests). */
void orc_green(const double* x, const double* nx, const double* y, const double* ny, double kappa,
               double out[8]) {
  pair_derivs(x, nx, y, ny, kappa, out);
}

/* K1..K4 at one pair, Eqs. for K1-K4. */
void orc_kernels(const double* x, const double* nx, const double* y, const double* ny, double eps,
                 double kappa, double K[4]) {
  double g[8];
  pair_derivs(x, nx, y, ny, kappa, g);
  K[0] = g[0] - g[1];
  K[1] = eps * g[3] - g[2];
  K[2] = g[4] - g[5] / eps;
  K[3] = g[7] - g[6];
}

/* b = [S1 ; S2], Eq. for the source terms.  nc charges at y with values q. */
void orc_source(int64_t n, const double* x, const double* nrm, int64_t nc, const double* y,
                const double* q, double eps_in, double* b) {
  int64_t i;
#pragma omp parallel for schedule(static)
  for (i = 0; i < n; ++i) {
    double s1 = 0.0, s2 = 0.0, g[8];
    for (int64_t k = 0; k < nc; ++k) {
      pair_derivs(x + 3 * i, nrm + 3 * i, y + 3 * k, NULL, 0.0, g);
      s1 += q[k] * g[0];
      s2 += q[k] * g[4];
    }
    b[i] = s1 / eps_in;
    b[n + i] = s2 / eps_in;
  }
}

/* out = A u, Eqs. 5-6.  u = [phi ; psi] (length 2n), out likewise. */
void orc_matvec(int64_t n, const double* x, const double* nrm, const double* area, double eps,
                double kappa, const double* u, double* out) {
  const double* phi = u;
  const double* psi = u + n;
  int64_t i;
#pragma omp parallel for schedule(static)
  for (i = 0; i < n; ++i) {
    double sp = 0.0, ss = 0.0, K[4];
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      orc_kernels(x + 3 * i, nrm + 3 * i, x + 3 * j, nrm + 3 * j, eps, kappa, K);
      sp += (K[0] * psi[j] + K[1] * phi[j]) * area[j];
      ss += (K[2] * psi[j] + K[3] * phi[j]) * area[j];
    }
    out[i] = 0.5 * (1.0 + eps) * phi[i] - sp;
    out[n + i] = 0.5 * (1.0 + 1.0 / eps) * psi[i] - ss;
  }
}

/* Selected rows of A u: out[r] = row rows[r] of orc_matvec (0 <= rows[r] < 2n). */
void orc_matvec_rows(int64_t n, const double* x, const double* nrm, const double* area, double eps,
                     double kappa, const double* u, int64_t nrows, const int64_t* rows, double* out) {
  const double* phi = u;
  const double* psi = u + n;
  int64_t r;
#pragma omp parallel for schedule(static)
  for (r = 0; r < nrows; ++r) {
    int64_t row = rows[r];
    int64_t i = row < n ? row : row - n;
    double acc = 0.0, K[4];
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      orc_kernels(x + 3 * i, nrm + 3 * i, x + 3 * j, nrm + 3 * j, eps, kappa, K);
      acc += (row < n ? (K[0] * psi[j] + K[1] * phi[j]) : (K[2] * psi[j] + K[3] * phi[j])) * area[j];
    }
    out[r] = row < n ? 0.5 * (1.0 + eps) * phi[i] - acc : 0.5 * (1.0 + 1.0 / eps) * psi[i] - acc;
  }
}

/* out = A^T w: the transpose of the operator of orc_matvec. */
void orc_matvec_t(int64_t n, const double* x, const double* nrm, const double* area, double eps,
                  double kappa, const double* w, double* out) {
  const double* wp = w;
  const double* ws = w + n;
  int64_t j;
#pragma omp parallel for schedule(static)
  for (j = 0; j < n; ++j) {
    double zp = 0.0, zs = 0.0, K[4];
    for (int64_t i = 0; i < n; ++i) {
      if (i == j) continue;
      orc_kernels(x + 3 * i, nrm + 3 * i, x + 3 * j, nrm + 3 * j, eps, kappa, K);
      zp += K[1] * wp[i] + K[3] * ws[i];
      zs += K[0] * wp[i] + K[2] * ws[i];
    }
    out[j] = 0.5 * (1.0 + eps) * wp[j] - area[j] * zp;
    out[n + j] = 0.5 * (1.0 + 1.0 / eps) * ws[j] - area[j] * zs;
  }
}

/* Selected rows of A^T w: out[r] = row rows[r] of orc_matvec_t (0 <= rows[r] < 2n). */
void orc_matvec_t_rows(int64_t n, const double* x, const double* nrm, const double* area, double eps,
                       double kappa, const double* w, int64_t nrows, const int64_t* rows, double* out) {
  const double* wp = w;
  const double* ws = w + n;
  int64_t r;
#pragma omp parallel for schedule(static)
  for (r = 0; r < nrows; ++r) {
    int64_t row = rows[r];
    int64_t j = row < n ? row : row - n;
    double z = 0.0, K[4];
    for (int64_t i = 0; i < n; ++i) {
      if (i == j) continue;
      orc_kernels(x + 3 * i, nrm + 3 * i, x + 3 * j, nrm + 3 * j, eps, kappa, K);
      z += row < n ? K[1] * wp[i] + K[3] * ws[i] : K[0] * wp[i] + K[2] * ws[i];
    }
    out[r] = row < n ? 0.5 * (1.0 + eps) * wp[j] - area[j] * z : 0.5 * (1.0 + 1.0 / eps) * ws[j] - area[j] * z;
  }
}

/*
 * Mat-vec sums of targets over a list of source records (the far-field
 * treecode of Sec. 2.2.3 sums each target over its near elements and the
 * proxy sources of its far clusters).  Record j has a position y_j, a_j
 * (ds psi for an element) and a vector m_j (ds phi n_j for an element).  K2
 * and K4 are linear in the source normal, so they are taken with m_j in its
 * place:
 *   out[2t]     = sum_j [K1(x_t, y_j) a_j + K2(x_t, y_j; m_j)]
 *   out[2t + 1] = sum_j [K3(x_t, y_j) a_j + K4(x_t, y_j; m_j)]
 * A record whose id equals the target's id (the self pair) is skipped.
 */
void orc_record_sums(int64_t nt, const double* xt, const double* nrm_t, const int64_t* tid, int64_t ns,
                     const double* ys, const double* a, const double* m, const int64_t* sid, double eps,
                     double kappa, double* out) {
  int64_t t;
#pragma omp parallel for schedule(static)
  for (t = 0; t < nt; ++t) {
    double sp = 0.0, ss = 0.0, K[4];
    for (int64_t j = 0; j < ns; ++j) {
      if (sid[j] == tid[t]) continue;
      orc_kernels(xt + 3 * t, nrm_t + 3 * t, ys + 3 * j, m + 3 * j, eps, kappa, K);
      sp += K[0] * a[j] + K[1];
      ss += K[2] * a[j] + K[3];
    }
    out[2 * t] = sp;
    out[2 * t + 1] = ss;
  }
}

/*
 * The same sums for A^T w.  Output element t (position x_t, normal n_t)
 * gathers column t of A: the entries of row element i depend on n_i only
 * through the kernels K3 and K4 (normal derivatives at x_i), linearly, so a
 * record j carries a position y_j, w_j (wphi of an element) and a vector
 * p_j (wpsi n_i of an element) in place of the row normal:
 *   out[2t]     = sum_j [K2(y_j, x_t) w_j + K4(y_j, x_t; p_j)]   (phi output)
 *   out[2t + 1] = sum_j [K1(y_j, x_t) w_j + K3(y_j, x_t; p_j)]   (psi output)
 * with the kernels evaluated with y_j as the collocation point and x_t as the
 * source, as in orc_matvec_t.  The output element's area multiplies the sums
 * outside.  A record whose id equals the target's id is skipped.
 */
void orc_record_sums_t(int64_t nt, const double* xt, const double* nrm_t, const int64_t* tid, int64_t ns,
                       const double* ys, const double* w, const double* p, const int64_t* sid, double eps,
                       double kappa, double* out) {
  int64_t t;
#pragma omp parallel for schedule(static)
  for (t = 0; t < nt; ++t) {
    double zp = 0.0, zs = 0.0, K[4];
    for (int64_t j = 0; j < ns; ++j) {
      if (sid[j] == tid[t]) continue;
      orc_kernels(ys + 3 * j, p + 3 * j, xt + 3 * t, nrm_t + 3 * t, eps, kappa, K);
      zp += K[1] * w[j] + K[3];
      zs += K[0] * w[j] + K[2];
    }
    out[2 * t] = zp;
    out[2 * t + 1] = zs;
  }
}

/* Dense A (2n x 2n, row-major), same entries as orc_matvec. */
void orc_assemble(int64_t n, const double* x, const double* nrm, const double* area, double eps,
                  double kappa, double* A) {
  int64_t m = 2 * n, i;
#pragma omp parallel for schedule(static)
  for (i = 0; i < n; ++i) {
    double K[4];
    for (int64_t j = 0; j < n; ++j) {
      double* r0 = A + i * m;
      double* r1 = A + (n + i) * m;
      if (j == i) {
        r0[j] = 0.5 * (1.0 + eps);
        r0[n + j] = 0.0;
        r1[j] = 0.0;
        r1[n + j] = 0.5 * (1.0 + 1.0 / eps);
        continue;
      }
      orc_kernels(x + 3 * i, nrm + 3 * i, x + 3 * j, nrm + 3 * j, eps, kappa, K);
      r0[j] = -K[1] * area[j];
      r0[n + j] = -K[0] * area[j];
      r1[j] = -K[3] * area[j];
      r1[n + j] = -K[2] * area[j];
    }
  }
}

/*
 * Gaussian elimination with partial pivoting, in place: A (m x m, row-major)
 * is overwritten, B (m x nrhs, row-major) becomes the solution.
 * Returns 0, or 1 + the column where a zero pivot appeared.
 */
int orc_gesv(int64_t m, double* A, int64_t nrhs, double* B) {
  for (int64_t k = 0; k < m; ++k) {
    int64_t p = k;
    double best = fabs(A[k * m + k]);
    for (int64_t r = k + 1; r < m; ++r) {
      double v = fabs(A[r * m + k]);
      if (v > best) { best = v; p = r; }
    }
    if (best == 0.0) return (int)(k + 1);
    if (p != k) {
      for (int64_t c = 0; c < m; ++c) { double t = A[k * m + c]; A[k * m + c] = A[p * m + c]; A[p * m + c] = t; }
      for (int64_t c = 0; c < nrhs; ++c) { double t = B[k * nrhs + c]; B[k * nrhs + c] = B[p * nrhs + c]; B[p * nrhs + c] = t; }
    }
    double piv = A[k * m + k];
    int64_t r;
#pragma omp parallel for schedule(static)
    for (r = k + 1; r < m; ++r) {
      double f = A[r * m + k] / piv;
      if (f == 0.0) continue;
      A[r * m + k] = 0.0;
      for (int64_t c = k + 1; c < m; ++c) A[r * m + c] -= f * A[k * m + c];
      for (int64_t c = 0; c < nrhs; ++c) B[r * nrhs + c] -= f * B[k * nrhs + c];
    }
  }
  for (int64_t k = m - 1; k >= 0; --k) {
    for (int64_t c = 0; c < nrhs; ++c) {
      double s = B[k * nrhs + c];
      for (int64_t j = k + 1; j < m; ++j) s -= A[k * m + j] * B[j * nrhs + c];
      B[k * nrhs + c] = s / A[k * m + k];
    }
  }
  return 0;
}

/*
 * Energy row c (length 2n): E = 1/2 c . u with
 *   c_phi_j = ds_j sum_k q_k K2(y_k, x_j),  c_psi_j = ds_j sum_k q_k K1(y_k, x_j)
 * (Eq. for E_sol; K2 at a charge uses only the source normal n_j).
 */
void orc_energy_row(int64_t n, const double* x, const double* nrm, const double* area, double eps,
                    double kappa, int64_t nc, const double* y, const double* q, double* c) {
  int64_t j;
#pragma omp parallel for schedule(static)
  for (j = 0; j < n; ++j) {
    double cp = 0.0, cs = 0.0, g[8];
    for (int64_t k = 0; k < nc; ++k) {
      pair_derivs(y + 3 * k, NULL, x + 3 * j, nrm + 3 * j, kappa, g);
      cp += q[k] * (eps * g[3] - g[2]);
      cs += q[k] * (g[0] - g[1]);
    }
    c[j] = area[j] * cp;
    c[n + j] = area[j] * cs;
  }
}

/*
 * Reaction potential at every charge, in the units of the unknowns:
 *   phi_reac(y_k) = sum_j ds_j [K1(y_k, x_j) psi_j + K2(y_k, x_j) phi_j]
 * and E_sol = 1/2 sum_k q_k phi_reac(y_k) (Eq. for E_sol).
 */
double orc_energy(int64_t n, const double* x, const double* nrm, const double* area, double eps,
                  double kappa, int64_t nc, const double* y, const double* q, const double* u,
                  double* phi_reac) {
  const double* phi = u;
  const double* psi = u + n;
  int64_t k;
#pragma omp parallel for schedule(static)
  for (k = 0; k < nc; ++k) {
    double s = 0.0, g[8];
    for (int64_t j = 0; j < n; ++j) {
      pair_derivs(y + 3 * k, NULL, x + 3 * j, nrm + 3 * j, kappa, g);
      s += area[j] * ((g[0] - g[1]) * psi[j] + (eps * g[3] - g[2]) * phi[j]);
    }
    phi_reac[k] = s;
  }
  double e = 0.0;
  for (k = 0; k < nc; ++k) e += q[k] * phi_reac[k];
  return 0.5 * e;
}

/*
 * Gradient of E = 1/2 c(q, y) . u with A u = b(q, y) and A^T lam = c:
 *   dE/dtheta = 1/2 [ (dc/dtheta) . u + lam . (db/dtheta) ].
 * Per charge k:
 *   dE/dq_k = 1/2 [ sum_j ds_j (K2(y_k,x_j) phi_j + K1(y_k,x_j) psi_j)
 *                 + (1/eps_in) sum_i (lam_phi_i G0(x_i,y_k) + lam_psi_i dG0(x_i,y_k)/dnu_x) ]
 *   dE/dy_k = 1/2 q_k [ sum_j ds_j (phi_j grad_y K2(y,x_j) + psi_j grad_y K1(y,x_j))
 *                 + (1/eps_in) sum_i (lam_phi_i grad_y G0(x_i,y) + lam_psi_i grad_y dG0(x_i,y)/dnu_x) ]
 * The gradients in y are taken by the chain rule of the radial derivatives:
 *   grad_y K1(y, x_j)    = (g0'(r) - gk'(r)) dhat,                    d = y - x_j
 *   grad_y K2(y, x_j)    = eps grad_y[-gk'(r) n_j.dhat] - grad_y[-g0'(r) n_j.dhat]
 *   grad_y G0(x_i, y)    = -g0'(r) dhat,                              d = x_i - y
 *   grad_y dG0/dnu_x     = grad_y[g0'(r) n_i.dhat]
 * with grad_z[h(r) n.dhat] = h'(r) (n.dhat) dhat + h(r) (n - (n.dhat) dhat) / r
 * for d = z - const, and the sign flipped when d = const - z.
 */
static void grad_radial_dot(double h, double hr, const double* nv, const double* dh, double r,
                            double out[3]) {
  double c = nv[0] * dh[0] + nv[1] * dh[1] + nv[2] * dh[2];
  for (int m = 0; m < 3; ++m) out[m] = hr * c * dh[m] + h * (nv[m] - c * dh[m]) / r;
}

void orc_grad(int64_t n, const double* x, const double* nrm, const double* area, double eps,
              double kappa, double eps_in, int64_t nc, const double* y, const double* q,
              const double* u, const double* lam, double* dE_dq, double* dE_dy) {
  const double* phi = u;
  const double* psi = u + n;
  const double* lp = lam;
  const double* ls = lam + n;
  int64_t k;
#pragma omp parallel for schedule(static)
  for (k = 0; k < nc; ++k) {
    const double* yk = y + 3 * k;
    double sq = 0.0, gy[3] = {0.0, 0.0, 0.0};
    /* energy-row part, d = y_k - x_j */
    for (int64_t j = 0; j < n; ++j) {
      const double* xj = x + 3 * j;
      const double* nj = nrm + 3 * j;
      double d[3] = {yk[0] - xj[0], yk[1] - xj[1], yk[2] - xj[2]};
      double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      double dh[3] = {d[0] / r, d[1] / r, d[2] / r};
      double cj = nj[0] * dh[0] + nj[1] * dh[1] + nj[2] * dh[2];
      double K1 = g0(r) - gk(r, kappa);
      double K2 = eps * (-gk_r(r, kappa) * cj) - (-g0_r(r) * cj);
      sq += area[j] * (K2 * phi[j] + K1 * psi[j]);
      double a0[3], ak[3];
      grad_radial_dot(-g0_r(r), -g0_rr(r), nj, dh, r, a0);
      grad_radial_dot(-gk_r(r, kappa), -gk_rr(r, kappa), nj, dh, r, ak);
      double k1r = g0_r(r) - gk_r(r, kappa);
      for (int m = 0; m < 3; ++m)
        gy[m] += area[j] * (phi[j] * (eps * ak[m] - a0[m]) + psi[j] * k1r * dh[m]);
    }
    /* source-column part, d = x_i - y_k */
    double sl = 0.0, gl[3] = {0.0, 0.0, 0.0};
    for (int64_t i = 0; i < n; ++i) {
      const double* xi = x + 3 * i;
      const double* ni = nrm + 3 * i;
      double d[3] = {xi[0] - yk[0], xi[1] - yk[1], xi[2] - yk[2]};
      double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      double dh[3] = {d[0] / r, d[1] / r, d[2] / r};
      double ci = ni[0] * dh[0] + ni[1] * dh[1] + ni[2] * dh[2];
      sl += lp[i] * g0(r) + ls[i] * g0_r(r) * ci;
      double b0[3];
      grad_radial_dot(g0_r(r), g0_rr(r), ni, dh, r, b0);
      for (int m = 0; m < 3; ++m) gl[m] += -lp[i] * g0_r(r) * dh[m] - ls[i] * b0[m];
    }
    dE_dq[k] = 0.5 * (sq + sl / eps_in);
    for (int m = 0; m < 3; ++m) dE_dy[3 * k + m] = 0.5 * q[k] * (gy[m] + gl[m] / eps_in);
  }
}

/* Potential at np points p (units of the unknowns), Eq. eq_inside for
 * inside != 0 (then the nc charges y, q enter through S1) and Eq. eqbim_2
 * otherwise.  u = [phi ; psi] on the n elements. */
void orc_potential(int64_t n, const double* x, const double* nrm, const double* area, double eps,
                   double kappa, const double* u, int64_t np, const double* p, int inside, int64_t nc,
                   const double* y, const double* q, double eps_in, double* out) {
  const double* phi = u;
  const double* psi = u + n;
  int64_t i;
#pragma omp parallel for schedule(static)
  for (i = 0; i < np; ++i) {
    double s = 0.0, g[8];
    for (int64_t j = 0; j < n; ++j) {
      pair_derivs(p + 3 * i, NULL, x + 3 * j, nrm + 3 * j, kappa, g);
      if (inside)
        s += area[j] * ((g[0] - g[1]) * psi[j] + (eps * g[3] - g[2]) * phi[j]);
      else
        s += area[j] * (-g[1] * psi[j] / eps + g[3] * phi[j]);
    }
    if (inside) {
      double s1 = 0.0;
      for (int64_t k = 0; k < nc; ++k) {
        pair_derivs(p + 3 * i, NULL, y + 3 * k, NULL, 0.0, g);
        s1 += q[k] * g[0];
      }
      s += s1 / eps_in;
    }
    out[i] = s;
  }
}

/* E_coul = 1/2 (1/eps_in) sum_{k != l} q_k q_l G0(y_k, y_l), units of the unknowns. */
double orc_coulomb(int64_t nc, const double* y, const double* q, double eps_in) {
  double e = 0.0;
  for (int64_t k = 0; k < nc; ++k)
    for (int64_t l = 0; l < nc; ++l) {
      if (l == k) continue;
      double d[3] = {y[3 * k] - y[3 * l], y[3 * k + 1] - y[3 * l + 1], y[3 * k + 2] - y[3 * l + 2]};
      e += q[k] * q[l] * g0(sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]));
    }
  return 0.5 * e / eps_in;
}
