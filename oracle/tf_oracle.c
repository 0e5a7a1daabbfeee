/*
 * tf_oracle.c -- plain FP64 CPU oracle of the Newton--ADI thin-film time step.
 *
 * TEST INFRASTRUCTURE ONLY: the CUDA library never includes, links or calls
 * this file; only tests, the smoke check and the benchmark's CPU-baseline leg
 * do.  It is written for a reader checking it against the paper by eye:
 * every quantity is formed the way the paper defines it, one face flux or one
 * matrix entry at a time, with no fusion or reordering beyond that.
 * Compile without FMA contraction (-ffp-contract=off).
 *
 * Paper: Lam, Cummings & Kondic, "Computing dynamics of thin films via large
 * scale GPU-based simulations".  Readings of silent or garbled passages:
 *   - f1 = h^3 Pi'(h) (not divided by C): reproduces the printed LSA values.
 *   - J_x holds every derivative of the x-face fluxes except the one through
 *     the y-part of the Laplacian (that part is the neglected mixed term J_xy,
 *     eq. DirectionSplit); the coefficient-derivative terms use the full
 *     explicit Laplacian.  J_y likewise with x and y exchanged.
 *   - ADI order: x-lines first, then y-lines: (I+th dt Jx) w = -G,
 *     (I+th dt Jy) v = w, u_{k+1} = u_k + v.
 *   - Face mobility = mean of the two adjacent cell-centre values of f.
 *   - No-flux walls by even reflection: u_{-1} = u_0, u_{-2} = u_1, which
 *     makes every wall-face flux exactly zero.
 */
#include "tf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(M, i, j) ((size_t)(j) * (size_t)(M)->nx + (size_t)(i))

static double ipow(double x, int k) {
  double r = 1.0;
  for (int i = 0; i < k; ++i) r *= x;
  return r;
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* kappa = (1 - cos theta_c) / (b M), M = (n-m)/((m-1)(n-1)): the strength of
 * the power-law disjoining pressure that gives contact angle theta_c. */
double or_kappa_from_contact_angle(double th, double b, int n, int m) {
  double Mf = (double)(n - m) / ((double)(m - 1) * (double)(n - 1));
  return (1.0 - cos(th)) / (b * Mf);
}

/* Disjoining pressure and its first two derivatives, Sec. Thin Film Models.
 *
 * Power law: Pi = kappa[r^n - r^m], r = b/h, so Pi' = kappa[m r^m - n r^n]/h
 * and Pi'' = kappa[n(n+1) r^n - m(m+1) r^m]/h^2.
 *
 * NLC (eqs. DisjPressNLC, mh_model): Pi = K[r^3 - r^2] + (N/2) q^2 with
 * q = m(h)/h = g(h) h/(h^2 + beta^2), g = [1 + tanh(s)]/2, s = (h - 2b)/w:
 *   g' = (1 - tanh^2 s)/(2w),  g'' = -tanh(s)(1 - tanh^2 s)/w^2,
 *   q' = g' h/D + g (beta^2 - h^2)/D^2,  D = h^2 + beta^2,
 *   q'' = g'' h/D + 2 g' (beta^2 - h^2)/D^2 + g 2h(h^2 - 3 beta^2)/D^3,
 *   (N/2 q^2)' = N q q',  (N/2 q^2)'' = N (q'^2 + q q'').
 *
 * Polymer (eq. DisjPressPolymer): Pi = -psi' with
 * psi = Cp h^-8 - A1/(12 pi) h^-2 + (A1 - A2)/(12 pi) (h + d)^-2:
 *   Pi   =   8 Cp h^-9  -  A1/(6 pi) h^-3 + (A1 - A2)/(6 pi) (h + d)^-3,
 *   Pi'  = -72 Cp h^-10 +  A1/(2 pi) h^-4 - (A1 - A2)/(2 pi) (h + d)^-4,
 *   Pi'' = 720 Cp h^-11 - 2 A1/pi   h^-5 + 2 (A1 - A2)/pi   (h + d)^-5. */
void or_pi(const or_model* M, double h, double* pi, double* dpi, double* d2pi) {
  if (M->model == OR_MODEL_POLYMER) {
    const double PI = 3.14159265358979323846;
    double A1 = M->pol_A1, A12 = M->pol_A1 - M->pol_A2, Cp = M->pol_C, e = h + M->pol_d;
    *pi = 8.0 * Cp / ipow(h, 9) - A1 / (6.0 * PI * ipow(h, 3)) + A12 / (6.0 * PI * ipow(e, 3));
    *dpi = -72.0 * Cp / ipow(h, 10) + A1 / (2.0 * PI * ipow(h, 4)) - A12 / (2.0 * PI * ipow(e, 4));
    *d2pi = 720.0 * Cp / ipow(h, 11) - 2.0 * A1 / (PI * ipow(h, 5)) + 2.0 * A12 / (PI * ipow(e, 5));
    return;
  }
  if (M->model == OR_MODEL_NLC) {
    double r = M->b / h, K = M->nlc_K, N = M->nlc_N, w = M->nlc_w, be2 = M->nlc_beta * M->nlc_beta;
    double p1 = K * (r * r * r - r * r);
    double dp1 = K * (2.0 * r * r - 3.0 * r * r * r) / h;
    double d2p1 = K * (12.0 * r * r * r - 6.0 * r * r) / (h * h);
    double t = tanh((h - 2.0 * M->b) / w), sech2 = 1.0 - t * t;
    double g = 0.5 * (1.0 + t), dg = sech2 / (2.0 * w), d2g = -t * sech2 / (w * w);
    double D = h * h + be2;
    double q = g * h / D;
    double dq = dg * h / D + g * (be2 - h * h) / (D * D);
    double d2q = d2g * h / D + 2.0 * dg * (be2 - h * h) / (D * D) + g * 2.0 * h * (h * h - 3.0 * be2) / (D * D * D);
    *pi = p1 + 0.5 * N * q * q;
    *dpi = dp1 + N * q * dq;
    *d2pi = d2p1 + N * (dq * dq + q * d2q);
    return;
  }
  double r = M->b / h;
  double rn = ipow(r, M->n), rm = ipow(r, M->m);
  double n = (double)M->n, m = (double)M->m;
  *pi = M->kappa * (rn - rm);
  *dpi = M->kappa * (m * rm - n * rn) / h;
  *d2pi = M->kappa * (n * (n + 1.0) * rn - m * (m + 1.0) * rm) / (h * h);
}

double or_dpi(const or_model* M, double h) {
  double p, d1, d2;
  or_pi(M, h, &p, &d1, &d2);
  return d1;
}

/* Sec. Thin Film Models, eq. GeneralDisPreForm: f0 = C h^3, f1 = h^3 Pi'(h).
 * Derivatives: f0' = 3 C h^2, f1' = 3 h^2 Pi' + h^3 Pi''. */
void or_mobility(const or_model* M, double h, double* f0, double* f1,
                 double* df0, double* df1) {
  if (M->model == OR_MODEL_LINEAR) {
    *f0 = M->c0;
    *f1 = M->c1;
    *df0 = 0.0;
    *df1 = 0.0;
    return;
  }
  double pi, dpi, d2pi;
  or_pi(M, h, &pi, &dpi, &d2pi);
  *f0 = M->cap_C * h * h * h;
  *df0 = 3.0 * M->cap_C * h * h;
  *f1 = h * h * h * dpi;
  *df1 = 3.0 * h * h * dpi + h * h * h * d2pi;
}

/* Sec. Linear Stability Analysis, read as sigma = q^2 (f1 - f0 q^2):
 * q_m = sqrt(f1/(2 f0)), sigma_m = f1^2/(4 f0). */
void or_lsa(const or_model* M, double h0, double* qm, double* sigma_m) {
  double f0, f1, d0, d1;
  or_mobility(M, h0, &f0, &f1, &d0, &d1);
  if (f1 <= 0.0) {
    *qm = 0.0;
    *sigma_m = 0.0;
    return;
  }
  *qm = sqrt(f1 / (2.0 * f0));
  *sigma_m = f1 * f1 / (4.0 * f0);
}

/* The linear operator L = lap u at cell centres (Sec. Flux Discretization,
 * item 2), five points, walls by even reflection (Sec. Boundary Conditions):
 * a missing neighbour equals the cell itself and contributes nothing. */
void or_laplacian(const or_model* M, const double* u, double* lap) {
  const int nx = M->nx, ny = M->ny;
  const double inv_ds2 = 1.0 / (M->ds * M->ds);
#pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; ++j) {
    for (int i = 0; i < nx; ++i) {
      double c = u[IDX(M, i, j)];
      double s = 0.0;
      if (i + 1 < nx) s += u[IDX(M, i + 1, j)] - c;
      if (i > 0) s += u[IDX(M, i - 1, j)] - c;
      if (j + 1 < ny) s += u[IDX(M, i, j + 1)] - c;
      if (j > 0) s += u[IDX(M, i, j - 1)] - c;
      lap[IDX(M, i, j)] = s * inv_ds2;
    }
  }
}

/* One face flux F = fbar0 (L_q - L_p)/ds + fbar1 (u_q - u_p)/ds between cells
 * p and q (q the neighbour in +x or +y), with fbar the mean of the two
 * cell-centre values (Sec. Flux Discretization, item 3). */
static double face_flux(const or_model* M, double up, double uq, double lp,
                        double lq) {
  double f0p, f1p, f0q, f1q, d0, d1;
  or_mobility(M, up, &f0p, &f1p, &d0, &d1);
  or_mobility(M, uq, &f0q, &f1q, &d0, &d1);
  double fbar0 = 0.5 * (f0p + f0q);
  double fbar1 = 0.5 * (f1p + f1q);
  return fbar0 * (lq - lp) / M->ds + fbar1 * (uq - up) / M->ds;
}

/* eq. GovEqnCell2 / eq. FluxDiffOper:
 * D_ij = [F_x(i+1/2) - F_x(i-1/2) + F_y(j+1/2) - F_y(j-1/2)] / ds,
 * with zero flux through the walls.  Each interior face flux is formed once
 * (arrays Fx, Fy) and then differenced. */
void or_operator_D(const or_model* M, const double* u, double* D) {
  const int nx = M->nx, ny = M->ny;
  const size_t N = (size_t)nx * (size_t)ny;
  double* lap = (double*)malloc(N * sizeof(double));
  /* Fx[j*(nx-1) + i] is the flux through the face between (i,j), (i+1,j);
   * Fy[j*nx + i] the one between (i,j), (i,j+1). */
  size_t nfx = (size_t)(nx > 1 ? nx - 1 : 0) * (size_t)ny;
  size_t nfy = (size_t)nx * (size_t)(ny > 1 ? ny - 1 : 0);
  double* Fx = (double*)malloc((nfx ? nfx : 1) * sizeof(double));
  double* Fy = (double*)malloc((nfy ? nfy : 1) * sizeof(double));
  or_laplacian(M, u, lap);
#pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i + 1 < nx; ++i)
      Fx[(size_t)j * (nx - 1) + i] =
          face_flux(M, u[IDX(M, i, j)], u[IDX(M, i + 1, j)],
                    lap[IDX(M, i, j)], lap[IDX(M, i + 1, j)]);
#pragma omp parallel for schedule(static)
  for (int j = 0; j < ny - 1; ++j)
    for (int i = 0; i < nx; ++i)
      Fy[(size_t)j * nx + i] =
          face_flux(M, u[IDX(M, i, j)], u[IDX(M, i, j + 1)],
                    lap[IDX(M, i, j)], lap[IDX(M, i, j + 1)]);
#pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; ++j) {
    for (int i = 0; i < nx; ++i) {
      double fe = (i + 1 < nx) ? Fx[(size_t)j * (nx - 1) + i] : 0.0;
      double fw = (i > 0) ? Fx[(size_t)j * (nx - 1) + i - 1] : 0.0;
      double fn = (j + 1 < ny) ? Fy[(size_t)j * nx + i] : 0.0;
      double fs = (j > 0) ? Fy[(size_t)(j - 1) * nx + i] : 0.0;
      D[IDX(M, i, j)] = (fe - fw + fn - fs) / M->ds;
    }
  }
  free(lap);
  free(Fx);
  free(Fy);
}

/* eq. TrapRule with weight theta: the explicit, iteration-independent part
 * b^n = (I - (1-theta) dt D) u^n, formed once per time step. */
void or_explicit_part(const or_model* M, const double* un, double dt, double* bn) {
  const size_t N = (size_t)M->nx * (size_t)M->ny;
  double* D = (double*)malloc(N * sizeof(double));
  or_operator_D(M, un, D);
  for (size_t p = 0; p < N; ++p) bn[p] = un[p] - (1.0 - M->theta) * dt * D[p];
  free(D);
}

/* The Newton residual (Sec. Newton Iterative Scheme):
 * G(u_k) = (I + theta dt D) u_k - b^n. */
void or_residual(const or_model* M, const double* uk, const double* bn,
                 double dt, double* G) {
  const size_t N = (size_t)M->nx * (size_t)M->ny;
  double* D = (double*)malloc(N * sizeof(double));
  or_operator_D(M, uk, D);
  for (size_t p = 0; p < N; ++p) G[p] = uk[p] + M->theta * dt * D[p] - bn[p];
  free(D);
}

/* d(Lxx_c)/du_col for the one-directional part of the Laplacian along a line
 * of n cells, walls by reflection:
 * Lxx_c = [(u_{c+1}-u_c)[c<n-1] - (u_c-u_{c-1})[c>0]] / ds^2. */
static double dlap1_du(int c, int col, int n, double inv_ds2) {
  if (col == c + 1) return (c < n - 1) ? inv_ds2 : 0.0;
  if (col == c - 1) return (c > 0) ? inv_ds2 : 0.0;
  if (col == c) return -(double)((c < n - 1) + (c > 0)) * inv_ds2;
  return 0.0;
}

/* Band of I + theta dt J along one line of n cells.  u, lap: line values
 * (lap the full two-dimensional Laplacian); stride: distance between
 * consecutive line cells in the arrays.  For each interior face between line
 * cells p and q = p+1, the derivative of F = fbar0 gL + fbar1 gU with respect
 * to u_{p-1..p+2} is, term by term (Sec. Flux Discretization with the J_x /
 * J_y split of eq. DirectionSplit):
 *   d fbar0 = f0'/2 du (at p and q)  times gL = (L_q - L_p)/ds, explicit;
 *   d fbar1 = f1'/2 du (at p and q)  times gU = (u_q - u_p)/ds, explicit;
 *   fbar0 (dLxx_q - dLxx_p)/ds       (along-line third difference);
 *   fbar1 (du_q - du_p)/ds.
 * Row p receives +dF/ds, row q receives -dF/ds (D = (F_+ - F_-)/ds). */
static void line_band(const or_model* M, int n, const double* u,
                      const double* lap, size_t stride, double dt,
                      double* band) {
  const double ds = M->ds, inv_ds2 = 1.0 / (ds * ds);
  const double tdt = M->theta * dt;
  for (int r = 0; r < n; ++r) {
    for (int c = 0; c < 5; ++c) band[5 * r + c] = 0.0;
    band[5 * r + 2] = 1.0;
  }
  for (int p = 0; p + 1 < n; ++p) {
    int q = p + 1;
    double up = u[(size_t)p * stride], uq = u[(size_t)q * stride];
    double lp = lap[(size_t)p * stride], lq = lap[(size_t)q * stride];
    double f0p, f1p, d0p, d1p, f0q, f1q, d0q, d1q;
    or_mobility(M, up, &f0p, &f1p, &d0p, &d1p);
    or_mobility(M, uq, &f0q, &f1q, &d0q, &d1q);
    double fbar0 = 0.5 * (f0p + f0q), fbar1 = 0.5 * (f1p + f1q);
    double gL = (lq - lp) / ds, gU = (uq - up) / ds;
    double dF[4]; /* columns p-1, p, p+1, p+2 */
    for (int a = 0; a < 4; ++a) {
      int col = p - 1 + a;
      double v = fbar0 * (dlap1_du(q, col, n, inv_ds2) - dlap1_du(p, col, n, inv_ds2)) / ds;
      if (col == p) v += 0.5 * d0p * gL + 0.5 * d1p * gU - fbar1 / ds;
      if (col == q) v += 0.5 * d0q * gL + 0.5 * d1q * gU + fbar1 / ds;
      dF[a] = v;
    }
    for (int a = 0; a < 4; ++a) {
      int col = p - 1 + a;
      if (col < 0 || col >= n) continue;
      band[5 * p + (col - p + 2)] += tdt * dF[a] / ds;
      band[5 * q + (col - q + 2)] -= tdt * dF[a] / ds;
    }
  }
}

void or_jx_row(const or_model* M, const double* uk, double dt, int j, double* band) {
  const size_t N = (size_t)M->nx * (size_t)M->ny;
  double* lap = (double*)malloc(N * sizeof(double));
  or_laplacian(M, uk, lap);
  line_band(M, M->nx, uk + IDX(M, 0, j), lap + IDX(M, 0, j), 1, dt, band);
  free(lap);
}

void or_jy_col(const or_model* M, const double* uk, double dt, int i, double* band) {
  const size_t N = (size_t)M->nx * (size_t)M->ny;
  double* lap = (double*)malloc(N * sizeof(double));
  or_laplacian(M, uk, lap);
  line_band(M, M->ny, uk + i, lap + i, (size_t)M->nx, dt, band);
  free(lap);
}

/* Banded Gaussian elimination without pivoting (lower and upper bandwidth
 * 2), then back substitution: the LU solve of eq. LUFactorization. */
int or_penta_solve(int n, const double* band, const double* rhs, double* x) {
  double* A = (double*)malloc((size_t)5 * (n > 0 ? n : 1) * sizeof(double));
  double* y = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  memcpy(A, band, (size_t)5 * n * sizeof(double));
  memcpy(y, rhs, (size_t)n * sizeof(double));
#define AT(r, c) A[5 * (r) + ((c) - (r) + 2)]
  int status = 0;
  for (int k = 0; k < n && !status; ++k) {
    double piv = AT(k, k);
    if (piv == 0.0 || !isfinite(piv)) {
      status = 3;
      break;
    }
    for (int r = k + 1; r <= k + 2 && r < n; ++r) {
      double l = AT(r, k) / piv;
      for (int c = k; c <= k + 2 && c < n; ++c) AT(r, c) -= l * AT(k, c);
      y[r] -= l * y[k];
    }
  }
  if (!status) {
    for (int k = n - 1; k >= 0; --k) {
      double s = y[k];
      for (int c = k + 1; c <= k + 2 && c < n; ++c) s -= AT(k, c) * x[c];
      x[k] = s / AT(k, k);
    }
  }
#undef AT
  free(A);
  free(y);
  return status;
}

/* eqs. JacobianSystem1-3, x-lines first:
 *   (I + theta dt J_x) w = -G(u_k)     for every row j,
 *   (I + theta dt J_y) v = w           for every column i,
 *   u_{k+1} = u_k + v,  err = max |v / u_k|   (eq. NewtonError). */
int or_newton_iteration(const or_model* M, const double* uk, const double* bn,
                        double dt, double* G, double* w, double* v,
                        double* unew, double* err, double* gnorm) {
  const int nx = M->nx, ny = M->ny;
  const size_t N = (size_t)nx * (size_t)ny;
  double* lap = (double*)malloc(N * sizeof(double));
  int status = 0;
  or_residual(M, uk, bn, dt, G);
  or_laplacian(M, uk, lap);
  double gmax = 0.0;
  for (size_t p = 0; p < N; ++p) gmax = fmax(gmax, fabs(G[p]));
#pragma omp parallel
  {
    int lmax = nx > ny ? nx : ny;
    double* band = (double*)malloc((size_t)5 * lmax * sizeof(double));
    double* rhs = (double*)malloc((size_t)lmax * sizeof(double));
    double* sol = (double*)malloc((size_t)lmax * sizeof(double));
#pragma omp for schedule(static)
    for (int j = 0; j < ny; ++j) {
      line_band(M, nx, uk + IDX(M, 0, j), lap + IDX(M, 0, j), 1, dt, band);
      for (int i = 0; i < nx; ++i) rhs[i] = -G[IDX(M, i, j)];
      int s = or_penta_solve(nx, band, rhs, sol);
      if (s) {
#pragma omp atomic write
        status = s;
      }
      for (int i = 0; i < nx; ++i) w[IDX(M, i, j)] = s ? 0.0 : sol[i];
    }
#pragma omp for schedule(static)
    for (int i = 0; i < nx; ++i) {
      line_band(M, ny, uk + i, lap + i, (size_t)nx, dt, band);
      for (int j = 0; j < ny; ++j) rhs[j] = w[IDX(M, i, j)];
      int s = or_penta_solve(ny, band, rhs, sol);
      if (s) {
#pragma omp atomic write
        status = s;
      }
      for (int j = 0; j < ny; ++j) v[IDX(M, i, j)] = s ? 0.0 : sol[j];
    }
    free(band);
    free(rhs);
    free(sol);
  }
  double e = 0.0;
  for (size_t p = 0; p < N; ++p) {
    unew[p] = uk[p] + v[p];
    double r = fabs(v[p] / uk[p]);
    if (!(r <= e)) e = r; /* a NaN ratio propagates */
  }
  free(lap);
  *err = e;
  *gnorm = gmax;
  return status;
}

/* Neumaier-compensated sum of the grid (the mass diagnostic of
 * Sec. Conservation of Mass, before the 1/(IJ) factor). */
static double grid_mass(const double* u, size_t N) {
  double s = 0.0, c = 0.0;
  for (size_t p = 0; p < N; ++p) {
    double t = s + u[p];
    if (fabs(s) >= fabs(u[p]))
      c += (s - t) + u[p];
    else
      c += (u[p] - t) + s;
    s = t;
  }
  return s + c;
}

static int grid_positive_finite(const double* u, size_t N, double* hmin) {
  double mn = INFINITY;
  int ok = 1;
  for (size_t p = 0; p < N; ++p) {
    if (!(u[p] > 0.0) || !isfinite(u[p])) ok = 0;
    if (u[p] < mn) mn = u[p];
  }
  *hmin = mn;
  return ok;
}

/* The inner loop of Fig. FlowChartTime: u_(0) = u^n, iterate eqs.
 * JacobianSystem1-3 until eq. NewtonError holds (or K iterations fail). */
int or_step(const or_model* M, const or_control* C, const double* un,
            double dt, double* unew, or_step_info* info) {
  const size_t N = (size_t)M->nx * (size_t)M->ny;
  double* bn = (double*)malloc(N * sizeof(double));
  double* uk = (double*)malloc(N * sizeof(double));
  double* G = (double*)malloc(N * sizeof(double));
  double* w = (double*)malloc(N * sizeof(double));
  double* v = (double*)malloc(N * sizeof(double));
  or_explicit_part(M, un, dt, bn);
  memcpy(uk, un, N * sizeof(double));
  int status = 1, it = 0;
  double err = 0.0, gnorm = 0.0, hmin = 0.0;
  int kmax = C->fixed_iter > 0 ? C->fixed_iter : C->max_iter;
  for (int k = 0; k < kmax; ++k) {
    int s = or_newton_iteration(M, uk, bn, dt, G, w, v, unew, &err, &gnorm);
    it = k + 1;
    if (s) {
      status = s;
      break;
    }
    if (!grid_positive_finite(unew, N, &hmin)) {
      status = 2;
      break;
    }
    if (C->fixed_iter > 0) {
      if (it == C->fixed_iter) {
        status = 0;
        break;
      }
    } else if (err < C->tol) {
      status = 0;
      break;
    }
    memcpy(uk, unew, N * sizeof(double));
  }
  info->status = status;
  info->iterations = it;
  info->err = err;
  info->gnorm = gnorm;
  info->mass = grid_mass(unew, N);
  grid_positive_finite(unew, N, &hmin);
  info->hmin = hmin;
  free(bn);
  free(uk);
  free(G);
  free(w);
  free(v);
  return status;
}

/* Fig. FlowChartTime: accept -> advance t, grow dt by dt_grow after
 * grow_after consecutive accepted steps (bounded by dt_max); reject -> shrink
 * dt by dt_shrink and fail below dt_min.  The final step is clipped to land
 * on t_end.  In replay mode every attempt is one accepted step of the
 * recorded sequence, with its step size and (optionally) iteration count. */
int or_advance(const or_model* M, const or_control* C, double* h, double t0,
               double t_end, double dt0, int max_attempts,
               const double* dt_replay, const int* iter_replay,
               or_record* records, double* t_out, double* dt_out, int* status) {
  const size_t N = (size_t)M->nx * (size_t)M->ny;
  double* hn = (double*)malloc(N * sizeof(double));
  double t = t0, dt = dt0;
  int streak = 0, a = 0;
  *status = 1;
  while (a < max_attempts) {
    if (t >= t_end) {
      *status = 0;
      break;
    }
    or_control c = *C;
    double step_dt;
    int last = 0;
    if (dt_replay) {
      step_dt = dt_replay[a];
      if (iter_replay) c.fixed_iter = iter_replay[a];
    } else if (t_end - t <= dt) {
      step_dt = t_end - t;
      last = 1;
    } else {
      step_dt = dt;
    }
    or_step_info info;
    int s = or_step(M, &c, h, step_dt, hn, &info);
    if (records) {
      or_record* r = &records[a];
      r->t = t;
      r->dt = step_dt;
      r->accepted = (s == 0);
      r->iterations = info.iterations;
      r->status = s;
      r->err = info.err;
      r->gnorm = info.gnorm;
      r->mass = info.mass;
      r->hmin = info.hmin;
    }
    ++a;
    if (s == 0) {
      memcpy(h, hn, N * sizeof(double));
      t = last ? t_end : t + step_dt;
      if (!dt_replay && ++streak >= C->grow_after) {
        dt = fmin(dt * C->dt_grow, C->dt_max);
        streak = 0;
      }
      if (C->rupture_h > 0.0 && info.hmin < C->rupture_h) {
        *status = 3;
        break;
      }
    } else {
      if (dt_replay) { /* a replayed step must succeed; report and stop */
        *status = 2;
        break;
      }
      streak = 0;
      dt = step_dt * C->dt_shrink; /* shrink the step actually tried */
      if (dt < C->dt_min) {
        *status = 2;
        break;
      }
    }
  }
  if (a >= max_attempts && *status == 1 && t >= t_end) *status = 0;
  *t_out = t;
  *dt_out = dt;
  free(hn);
  return a;
}
