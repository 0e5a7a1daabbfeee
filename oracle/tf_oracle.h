/*
 * tf_oracle.h -- plain FP64 CPU oracle of the Newton--ADI thin-film time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library
 * and its Python binding) may include, link, load or call this code.  Only
 * the tests, the smoke check and the CPU-baseline leg of the benchmark use it.
 *
 * What it computes (Lam, Cummings & Kondic, "Computing dynamics of thin films
 * via large scale GPU-based simulations"):
 *   u_t + div[ f0(u) grad lap u + f1(u) grad u ] = 0       (eq. GoverningEquation)
 *   f0 = C h^3, f1 = h^3 Pi'(h), Pi = kappa[(b/h)^n - (b/h)^m] (eq. GeneralDisPreForm),
 *   or Pi = Pi_NLC (eqs. DisjPressNLC, mh_model) or Pi_POL (eq. DisjPressPolymer),
 * discretised by cell-centred finite volumes (Sec. Conservation Law,
 * Sec. Flux Discretization), Crank--Nicolson / theta in time (eq. TrapRule),
 * solved by the pseudo-Newton ADI iteration (eqs. JacobianSystem1-3) with the
 * adaptive time-step state machine of Fig. FlowChartTime.
 *
 * Layout: a grid of nx*ny cells, row-major, u[j*nx + i]; i (x) is contiguous.
 * Every routine is single-precision-free: all arithmetic is IEEE double,
 * compiled without FMA contraction.
 */
#ifndef TF_ORACLE_H
#define TF_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_MODEL_POWERLAW = 0, OR_MODEL_LINEAR = 1, OR_MODEL_NLC = 2, OR_MODEL_POLYMER = 3 };

typedef struct {
  int nx, ny;          /* cells in x and y                                  */
  double ds;           /* grid spacing, equal in x and y                    */
  int model;           /* OR_MODEL_POWERLAW or OR_MODEL_LINEAR              */
  double cap_C;        /* f0 = C h^3                                        */
  double b, kappa;     /* Pi = kappa[(b/h)^n - (b/h)^m]                     */
  int n, m;            /* exponents, n > m >= 1                             */
  double c0, c1;       /* linear model: f0 = c0, f1 = c1                    */
  double theta;        /* time weighting; 0.5 = Crank--Nicolson             */
  /* NLC model (eqs. DisjPressNLC, mh_model): Pi = K[(b/h)^3 - (b/h)^2]
     + (N/2)(m(h)/h)^2, m(h) = g(h) h^2/(h^2 + beta^2),
     g(h) = [1 + tanh((h - 2b)/w)]/2                                       */
  double nlc_K, nlc_N, nlc_beta, nlc_w;
  /* polymer model (eq. DisjPressPolymer): Pi = -psi'(h),
     psi = Cp/h^8 - A1/(12 pi h^2) + (A1 - A2)/(12 pi (h + d)^2),
     A1 = A_SiOx, A2 = A_Si                                                 */
  double pol_C, pol_A1, pol_A2, pol_d;
} or_model;

typedef struct {
  double tol;          /* Newton tolerance on max|v/u_k| (eq. NewtonError)  */
  int max_iter;        /* K, iterations before a step is rejected           */
  int fixed_iter;      /* >0: run exactly this many iterations, no test     */
  double dt_min, dt_max, dt_shrink, dt_grow;
  int grow_after;      /* consecutive accepted steps before dt grows        */
  double rupture_h;    /* stop when min h < rupture_h (0 = off)             */
} or_control;

typedef struct {
  int status;          /* 0 converged; 1 not converged; 2 non-positive or
                          non-finite h; 3 zero pivot                        */
  int iterations;      /* Newton iterations taken                           */
  double err;          /* max|v/u_k| of the last iteration                  */
  double gnorm;        /* max|G(u_k)| at the start of the last iteration    */
  double mass;         /* sum of u over the grid after the step             */
  double hmin;         /* min u after the step                              */
} or_step_info;

typedef struct {
  double t, dt;        /* time before the attempt, step size tried          */
  int accepted, iterations, status;
  double err, gnorm, mass, hmin;
} or_record;

/* kappa from the contact angle: kappa = (1 - cos th) / (b M),
 * M = (n - m) / ((m - 1)(n - 1)).                                          */
double or_kappa_from_contact_angle(double theta_c, double b, int n, int m);

/* Pi(h), Pi'(h) and Pi''(h) of the model (power law, NLC or polymer). */
void or_pi(const or_model* M, double h, double* pi, double* dpi, double* d2pi);

/* Pi'(h). */
double or_dpi(const or_model* M, double h);

/* Mobilities f0, f1 and their derivatives at one height.                   */
void or_mobility(const or_model* M, double h, double* f0, double* f1,
                 double* df0, double* df1);

/* Linear stability of a flat film h0: sigma(q) = q^2 (f1 - f0 q^2),
 * q_m = sqrt(f1 / (2 f0)), sigma_m = f1^2 / (4 f0).                        */
void or_lsa(const or_model* M, double h0, double* qm, double* sigma_m);

/* Five-point Laplacian with even reflection at the walls.                  */
void or_laplacian(const or_model* M, const double* u, double* lap);

/* D(u): the discrete flux divergence, u_t = -D(u) (eq. GovEqnCell2).       */
void or_operator_D(const or_model* M, const double* u, double* D);

/* b^n = u^n - (1-theta) dt D(u^n).                                         */
void or_explicit_part(const or_model* M, const double* un, double dt, double* bn);

/* G(u_k) = u_k + theta dt D(u_k) - b^n.                                    */
void or_residual(const or_model* M, const double* uk, const double* bn,
                 double dt, double* G);

/* Band of I + theta dt J_x on row j (band[5*i + c] multiplies u_{i+c-2}),
 * and of I + theta dt J_y on column i (band[5*j + c] multiplies u_{j+c-2}). */
void or_jx_row(const or_model* M, const double* uk, double dt, int j, double* band);
void or_jy_col(const or_model* M, const double* uk, double dt, int i, double* band);

/* Banded Gaussian elimination without pivoting on an n x n pentadiagonal
 * band (layout as above).  Returns 0, or 3 on a zero / non-finite pivot.   */
int or_penta_solve(int n, const double* band, const double* rhs, double* x);

/* One pseudo-Newton ADI iteration from u_k: G, x-lines, y-lines, update.
 * w (the x-solve output), v and unew may be NULL-free scratch provided by
 * the caller (each nx*ny).  Returns 0 or 3 (zero pivot).                    */
int or_newton_iteration(const or_model* M, const double* uk, const double* bn,
                        double dt, double* G, double* w, double* v,
                        double* unew, double* err, double* gnorm);

/* A whole time step from u^n with step size dt.                            */
int or_step(const or_model* M, const or_control* C, const double* un,
            double dt, double* unew, or_step_info* info);

/* Adaptive time stepping (Fig. FlowChartTime).  h is advanced in place from
 * t0 toward t_end; at most max_attempts step attempts are made.  If
 * dt_replay is not NULL, attempt a uses dt_replay[a] and, if iter_replay is
 * not NULL, exactly iter_replay[a] Newton iterations.  records (nullable)
 * receives one entry per attempt.  Returns the number of attempts made;
 * *status receives 0 (reached t_end), 1 (attempt limit), 2 (dt below
 * dt_min), 3 (rupture).                                                     */
int or_advance(const or_model* M, const or_control* C, double* h, double t0,
               double t_end, double dt0, int max_attempts,
               const double* dt_replay, const int* iter_replay,
               or_record* records, double* t_out, double* dt_out, int* status);

/* Number of OpenMP threads the oracle uses (1 if built without OpenMP).    */
int or_num_threads(void);
/* Threads of the following calls (n > 0); every line is still computed by
 * one thread with the same arithmetic, so results do not depend on n. */
void or_set_num_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
