/*
 * tf.h -- C ABI of the GB300 Newton--ADI thin-film solver (libtfadi.so).
 *
 * The library advances the two-dimensional thin-film equation
 *     h_t + div[ f0(h) grad lap h + f1(h) grad h ] = 0,
 *     f0 = C h^3,  f1 = h^3 Pi'(h),  Pi(h) = kappa[(b/h)^n - (b/h)^m]
 * (Lam, Cummings & Kondic, eq. GoverningEquation and eq. GeneralDisPreForm,
 * read with f1 = h^3 Pi' so that the printed stability values hold) on a
 * uniform cell-centred grid with no-flux walls (eq. BoundaryConditions),
 * using the conservative flux discretisation (eq. GovEqnCell2 and Sec. Flux
 * Discretization), the trapezoidal (Crank--Nicolson) rule (eq. TrapRule),
 * the pseudo-Newton ADI iteration (eqs. JacobianSystem1-3, x-lines first,
 * then y-lines) and the adaptive time-step state machine (Fig.
 * FlowChartTime, eq. NewtonError).
 *
 * Conventions
 *   Grids: nx*ny cells, IEEE double, row-major [ny][nx] (x contiguous),
 *   DEVICE memory owned by the caller, 8-byte aligned.  The library never
 *   frees caller memory.  Input and output grids of one call must not
 *   overlap unless stated.
 *   Streams: all GPU work of a context runs on the stream given to
 *   tf_init (a cudaStream_t passed as void*; NULL = legacy default stream).
 *   Calls that return scalars (tf_residual, tf_newton_adi_step,
 *   tf_advance) synchronise that stream before returning.
 *   Errors: every call returns an int.  0 = success; negative = API or CUDA
 *   error (tf_strerror gives text; the context stays usable for TF_ERR_ARG,
 *   and should be destroyed after TF_ERR_CUDA).  Positive values of
 *   tf_newton_adi_step are step outcomes (TF_STEP_*).  No call aborts, traps
 *   or throws across this interface.
 */
#ifndef TFADI_TF_H
#define TFADI_TF_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------ */
#define TF_OK 0
#define TF_ERR_ARG (-1)   /* invalid argument (sizes, NULL, parameters)    */
#define TF_ERR_CUDA (-2)  /* a CUDA runtime call failed                    */
#define TF_ERR_NOMEM (-3) /* device or host allocation failed              */

/* step outcomes (tf_step_info.status, tf_step_record.status) */
#define TF_STEP_CONVERGED 0     /* max|v/u_k| < newton_tol (eq. NewtonError) */
#define TF_STEP_NOT_CONVERGED 1 /* K iterations without convergence          */
#define TF_STEP_NONPOSITIVE 2   /* an iterate had h <= 0 or a non-finite value */
#define TF_STEP_ZERO_PIVOT 3    /* zero or non-finite pivot in a line solve   */

/* tf_advance_info.status */
#define TF_ADV_DONE 0        /* reached t_end                              */
#define TF_ADV_MAX_ATTEMPTS 1/* attempt limit reached before t_end         */
#define TF_ADV_DT_MIN 2      /* dt fell below dt_min (or a replayed step failed) */
#define TF_ADV_RUPTURE 3     /* min h fell below rupture_h                 */

/* models (Sec. Thin Film Models) */
#define TF_MODEL_POWERLAW 0 /* f0 = C h^3, f1 = h^3 Pi'(h), power-law Pi    */
#define TF_MODEL_LINEAR 1   /* f0 = c0, f1 = c1 (the linear test model)      */
#define TF_MODEL_NLC 2      /* f0 = C h^3, f1 = h^3 Pi_NLC'(h): eqs. DisjPressNLC,
                               mh_model (nematic liquid crystal film)          */
#define TF_MODEL_POLYMER 3  /* f0 = C h^3, f1 = h^3 Pi_POL'(h): eq.
                               DisjPressPolymer (polymer film on SiOx/Si)     */

/* precision modes */
#define TF_FP64 0      /* every operation in IEEE double                       */
#define TF_FP32_BULK 1 /* residual, explicit part, update and norms in
                          double-float (FP32 pairs, >= 47-bit significand) on
                          the FP32 pipes; Jacobian assembly and pentadiagonal
                          solves in FP32; state stays IEEE double           */

/* line solvers of the pentadiagonal systems (eq. LUFactorization); both
   solve every line exactly, without pivoting                              */
#define TF_SOLVER_TWISTED 0     /* two threads per line meet in the middle;
                                   LU factors kept in device scratch        */
#define TF_SOLVER_PARTITIONED 1 /* lines cut into segments of 64 (x) and 32
                                   (y) cells solved independently, with a
                                   2 x 2 block-tridiagonal reduced system on
                                   two-cell separators per line (the
                                   partition idea of Sec. Conclusions); only
                                   TF_FP32_BULK with the (3, 2) power law   */
#define TF_SOLVER_AUTO 2        /* the solver tf_tune_line_solver chose for
                                   this grid shape and arithmetic, else
                                   TF_SOLVER_TWISTED                        */

typedef struct {
  int nx, ny;            /* cells in x and y, 1..65536 each, nx*ny < 2^31       */
  double ds;             /* grid spacing (both directions), > 0               */
  int model;             /* TF_MODEL_*                                         */
  double cap_C;          /* f0 = C h^3                                         */
  double b;              /* precursor scale of Pi                              */
  int n, m;              /* exponents of Pi, n > m >= 1                        */
  double kappa;          /* strength of Pi; if <= 0 it is derived from
                            contact_angle: kappa = (1 - cos th)/(b M),
                            M = (n-m)/((m-1)(n-1))  (requires m >= 2)         */
  double contact_angle;  /* radians                                           */
  double c0, c1;         /* TF_MODEL_LINEAR coefficients                       */
  double theta;          /* time weighting, 0.5 = Crank--Nicolson, in [0,1]   */
  double newton_tol;     /* tolerance on max|v/u_k|                            */
  int newton_max_iter;   /* K: iterations before a step is rejected (>= 1)    */
  int newton_fixed_iter; /* > 0: run exactly this many iterations, no test    */
  double dt_min, dt_max; /* step-size bounds of the controller                 */
  double dt_shrink;      /* factor on rejection, in (0,1)                     */
  double dt_grow;        /* factor after grow_after accepted steps, >= 1      */
  int grow_after;        /* consecutive accepted steps before dt grows        */
  double rupture_h;      /* tf_advance stops when min h < rupture_h (0 = off) */
  int precision;         /* TF_FP64 or TF_FP32_BULK                            */
  /* TF_MODEL_NLC: Pi = K[(b/h)^3 - (b/h)^2] + (N/2)(m(h)/h)^2,
     m(h) = g(h) h^2/(h^2 + beta^2), g(h) = [1 + tanh((h - 2b)/w)]/2, with b
     above; the paper's set (eq. NLC_paras) is C = 0.0857, K = 36, N = 1.67,
     beta = 1, w = 0.05, b = 0.01.  All > 0.                               */
  double nlc_K, nlc_N, nlc_beta, nlc_w;
  /* TF_MODEL_POLYMER: Pi = -psi'(h), psi = Cp/h^8 - A_SiOx/(12 pi h^2)
     + (A_SiOx - A_Si)/(12 pi (h + d)^2); the paper's set (eq.
     Polymer_scales) is C = 0.00581, Cp = 1.181, A_SiOx = 41.25,
     A_Si = -243.75, d = 191.  Cp > 0, d >= 0.                            */
  double pol_C, pol_A_SiOx, pol_A_Si, pol_d;
  int line_solver;       /* TF_SOLVER_TWISTED (default), TF_SOLVER_PARTITIONED or
                            TF_SOLVER_AUTO; the solvers give the same
                            solutions to FP32 rounding, at speeds that
                            depend on the grid                              */
} tf_params;

typedef struct tf_ctx tf_ctx;

typedef struct {
  double gnorm; /* max |G| over the grid                                     */
  double mass;  /* sum of the grid values (of h_k): each value rounded to a
                   multiple of 2^-36 and summed exactly in 128-bit integer
                   arithmetic (heights below 2^27), so the sum does not
                   depend on the order of the additions; converted to
                   double once                                          */
  double hmin;  /* min of h_k                                                 */
} tf_norms;

typedef struct {
  int status;     /* TF_STEP_*                                               */
  int iterations; /* Newton iterations run                                   */
  double err;     /* max|v/u_k| of the last iteration                        */
  double gnorm;   /* max|G(u_k)| at the start of the last iteration          */
  double mass;    /* sum of h_new                                            */
  double hmin;    /* min of h_new                                            */
} tf_step_info;

typedef struct {
  double t, dt;   /* time before the attempt and the step size tried        */
  int accepted, iterations, status;
  double err, gnorm, mass, hmin;
} tf_step_record;

typedef struct {
  int status;            /* TF_ADV_*                                         */
  int attempts;          /* step attempts made                               */
  int accepted;          /* accepted steps                                   */
  int newton_iterations; /* Newton iterations over all attempts              */
  double t;              /* time reached                                     */
  double dt;             /* step size the controller would try next          */
} tf_advance_info;

/* Fill *p with the defaults: power-law model, C = 1, b = 0.1, n = 3, m = 2,
 * contact angle 20 degrees (kappa derived), theta = 0.5, tol 1e-10, K = 10,
 * dt_min 1e-9, dt_max 1e30, shrink 0.5, grow 1.25 after 5, no rupture stop,
 * TF_FP64, TF_SOLVER_TWISTED; the NLC and polymer parameters hold the
 * paper's sets (C and b must still be set for those models).  nx, ny, ds are set to 0 and must
 * be filled in.                                                          */
void tf_params_default(tf_params* p);

/* Create a context: validates *p, allocates the device workspace (about
 * 10 FP64 grids in TF_FP64, 6 in TF_FP32_BULK) and pinned host scalars.
 * stream: cudaStream_t (as void*) on which every kernel of this context is
 * launched.  *out receives the context or NULL on error.                 */
int tf_init(const tf_params* p, void* stream, tf_ctx** out);

/* Release everything tf_init allocated.  NULL is ignored.                */
void tf_destroy(tf_ctx* ctx);

/* Text for a return code or step outcome (static storage).              */
const char* tf_strerror(int code);

/* Kappa actually used by the context (given or derived).                */
double tf_kappa(const tf_ctx* ctx);

/* Newton residual (Sec. Newton Iterative Scheme):
 *   b^n = h_old - (1-theta) dt D(h_old),
 *   G   = h_k + theta dt D(h_k) - b^n,
 * with D the discrete flux divergence of eq. GovEqnCell2.
 * h_k, h_old: device grids (may alias).  G: device grid or NULL.
 * out: host struct or NULL (gnorm = max|G|, mass and hmin of h_k).       */
int tf_residual(tf_ctx* ctx, const double* h_k, const double* h_old, double dt,
                double* G, tf_norms* out);

/* One pseudo-Newton ADI iteration from h_k (eqs. JacobianSystem1-3):
 *   (I + theta dt J_x) w = -G(h_k)   on every row (x-line),
 *   (I + theta dt J_y) v = w         on every column (y-line),
 *   h_next = h_k + v.
 * b^n is formed from h_old inside the call.  w, v: device grids or NULL
 * (written as double).  h_next must not overlap h_k or h_old.
 * info: status (TF_STEP_CONVERGED if err < newton_tol, else
 * TF_STEP_NOT_CONVERGED, or a failure code), err, gnorm, mass, hmin.     */
int tf_newton_iteration(tf_ctx* ctx, const double* h_k, const double* h_old,
                        double dt, double* w, double* v, double* h_next,
                        tf_step_info* info);

/* One time step of size dt from h_old (device) into h_new (device, must not
 * overlap h_old): iterate from u_0 = h_old until max|v/u_k| < newton_tol,
 * up to newton_max_iter iterations (or exactly newton_fixed_iter).
 * Returns the step outcome TF_STEP_* (>= 0) or a negative error.  On a
 * failed step h_new holds the last iterate; h_old is never modified.     */
int tf_newton_adi_step(tf_ctx* ctx, const double* h_old, double* h_new, double dt,
                       tf_step_info* info);

/* Adaptive time stepping (Fig. FlowChartTime) of the device grid h in place
 * from t0 toward t_end, starting with step size dt0; at most max_attempts
 * step attempts.  Accepted: t += dt; after grow_after consecutive accepted
 * steps dt = min(dt * dt_grow, dt_max).  Rejected: dt = (tried dt) *
 * dt_shrink, failing below dt_min.  The last step is clipped to land on
 * t_end.  Replay (host arrays, nullable): attempt a uses dt_replay[a] and,
 * if iter_replay != NULL, exactly iter_replay[a] Newton iterations, with
 * no controller; a failed replayed step ends the call with TF_ADV_DT_MIN.
 * records: host array of max_attempts entries or NULL.  info: host, required.
 * streak: host int or NULL, the controller's count of consecutive accepted
 * steps since dt last changed: read at the start (NULL = 0; negative values
 * are refused) and written at the end, so a run split over several calls,
 * each given the previous call's t, dt and streak, makes the same decisions
 * and grids as one call.
 * Returns TF_OK or a negative error.                                     */
int tf_advance(tf_ctx* ctx, double* h, double t0, double t_end, double dt0,
               int max_attempts, const double* dt_replay, const int* iter_replay,
               tf_step_record* records, tf_advance_info* info, int* streak);

/* Engines of tf_ensemble_advance. */
#define TF_ENSEMBLE_AUTO 0  /* the graph engine for every film it serves, else the host engine */
#define TF_ENSEMBLE_HOST 1  /* the host engine for every film                                   */

/* Advance n independent films together.  Film i is advanced exactly as
 * tf_advance(ctx[i], h[i], t0[i], t_end[i], dt0[i], max_attempts[i], NULL,
 * NULL, NULL, &info[i]) would advance it -- the same kernels in the same
 * order, the same decisions, bit-identical grids -- with the work of all
 * films queued on their contexts' streams at once, so that the kernels of
 * small films run side by side on the GPU (the many-film statistics runs of
 * Sec. Results; no counterpart in the paper's implementation).  Two
 * engines:
 *   graph engine (TF_ENSEMBLE_AUTO, for FP32-bulk contexts of the (3, 2)
 *     power law on the twisted sweeps): each film's whole run is one launch
 *     of a CUDA graph held by its context -- conditional WHILE nodes over
 *     attempts and Newton iterations whose conditions the reduction kernels
 *     set (their thread 0 runs tf_advance's decisions on the reduced
 *     scalars), with the film's Δt and Newton state in device memory.  The host waits once per film per
 *     call.  The graph is built on the context's first such call (a few
 *     milliseconds); that first call should come before any stream capture.
 *     With timing enabled only tf_timing.launches is counted for these
 *     films.
 *   host engine (TF_ENSEMBLE_HOST, and every other context): the state
 *     machine of tf_advance on the host, its waits on the GPU resumable, four
 *     host threads polling the films' events.
 * Give each context its own stream: contexts that share a stream are
 * correct but serialised.  ctx: n distinct contexts; h: n device grids,
 * each of its context's shape (advanced in place); t0, t_end, dt0,
 * max_attempts: n host values each; info: n host records, required;
 * streak: n host values (each film's accept streak, in and out, as in
 * tf_advance) or NULL; engine: TF_ENSEMBLE_AUTO or TF_ENSEMBLE_HOST.
 * Returns TF_OK, or a negative error at the first failing call (work of
 * other films may then still be queued: synchronise or destroy the
 * contexts).                                                             */
int tf_ensemble_advance(int n, tf_ctx* const* ctx, double* const* h, const double* t0,
                        const double* t_end, const double* dt0, const int* max_attempts,
                        tf_advance_info* info, int* streak, int engine);

/* ---- line-solver tuning ---------------------------------------------------
 * The paper has no counterpart to this: it picks, per grid shape, the
 * faster of the line solvers for the many-film runs of Sec. Results, whose
 * films range from 128^2 to 1024^2.  tf_tune_line_solver runs `copies`
 * (1..256) films of p's shape at once, each in a context and on a stream of
 * its own and each iterating from the device film h (not modified) at step
 * dt: one untimed round, then `iters` (>= 1) timed rounds of one Newton
 * iteration on every film followed by a wait for all of them; this for
 * each solver that applies to *p.  The faster (in film iterations per
 * second) goes into a table of this process keyed by (nx, ny, precision,
 * model, n, m).  With copies = 1 it measures a film alone; with many it
 * measures the throughput a solver gives when films share the GPU, which
 * can rank the solvers the other way.  *best receives the chosen solver;
 * ms (host, 2 entries, or NULL) the milliseconds per film iteration of
 * TF_SOLVER_TWISTED and TF_SOLVER_PARTITIONED (-1 where a solver does not
 * apply).  A later call for the same key replaces the entry.  Contexts
 * created with line_solver = TF_SOLVER_AUTO read the table once, in
 * tf_init, so a context never changes solver.  Allocates `copies`
 * temporary contexts and streams per solver; synchronises the device.
 * Returns TF_OK, TF_ERR_ARG or a context's error.                        */
int tf_tune_line_solver(const tf_params* p, void* stream, const double* h, double dt, int iters,
                        int copies, int* best, double* ms);
/* The table's entry for *p's key (TF_SOLVER_*), or -1 if there is none.   */
int tf_tuned_line_solver(const tf_params* p);
/* The solver a context uses (TF_SOLVER_TWISTED or TF_SOLVER_PARTITIONED),
 * or -1 for NULL.                                                         */
int tf_line_solver(const tf_ctx* ctx);

/* FMA throughput of the current GPU, for the roofline of arithmetic-bound
 * kernels (the paper has no counterpart): precision TF_FP64 times FP64
 * fused multiply-adds, TF_FP32_BULK FP32 ones; 8 independent chains per
 * thread, 8 blocks of 256 threads per SM, on the given stream.  *tflops
 * receives 2 x FMAs / s / 1e12.  Allocates a small output buffer;
 * synchronises the stream.  Returns TF_OK, TF_ERR_ARG, TF_ERR_NOMEM or
 * TF_ERR_CUDA.                                                            */
int tf_probe_fma(int precision, void* stream, double* tflops);

/* Kernel timing of a context, for measurement.  While enabled, the library
 * records CUDA events on its stream around every kernel it launches and
 * accumulates their durations per kernel kind; the sums are taken at the
 * synchronisation point that ends each Newton iteration.  Counters reset
 * when timing is enabled. */
typedef struct {
  int enabled;
  int launches;          /* kernels launched while enabled (all kinds)       */
  int explicit_launches; /* b^n launches (in tf_newton_adi_step, tf_advance and
                            ensembles they also form the right side of the
                            step's first iteration, which then has no
                            residual launch of its own)                    */
  int rhs_launches;      /* residual (right side of the x solve) launches    */
  int x_launches;        /* x-line sweep launches                            */
  int y_launches;        /* y-line sweep launches                            */
  double explicit_ms, rhs_ms, x_ms, y_ms; /* summed event durations, ms      */
} tf_timing;

int tf_timing_enable(tf_ctx* ctx, int on);
int tf_timing_get(const tf_ctx* ctx, tf_timing* out);

/* ---- residual without allocation ----------------------------------------
 * The paper has no counterpart to this entry point: it is a service to
 * callers that may not allocate device memory (a host framework that owns
 * every allocation, a latency-bounded loop, a plugin handed buffers but no
 * right to create a context).  It computes what tf_residual computes,
 *   G = h_k + theta dt D(h_k) - [h_old - (1-theta) dt D(h_old)],
 * for the parameters *p on the given stream (cudaStream_t as void*, NULL = legacy default stream).
 * h_k, h_old: device grids [ny][nx]; G: device output grid (required);
 * out: host struct or NULL (gnorm = max|G|, mass and hmin of h_k; when
 * given, the call synchronises the stream).
 * Models: TF_MODEL_POWERLAW and TF_MODEL_LINEAR only (TF_MODEL_NLC and
 * TF_MODEL_POLYMER return TF_ERR_ARG); the other fields of *p are checked
 * as tf_init checks them.
 * Scratch: one fixed device array of this library (TF_NOALLOC_MAX_CELLS
 * cells plus partial results, about 16.3 MiB), present on every GPU that
 * loads the library until the process exits; grids larger than
 * TF_NOALLOC_MAX_CELLS cells return TF_ERR_ARG.  The call makes no
 * cudaMalloc, cudaFree or other allocating call.  The first call on each
 * device looks up the array's device address (with that device current);
 * make that first call before any stream capture.  Calls share the array,
 * which keeps the last call's contents (each call writes every element it
 * reads before reading it), so calls that overlap on the GPU race: the
 * caller must serialise them.  Returns TF_OK, TF_ERR_ARG or TF_ERR_CUDA. */
#define TF_NOALLOC_MAX_CELLS (1 << 21)
int tf_residual_noalloc(const tf_params* p, void* stream, const double* h_k,
                        const double* h_old, double dt, double* G, tf_norms* out);

/* ---- discrete adjoint of the fixed-iteration time step -------------------
 * The time step with exactly K Newton iterations at step size dt (Sec.
 * Numerical Method, no convergence test) is a smooth map
 *   u^n -> u^K:  b = u^n - (1-theta) dt D(u^n),  u_0 = u^n,
 *   (I + theta dt J_x(u_k)) w_k = -G(u_k),  (I + theta dt J_y(u_k)) v_k = w_k,
 *   u_{k+1} = u_k + v_k.
 * tf_adjoint_step runs it forward (the FP64 path, keeping every u_k, w_k,
 * v_k) and then its reverse: given the cotangent g of u^K it returns
 * g_h = (du^K/du^n)^T g and g_kappa = (du^K/dkappa)^T g, through transposed
 * line solves (y lines, then x lines, each iteration in reverse order) and
 * the transposed derivatives of D and of the line operators' dependence on
 * u (face-by-face partial derivatives, gathered per cell, no atomics).
 * The context must be TF_FP64 with the power-law or linear model.
 * h_old, g: device grids; h_new: device grid or NULL (receives u^K);
 * g_h: device output grid (not aliasing h_old, g or h_new); g_kappa,
 * g_theta: host outputs or NULL (g_theta = g_kappa dkappa/dtheta_c when
 * kappa was derived from the contact angle, else 0).  K: 1..64.
 * Workspace (3K + 19 grids) is allocated on first use and kept by the
 * context.  Synchronises the context's stream.  Returns TF_OK, TF_ERR_ARG,
 * TF_ERR_NOMEM or TF_ERR_CUDA (or a forward iteration's error).         */
int tf_adjoint_step(tf_ctx* ctx, const double* h_old, double dt, int K, const double* g,
                    double* h_new, double* g_h, double* g_kappa, double* g_theta);

/* Kernel time (ms, CUDA events) of the last tf_adjoint_step in this
 * process, by group: forward iterations, per-iterate tables and band
 * assembly, transposed line solves, x-line coefficient derivatives, y-line
 * coefficient derivatives, D derivatives, the copy of the kappa partial
 * sums.  n: entries wanted (up to 7).                                     */
int tf_adjoint_timing(double* ms, int n);

/* ---- adjoint of a trajectory of fixed steps, with checkpoints ----------
 * The map u^0 -> u^N of N time steps, each the fixed-iteration step above
 * (K Newton iterations at step size dt), and its reverse for a cotangent g
 * of u^N: g_h0 = (du^N/du^0)^T g and g_kappa = (du^N/dkappa)^T g, the
 * chain rule over the steps (Sec. Numerical Method; the adjoint of each step
 * is tf_adjoint_step's).  Uniform checkpoints: the forward keeps u^n at
 * n = 0, e, 2e, ... (ceil(N/e) grids); the reverse runs one segment of e
 * steps again from its checkpoint, keeping each step's iterates (u_k, w_k,
 * v_k: 3K grids), and reverses them, so memory is ceil(N/e) + 6Ke + 2 grids
 * (O(sqrt N) at e = ceil(sqrt(N))) for two forward passes and one reverse.
 * A segment is run again (on the context's stream, from a host worker
 * thread) while the next one is reversed (on the tape's own stream): two
 * banks of iterates.
 * Every segment recomputes exactly the forward's bits (the same kernels and
 * order), so the result does not depend on e.  The context must satisfy
 * tf_adjoint_step's conditions.                                          */
typedef struct tf_tape tf_tape;

/* A tape for nsteps >= 1 steps of K (1..64) iterations at dt > 0 on the
 * context's grid, checkpoint interval every (0: ceil(sqrt(nsteps)); else
 * 1..nsteps).  Allocates ceil(nsteps/every) + 6 K every + 2 device grids
 * (the reverse also uses the context's adjoint workspace).  The
 * context must outlive the tape.  Returns TF_OK, TF_ERR_ARG or
 * TF_ERR_NOMEM.                                                           */
int tf_tape_create(tf_ctx* ctx, int nsteps, int K, double dt, int every, tf_tape** out);
void tf_tape_destroy(tf_tape* tape);

/* every: the interval in use; checkpoints: ceil(nsteps/every); bytes: the
 * tape's device memory; forward_done: 1 once tf_tape_forward succeeded.    */
int tf_tape_info(const tf_tape* tape, int* every, int* checkpoints, size_t* bytes, int* forward_done);

/* Runs the N steps from h0 (device grid), keeping the checkpoints, and
 * writes u^N to hT (device grid, may equal h0; not inside the tape).
 * Returns TF_OK, a step failure TF_STEP_NONPOSITIVE / TF_STEP_ZERO_PIVOT of
 * the first step that had one (the trajectory left the model's domain; the
 * tape is then unusable), or a negative error.  Synchronises the stream.   */
int tf_tape_forward(tf_tape* tape, const double* h0, double* hT);

/* The reverse of the last forward: g (device grid, the cotangent of u^N),
 * g_h0 (device output grid, may equal g), g_kappa, g_theta (host outputs or
 * NULL; g_theta as in tf_adjoint_step).  Sums over the steps are taken in a
 * fixed order, so repeated calls give the same bits.  Waits for the
 * context's stream first; synchronises both streams before it returns.
 * Returns TF_OK, TF_ERR_ARG (no forward yet) or a negative error.          */
int tf_tape_backward(tf_tape* tape, const double* g, double* g_h0, double* g_kappa, double* g_theta);

/* Kernel time (ms, CUDA events) of the tape's last forward and backward:
 * [0] forward steps, [1] the segments' steps run again with their
 * iterates, then the seven tf_adjoint_timing groups summed over the reverse
 * steps (the "forward" group stays 0: the iterates come from [1]).  n: up
 * to 9.                                                                  */
int tf_tape_timing(const tf_tape* tape, double* ms, int n);

/* ---- radial Fourier analysis of a film (App. Radial Fourier Transform) ---
 * The dominant wavenumber of a film pattern, all steps on the GPU, in the
 * appendix's order:
 *  1. zeta = h - H0; A[q][p] = |C[q][p]| / (nx ny), where C is the 2-D
 *     DCT-II sum  sum_j sum_i zeta[j][i] cos(pi p (2i+1)/2nx)
 *     cos(pi q (2j+1)/2ny): the FFT magnitude of the film reflected evenly
 *     about its no-flux walls, normalised by the reflected film's size, at
 *     wave vector (pi p / Lx, pi q / Ly), L = n ds.  (A cosine mode
 *     eps cos(pi p x/Lx) cos(pi q y/Ly), p, q > 0, gives eps/4.)  FP32
 *     transform; every later step in FP64.
 *  2. Gaussian smoothing of A over (p, q): weights exp(-d^2 / 2 sigma^2),
 *     |d| <= ceil(3 sigma), normalised; outside 0..n-1 the reflected film's
 *     spectrum continues with period 2n (index -k is k, n is 0, n+k is n-k).
 *  3-4. One radial point per distinct |q| <= q_cut (eq.
 *     FFT_radial_averaging): the mean of the smoothed values with that |q|.
 *     Equality is exact on the integer key (p ny/g)^2 + (q nx/g)^2,
 *     g = gcd(nx, ny); the cut is key <= floor((q_cut/scale)^2) with
 *     scale = pi g / (ds nx ny), |q| = scale sqrt(key).
 *  5. Continuous piecewise-linear least squares (eq. PiecewiseFunction):
 *     nodes t_0 = 0, t_j = |q| of radial point j*ppi (j = 1..K-1),
 *     t_K = q_cut, K = max(1, ceil((M-1)/ppi)) for M radial points (every
 *     interval but the last holds ppi points, the last 2..ppi+1); node
 *     values a_0 = 0 and a_1..a_K fitted.
 *  6. The fit at n_eval equispaced points of [0, q_cut], smoothed by moving
 *     averages of half-widths 3, 2, 1 (windows cut at the ends).
 *  7. Local maxima: derivative by second-order differences (one-sided at
 *     the ends); a root in [q_e, q_e+1) where it is zero at q_e or changes
 *     sign, placed by linear interpolation; a maximum where the second
 *     derivative (the same differences of the derivative), interpolated to
 *     the root, is negative.  Listed highest value first.
 * Plans: nx, ny powers of two in 1..16384; ds > 0.  A plan allocates its
 * device workspace and builds the radial grouping (geometry only) once;
 * runs allocate nothing.  Every run synchronises the plan's stream.      */
typedef struct {
  double H0;               /* thickness subtracted before the transform         */
  double q_cut;            /* wavenumbers analysed, |q| <= q_cut (the paper:
                              5 q_m); > 0, at most 2^27 distinct keys below it */
  double sigma;            /* Gaussian std. deviation in wave-index steps, 0..16
                              (0 = no smoothing)                                */
  int points_per_interval; /* radial points per fit interval (the paper: 10), >= 1 */
  int n_eval;              /* samples of the fitted curve (the paper: 400), 3..4096 */
} tf_spectrum_params;

/* H0 = 1, q_cut = 0 (must be set), sigma = 1, points_per_interval = 10,
 * n_eval = 400.                                                          */
void tf_spectrum_params_default(tf_spectrum_params* sp);

typedef struct tf_spectrum_plan tf_spectrum_plan;

typedef struct {
  int n_p, n_q;          /* wave-index block of the radial points: p < n_p, q < n_q */
  int n_radii;           /* M: distinct |q| <= q_cut                          */
  int n_intervals;       /* K                                                 */
  int n_eval;            /* samples of the curve                              */
  int n_peaks;           /* local maxima found (0 before a run)               */
  double q_dominant;     /* wavenumber of the highest maximum (0 if none)     */
  double value_dominant; /* its value                                         */
} tf_spectrum_info;

/* Outputs of a run: HOST buffers, each NULL (not copied) or holding the
 * count stated (sizes from tf_spectrum_plan_info).                       */
typedef struct {
  double* amplitude;    /* [n_q][n_p]: step 1 (unsmoothed)                   */
  double* smoothed;     /* [n_q][n_p]: step 2                                */
  double* radial_q;     /* [n_radii], ascending                              */
  double* radial_value; /* [n_radii]                                          */
  double* node_q;       /* [n_intervals + 1]                                 */
  double* node_value;   /* [n_intervals + 1], node_value[0] = 0              */
  double* curve_q;      /* [n_eval]                                          */
  double* curve_value;  /* [n_eval], after the moving averages               */
  double* peak_q;       /* [peak_cap]: maxima, highest value first           */
  double* peak_value;   /* [peak_cap]                                         */
  int peak_cap;
} tf_spectrum_out;

/* stream: cudaStream_t (as void*) for every kernel of the plan.  Returns
 * TF_OK, TF_ERR_ARG (sizes, parameters, or fewer than two radial points),
 * TF_ERR_NOMEM or TF_ERR_CUDA; *out is NULL on error.                    */
int tf_spectrum_plan_create(int nx, int ny, double ds, const tf_spectrum_params* sp, void* stream,
                            tf_spectrum_plan** out);
void tf_spectrum_plan_destroy(tf_spectrum_plan* plan);
int tf_spectrum_plan_info(const tf_spectrum_plan* plan, tf_spectrum_info* info);

/* Analyse the device grid h [ny][nx] (FP64).  out: NULL or host buffers.
 * info: required.  Returns TF_OK, TF_ERR_ARG or TF_ERR_CUDA.             */
int tf_spectrum_run(tf_spectrum_plan* plan, const double* h, tf_spectrum_out* out,
                    tf_spectrum_info* info);

/* Durations (ms, CUDA events) of the last run's kernels, in order: row
 * DCTs, column DCTs, smoothing along p, smoothing along q, radial means,
 * and the fit with sampling and maxima (five kernels).  n: entries wanted
 * (up to 6).                                                             */
int tf_spectrum_timing(const tf_spectrum_plan* plan, double* ms, int n);

#ifdef __cplusplus
}
#endif
#endif
