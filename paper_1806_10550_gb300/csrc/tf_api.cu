// tf_api.cu -- C ABI of the Newton--ADI thin-film solver (see include/tf.h).
//
// Host side of the method: workspace management, the Newton iteration loop
// of one time step (Sec. Newton Iterative Scheme, eq. NewtonError) and the
// adaptive time-step state machine (Fig. FlowChartTime).  All grid work is
// done by the kernels of tf_kernels.cuh; the host reads back one small
// struct of reduced scalars per Newton iteration.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <thread>
#include <utility>
#include <vector>

#include "tf_internal.h"
#include "tf_ensemble_dev.cuh"

using tf::Scalars;

namespace {

int cuda_fail(cudaError_t e) { return e == cudaErrorMemoryAllocation ? TF_ERR_NOMEM : TF_ERR_CUDA; }

#define TF_CK(call)                     \
  do {                                  \
    cudaError_t e_ = (call);            \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)


// Reduce the partials of the last passes into the pinned c.hsc: the launch
// and the copy are queued on the context's stream; finalize() also waits.
int finalize_async(tf_ctx& c, int n_px, int n_py) {
  tf::k_finalize<<<1, 256, 0, c.stream>>>(c.px, n_px, c.py, n_py, c.dsc);
  TF_CK(cudaGetLastError());
  TF_CK(cudaMemcpyAsync(c.hsc, c.dsc, sizeof(Scalars), cudaMemcpyDeviceToHost, c.stream));
  return TF_OK;
}
// The same after an iteration of the partitioned path: the residual's
// partials and the accumulators of the partitioned kernels.
int finalize_part_async(tf_ctx& c) {
  TF_CK(tf::part::finalize(c));
  TF_CK(cudaGetLastError());
  TF_CK(cudaMemcpyAsync(c.hsc, c.dsc, sizeof(Scalars), cudaMemcpyDeviceToHost, c.stream));
  return TF_OK;
}
int finalize(tf_ctx& c, int n_px, int n_py) {
  int r = finalize_async(c, n_px, n_py);
  if (r) return r;
  TF_CK(cudaStreamSynchronize(c.stream));
  return TF_OK;
}

float elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.0f;
  return cudaEventElapsedTime(&ms, a, b) == cudaSuccess ? ms : 0.0f;
}

// One pseudo-Newton ADI iteration from u_k (b^n already formed):
// residual -> x sweep -> y sweep -> reductions, queued on the context's
// stream; iterate_collect() reads the result once the stream has reached it.
// rhs_ready: the residual of this iteration was formed with b^n (the first
// iteration of a step, explicit_launch with rhs0).
int iterate_launch(tf_ctx& c, const double* u_k, double dt, double* u_next, double* w_out,
                   double* v_out, bool rhs_ready = false) {
  const bool tm = c.timing.enabled;
  c.rhs_fused = rhs_ready;
  if (tm) TF_CK(cudaEventRecord(c.ev[0], c.stream));
  if (!rhs_ready) TF_CK(c.ops->rhs(c, u_k, dt));
  if (tm) TF_CK(cudaEventRecord(c.ev[1], c.stream));
  TF_CK(c.ops->xsweep(c, dt, u_k));
  if (tm) TF_CK(cudaEventRecord(c.ev[2], c.stream));
  if (w_out) TF_CK(c.ops->w_to_f64(c, w_out));
  if (tm) TF_CK(cudaEventRecord(c.ev[3], c.stream));
  TF_CK(c.ops->ysweep(c, u_k, dt, u_next, v_out));
  if (tm) TF_CK(cudaEventRecord(c.ev[4], c.stream));
  return c.part ? finalize_part_async(c) : finalize_async(c, c.n_rhs_parts + c.grid_x, c.grid_y);
}
void iterate_collect(tf_ctx& c, bool w_out, Scalars* s) {
  if (c.timing.enabled) {
    if (!c.rhs_fused) {
      c.timing.rhs_ms += elapsed(c.ev[0], c.ev[1]);
      c.timing.rhs_launches++;
    }
    c.timing.x_ms += elapsed(c.ev[1], c.ev[2]);
    c.timing.y_ms += elapsed(c.ev[3], c.ev[4]);
    c.timing.x_launches++;
    c.timing.y_launches++;
    const int sweeps = c.part ? tf::part::launches(c) : 2;
    c.timing.launches += (c.rhs_fused ? 2 : 3) + sweeps + (w_out && c.ops->lp_bytes != sizeof(double) ? 1 : 0);
  }
  *s = *c.hsc;
}
int iterate(tf_ctx& c, const double* u_k, double dt, double* u_next, double* w_out, double* v_out,
            Scalars* s, bool rhs_ready = false) {
  int r = iterate_launch(c, u_k, dt, u_next, w_out, v_out, rhs_ready);
  if (r) return r;
  TF_CK(cudaStreamSynchronize(c.stream));
  iterate_collect(c, w_out != nullptr, s);
  return TF_OK;
}

// The explicit part of a step -- with rhs0, also the right side of the
// step's first iteration from u_0 = h_old (one kernel in FP32-bulk, where
// D(h_old) serves both); with timing on, its events (5, 6) are read by
// explicit_collect() once the stream has passed them.
int explicit_launch(tf_ctx& c, const double* h_old, double dt, bool rhs0 = false) {
  const bool tm = c.timing.enabled;
  if (tm) TF_CK(cudaEventRecord(c.ev[5], c.stream));
  TF_CK(rhs0 ? c.ops->explicit_rhs0(c, h_old, dt) : c.ops->explicit_part(c, h_old, dt));
  if (tm) TF_CK(cudaEventRecord(c.ev[6], c.stream));
  return TF_OK;
}
void explicit_collect(tf_ctx& c) {
  if (!c.timing.enabled) return;
  c.timing.explicit_ms += elapsed(c.ev[5], c.ev[6]);
  c.timing.explicit_launches++;
  c.timing.launches += c.expl_kernels;
}

// Mass and min h of a film (once per step), into s->mass and s->hmin:
// stats_launch queues the reduction, stats_collect reads it.
int stats_launch(tf_ctx& c, const double* h) {
  tf::k_grid_stats<<<c.grid_stats, 256, 0, c.stream>>>(h, c.N, c.py);
  TF_CK(cudaGetLastError());
  if (c.timing.enabled) c.timing.launches += 2;
  return finalize_async(c, 0, c.grid_stats);
}
void stats_collect(tf_ctx& c, Scalars* s) {
  s->mass = c.hsc->mass;
  s->hmin = c.hsc->hmin;
}
int film_stats(tf_ctx& c, const double* h, Scalars* s) {
  int r = stats_launch(c, h);
  if (r) return r;
  TF_CK(cudaStreamSynchronize(c.stream));
  stats_collect(c, s);
  return TF_OK;
}

// Outcome of an iteration, in the oracle's order: pivot, positivity, test.
int classify(const tf_ctx& c, const Scalars& s, int it, int fixed_iter) {
  if (s.pivot) return TF_STEP_ZERO_PIVOT;
  if (s.nonfinite) return TF_STEP_NONPOSITIVE;
  if (fixed_iter > 0) return it >= fixed_iter ? TF_STEP_CONVERGED : TF_STEP_NOT_CONVERGED;
  if (s.err < c.p.newton_tol) return TF_STEP_CONVERGED;
  return TF_STEP_NOT_CONVERGED;
}

void fill_info(tf_step_info* info, int status, int it, const Scalars& s) {
  if (!info) return;
  info->status = status;
  info->iterations = it;
  info->err = s.err;
  info->gnorm = s.gnorm;
  info->mass = tf::mass_value(s.mass);
  info->hmin = s.hmin;
}

// A time step with an explicit fixed-iteration override (0 = none).
// The iterate ping-pongs between h_new and c.ubuf; the result is in h_new.
int step(tf_ctx& c, const double* h_old, double* h_new, double dt, int fixed_iter, tf_step_info* info) {
  int re = explicit_launch(c, h_old, dt, true);
  if (re) return re;
  const int kmax = fixed_iter > 0 ? fixed_iter : c.p.newton_max_iter;
  const double* uk = h_old;
  double* bufs[2] = {h_new, c.ubuf};
  Scalars s;
  memset(&s, 0, sizeof(s));
  int status = TF_STEP_NOT_CONVERGED, it = 0;
  for (int k = 0; k < kmax; ++k) {
    double* un = bufs[k & 1];
    int r = iterate(c, uk, dt, un, nullptr, nullptr, &s, k == 0);
    if (r) return r;
    if (k == 0) explicit_collect(c);
    it = k + 1;
    uk = un;
    status = classify(c, s, it, fixed_iter);
    if (status != TF_STEP_NOT_CONVERGED) break;
  }
  if (uk != h_new)
    TF_CK(cudaMemcpyAsync(h_new, uk, c.N * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
  int rs = film_stats(c, h_new, &s);
  if (rs) return rs;
  fill_info(info, status, it, s);
  return status;
}

// ---------------------------------------------------------------------------
// Ensembles of independent films (the many-film statistics runs of Sec.
// Results).  Each film runs the state machine of tf_advance -- the same
// kernels, in the same order, with the same decisions and results -- but
// every wait on the GPU becomes a resumable state, so one host thread keeps
// the work of many films queued on their own streams at once: small films
// leave most SMs idle, and their kernels then run side by side.

struct FilmRun {
  tf_ctx* c;
  double* h;
  double t, t_end, dt;
  int max_att;
  tf_advance_info* info;
  int* streak_io;  // the caller's accept streak (in and out), or NULL
  double *cur, *nxt;
  int streak, a, status;
  bool done;
  // the attempt in flight
  double step_dt;
  int last, fixed, kmax, k, it, sstatus, phase;  // phase 1: iterating, 2: film statistics
  const double* uk;
  double* bufs[2];
  Scalars s;
};

int film_finish(FilmRun& F) {
  if (F.status == TF_ADV_MAX_ATTEMPTS && F.t >= F.t_end) F.status = TF_ADV_DONE;
  if (F.cur != F.h)
    TF_CK(cudaMemcpyAsync(F.h, F.cur, F.c->N * sizeof(double), cudaMemcpyDeviceToDevice, F.c->stream));
  if (F.streak_io) *F.streak_io = F.streak;
  F.info->status = F.status;
  F.info->attempts = F.a;
  F.info->t = F.t;
  F.info->dt = F.dt;
  F.done = true;
  return TF_OK;
}

// Queue the explicit part and the first iteration of the next attempt (or
// finish the film).
int film_start_attempt(FilmRun& F) {
  tf_ctx& c = *F.c;
  if (F.a >= F.max_att) return film_finish(F);
  if (F.t >= F.t_end) {
    F.status = TF_ADV_DONE;
    return film_finish(F);
  }
  F.fixed = c.p.newton_fixed_iter;
  F.last = 0;
  if (F.t_end - F.t <= F.dt) {
    F.step_dt = F.t_end - F.t;
    F.last = 1;
  } else {
    F.step_dt = F.dt;
  }
  int r = explicit_launch(c, F.cur, F.step_dt, true);
  if (r) return r;
  F.kmax = F.fixed > 0 ? F.fixed : c.p.newton_max_iter;
  F.k = 0;
  F.uk = F.cur;
  F.bufs[0] = F.nxt;
  F.bufs[1] = c.ubuf;
  memset(&F.s, 0, sizeof(F.s));
  F.sstatus = TF_STEP_NOT_CONVERGED;
  F.it = 0;
  r = iterate_launch(c, F.uk, F.step_dt, F.bufs[0], nullptr, nullptr, true);
  if (r) return r;
  TF_CK(cudaEventRecord(c.ev[7], c.stream));
  F.phase = 1;
  return TF_OK;
}

// An iteration has landed: classify it as step() does, then queue the next
// iteration or the film statistics of the step's result.
int film_on_iteration(FilmRun& F) {
  tf_ctx& c = *F.c;
  iterate_collect(c, false, &F.s);
  if (F.k == 0) explicit_collect(c);
  F.it = F.k + 1;
  F.uk = F.bufs[F.k & 1];
  F.sstatus = classify(c, F.s, F.it, F.fixed);
  ++F.k;
  if (F.sstatus == TF_STEP_NOT_CONVERGED && F.k < F.kmax) {
    int r = iterate_launch(c, F.uk, F.step_dt, F.bufs[F.k & 1], nullptr, nullptr);
    if (r) return r;
  } else {
    if (F.uk != F.nxt)
      TF_CK(cudaMemcpyAsync(F.nxt, F.uk, c.N * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    int r = stats_launch(c, F.nxt);
    if (r) return r;
    F.phase = 2;
  }
  TF_CK(cudaEventRecord(c.ev[7], c.stream));
  return TF_OK;
}

// The step's film statistics have landed: the controller of tf_advance.
int film_on_stats(FilmRun& F) {
  tf_ctx& c = *F.c;
  const tf_params& P = c.p;
  stats_collect(c, &F.s);
  const int s = F.sstatus;
  ++F.a;
  F.info->newton_iterations += F.it;
  if (s == TF_STEP_CONVERGED) {
    double* tmp = F.cur;
    F.cur = F.nxt;
    F.nxt = tmp;
    F.t = F.last ? F.t_end : F.t + F.step_dt;
    F.info->accepted++;
    if (++F.streak >= P.grow_after) {
      F.dt = fmin(F.dt * P.dt_grow, P.dt_max);
      F.streak = 0;
    }
    if (P.rupture_h > 0.0 && F.s.hmin < P.rupture_h) {
      F.status = TF_ADV_RUPTURE;
      return film_finish(F);
    }
  } else {
    F.streak = 0;
    F.dt = F.step_dt * P.dt_shrink;
    if (F.dt < P.dt_min) {
      F.status = TF_ADV_DT_MIN;
      return film_finish(F);
    }
  }
  return film_start_attempt(F);
}

// ---------------------------------------------------------------------------
// Line-solver tuning table of the process: (nx, ny, precision, model, n, m)
// -> solver.

struct TuneKey {
  int nx, ny, precision, model, n, m;
  bool operator==(const TuneKey& o) const {
    return nx == o.nx && ny == o.ny && precision == o.precision && model == o.model && n == o.n && m == o.m;
  }
};
std::mutex g_tune_mutex;
std::vector<std::pair<TuneKey, int>> g_tune;
TuneKey tune_key(const tf_params& p) { return TuneKey{p.nx, p.ny, p.precision, p.model, p.n, p.m}; }

template <class T> int dalloc(T** p, size_t bytes) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
  if (e != cudaSuccess) return cuda_fail(e);
  *p = (T*)q;
  return TF_OK;
}

}  // namespace

namespace tf {
int fixed_iterates(tf_ctx& c, double dt, int K, double* const* U, double* const* W, double* const* V) {
  const int re = explicit_launch(c, U[0], dt, true);
  if (re) return re;
  for (int k = 0; k < K; ++k) {
    const int r = iterate_launch(c, U[k], dt, U[k + 1], W ? W[k] : nullptr, V ? V[k] : nullptr, k == 0);
    if (r) return r;
    if (c.timing.enabled) {  // the events are reused by the next iteration
      TF_CK(cudaStreamSynchronize(c.stream));
      if (k == 0) explicit_collect(c);
      Scalars s;
      iterate_collect(c, W != nullptr, &s);
    }
  }
  return TF_OK;
}

int fixed_step(tf_ctx& c, const double* h_old, double* h_new, double dt, int K) {
  tf_step_info info;
  const int s = step(c, h_old, h_new, dt, K, &info);
  if (s < 0) return s;
  return s == TF_STEP_CONVERGED ? TF_OK : s;
}
}  // namespace tf

extern "C" {

void tf_params_default(tf_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->model = TF_MODEL_POWERLAW;
  p->cap_C = 1.0;
  p->b = 0.1;
  p->n = 3;
  p->m = 2;
  p->kappa = 0.0;
  p->contact_angle = 20.0 * M_PI / 180.0;
  p->c0 = 1.0;
  p->c1 = 1.0;
  p->theta = 0.5;
  p->newton_tol = 1e-10;
  p->newton_max_iter = 10;
  p->newton_fixed_iter = 0;
  p->dt_min = 1e-9;
  p->dt_max = 1e30;
  p->dt_shrink = 0.5;
  p->dt_grow = 1.25;
  p->grow_after = 5;
  p->rupture_h = 0.0;
  p->precision = TF_FP64;
  p->nlc_K = 36.0;
  p->nlc_N = 1.67;
  p->nlc_beta = 1.0;
  p->nlc_w = 0.05;
  p->pol_C = 1.181;
  p->pol_A_SiOx = 41.25;
  p->pol_A_Si = -243.75;
  p->pol_d = 191.0;
  p->line_solver = TF_SOLVER_TWISTED;
}

const char* tf_strerror(int code) {
  switch (code) {
    case TF_OK: return "ok (step converged)";
    case TF_ERR_ARG: return "invalid argument";
    case TF_ERR_CUDA: return "CUDA runtime error";
    case TF_ERR_NOMEM: return "out of memory";
    case TF_STEP_NOT_CONVERGED: return "Newton iteration did not converge";
    case TF_STEP_NONPOSITIVE: return "non-positive or non-finite film height";
    case TF_STEP_ZERO_PIVOT: return "zero or non-finite pivot in a line solve";
    default: return "unknown code";
  }
}

void tf_destroy(tf_ctx* c) {
  if (!c) return;
  if (c->adj_ws) cudaFree(c->adj_ws);
  cudaFree(c->bn);
  cudaFree(c->w);
  cudaFree(c->ulp);
  cudaFree(c->fac_x);
  cudaFree(c->fac_y);
  cudaFree(c->recx);
  cudaFree(c->recy);
  cudaFree(c->xsx);
  cudaFree(c->xsy);
  cudaFree(c->acc);
  cudaFree(c->ubuf);
  cudaFree(c->ubuf2);
  cudaFree(c->px);
  cudaFree(c->py);
  cudaFree(c->dsc);
  if (c->hsc) cudaFreeHost(c->hsc);
  if (c->ens_exec) cudaGraphExecDestroy(c->ens_exec);
  cudaFree(c->ens_dev);
  if (c->ens_host) cudaFreeHost(c->ens_host);
  for (int k = 0; k < 8; ++k)
    if (c->ev[k]) cudaEventDestroy(c->ev[k]);
  free(c);
}

double tf_kappa(const tf_ctx* c) { return c ? c->kappa : 0.0; }

int tf_init(const tf_params* p, void* stream, tf_ctx** out) {
  if (!out) return TF_ERR_ARG;
  *out = nullptr;
  if (!p) return TF_ERR_ARG;
  if (p->nx < 1 || p->ny < 1 || !(p->ds > 0.0) || !isfinite(p->ds)) return TF_ERR_ARG;
  if ((double)p->nx * (double)p->ny >= 2147483647.0) return TF_ERR_ARG;
  if (p->nx > 65536 || p->ny > 65536) return TF_ERR_ARG;
  if (p->model < TF_MODEL_POWERLAW || p->model > TF_MODEL_POLYMER) return TF_ERR_ARG;
  if (p->model == TF_MODEL_NLC &&
      !(p->cap_C > 0.0 && p->b > 0.0 && p->nlc_K > 0.0 && p->nlc_N > 0.0 && p->nlc_beta > 0.0 && p->nlc_w > 0.0))
    return TF_ERR_ARG;
  if (p->model == TF_MODEL_POLYMER && !(p->cap_C > 0.0 && p->pol_C > 0.0 && p->pol_d >= 0.0 &&
                                        isfinite(p->pol_A_SiOx) && isfinite(p->pol_A_Si)))
    return TF_ERR_ARG;
  if (!(p->theta >= 0.0 && p->theta <= 1.0)) return TF_ERR_ARG;
  if (p->newton_max_iter < 1 || p->newton_fixed_iter < 0) return TF_ERR_ARG;
  if (!(p->dt_shrink > 0.0 && p->dt_shrink < 1.0) || !(p->dt_grow >= 1.0) || p->grow_after < 1)
    return TF_ERR_ARG;
  if (p->precision != TF_FP64 && p->precision != TF_FP32_BULK) return TF_ERR_ARG;
  if (p->line_solver < TF_SOLVER_TWISTED || p->line_solver > TF_SOLVER_AUTO) return TF_ERR_ARG;
  if (p->line_solver == TF_SOLVER_PARTITIONED &&
      !(p->precision == TF_FP32_BULK && p->model == TF_MODEL_POWERLAW && p->n == 3 && p->m == 2))
    return TF_ERR_ARG;
  double kappa = p->kappa;
  if (p->model == TF_MODEL_POWERLAW) {
    if (!(p->b > 0.0) || p->m < 1 || p->n <= p->m || p->n > 12 || !(p->cap_C > 0.0)) return TF_ERR_ARG;
    if (!(kappa > 0.0)) {
      if (p->m < 2) return TF_ERR_ARG;
      double Mf = (double)(p->n - p->m) / ((double)(p->m - 1) * (double)(p->n - 1));
      kappa = (1.0 - cos(p->contact_angle)) / (p->b * Mf);
      if (!(kappa > 0.0)) return TF_ERR_ARG;
    }
  }
  tf_ctx* c = (tf_ctx*)calloc(1, sizeof(tf_ctx));
  if (!c) return TF_ERR_NOMEM;
  c->p = *p;
  c->kappa = kappa;
  c->stream = (cudaStream_t)stream;
  c->ops = p->precision == TF_FP64 ? &tf::ops_fp64 : &tf::ops_f32b;
  c->N = (size_t)p->nx * (size_t)p->ny;
  tf::ModelK& mk = c->mk;
  mk.nx = p->nx;
  mk.ny = p->ny;
  mk.model = p->model;
  mk.n = p->n;
  mk.m = p->m;
  mk.inv_ds = 1.0 / p->ds;
  mk.inv_ds2 = mk.inv_ds * mk.inv_ds;
  mk.inv_ds3 = mk.inv_ds2 * mk.inv_ds;
  mk.C = p->cap_C;
  mk.A1 = kappa * (double)p->m * pow(p->b, p->m);
  mk.B1 = kappa * (double)p->n * pow(p->b, p->n);
  mk.c0 = p->c0;
  mk.c1 = p->c1;
  mk.nlc_K = p->nlc_K;
  mk.nlc_N = p->nlc_N;
  mk.nlc_beta = p->nlc_beta;
  mk.nlc_w = p->nlc_w;
  mk.b = p->b;
  mk.pol_C = p->pol_C;
  mk.pol_A1 = p->pol_A_SiOx;
  mk.pol_A2 = p->pol_A_Si;
  mk.pol_d = p->pol_d;
  c->grid_x = (p->ny + 31) / 32;
  c->grid_y = (p->nx + 31) / 32;
  c->grid_rx = (p->nx + 31) / 32;
  c->grid_ry = (p->ny + 31) / 32;
  {
    // residual strips: segments of 64 rows, halved (down to 16) until the
    // grid holds two waves of warps (about 24 resident per SM)
    const long strips = (p->nx + tf::kRhsStripCols - 1) / tf::kRhsStripCols;
    int rows = 64;
    while (rows > 16 && strips * ((p->ny + rows - 1) / rows) < 2L * 152 * 24) rows /= 2;
    const long warps = strips * ((p->ny + rows - 1) / rows);
    c->strip_n = (int)strips;
    c->strip_rows = rows;
    c->grid_pkx = (int)((warps + tf::kRhsStripWarps - 1) / tf::kRhsStripWarps);
  }
  c->packed_rhs = p->precision != TF_FP64 && p->model == TF_MODEL_POWERLAW && p->n == 3 && p->m == 2;
  c->n_rhs_parts = c->packed_rhs ? c->grid_pkx : c->grid_rx * c->grid_ry;
  c->grid_st_x = (p->nx + 15) / 16;
  c->grid_st_y = (p->ny + 15) / 16;
  c->grid_stats = 1216;  // 8 blocks of 256 threads per SM on 152 SMs
  {
    int a = c->n_rhs_parts + c->grid_x, b = c->grid_st_x * c->grid_st_y;
    c->n_px = a > b ? a : b;
  }
  c->n_py = c->grid_y > c->grid_stats ? c->grid_y : c->grid_stats;
  const size_t hp = c->ops->hp_bytes, lp = c->ops->lp_bytes;
  // factor scratch: one slab per block of 32 lines, line half and chunk
  const size_t facx = tf::fac_slab<tf::kCX>(c->grid_x, 0, 0, tf::chunks_per_half<tf::kCX>(p->nx));
  const size_t facy = tf::fac_slab<tf::kRY>(c->grid_y, 0, 0, tf::chunks_per_half<tf::kRY>(p->ny));
  int r = TF_OK;
  cudaError_t e = c->ops->prepare();
  if (e != cudaSuccess) r = cuda_fail(e);
  if (!r) r = dalloc(&c->bn, c->N * hp);
  if (!r) r = dalloc(&c->w, c->N * lp);
  if (!r && lp != sizeof(double)) r = dalloc(&c->ulp, c->N * lp);
  {
    int solver = p->line_solver;
    if (solver == TF_SOLVER_AUTO) {
      solver = tf_tuned_line_solver(p);
      if (solver < 0) solver = TF_SOLVER_TWISTED;
    }
    c->part = c->packed_rhs && solver == TF_SOLVER_PARTITIONED;
  }
  c->nsx = tf::part::nseg_x(p->nx);
  c->nsy = tf::part::nseg_y(p->ny);
  if (c->part) {
    const size_t rx = (size_t)(c->nsx - 1) * p->ny, ry = (size_t)(c->nsy - 1) * p->nx;
    if (!r) r = dalloc(&c->recx, rx * tf::part::kRecordValues * sizeof(float));
    if (!r) r = dalloc(&c->recy, ry * tf::part::kRecordValues * sizeof(float));
    if (!r) r = dalloc(&c->xsx, rx * 2 * sizeof(float));
    if (!r) r = dalloc(&c->xsy, ry * 2 * sizeof(float));
    if (!r) r = dalloc(&c->acc, tf::part::acc_bytes());
    if (!r && cudaMemset(c->acc, 0, tf::part::acc_bytes()) != cudaSuccess) r = TF_ERR_CUDA;
  } else {
    if (!r) r = dalloc(&c->fac_x, facx * lp);
    if (!r) r = dalloc(&c->fac_y, facy * lp);
  }
  if (!r) r = dalloc(&c->ubuf, c->N * sizeof(double));
  if (!r) r = dalloc(&c->ubuf2, c->N * sizeof(double));
  if (!r) r = dalloc(&c->px, (size_t)c->n_px * sizeof(tf::PartX));
  if (!r) r = dalloc(&c->py, (size_t)c->n_py * sizeof(tf::PartY));
  if (!r) r = dalloc(&c->dsc, sizeof(Scalars));
  if (!r) {
    e = cudaMallocHost((void**)&c->hsc, sizeof(Scalars));
    if (e != cudaSuccess) r = cuda_fail(e);
  }
  for (int k = 0; k < 8 && !r; ++k) {
    e = k < 7 ? cudaEventCreate(&c->ev[k]) : cudaEventCreateWithFlags(&c->ev[k], cudaEventDisableTiming);
    if (e != cudaSuccess) r = cuda_fail(e);
  }
  if (r) {
    tf_destroy(c);
    return r;
  }
  *out = c;
  return TF_OK;
}

int tf_residual(tf_ctx* c, const double* h_k, const double* h_old, double dt, double* G,
                tf_norms* out) {
  if (!c || !h_k || !h_old || !isfinite(dt)) return TF_ERR_ARG;
  TF_CK(c->ops->explicit_part(*c, h_old, dt));
  TF_CK(c->ops->residual_g(*c, h_k, dt, G ? G : c->ubuf));
  tf::k_grid_stats<<<c->grid_stats, 256, 0, c->stream>>>(h_k, c->N, c->py);
  TF_CK(cudaGetLastError());
  int r = finalize(*c, c->grid_st_x * c->grid_st_y, c->grid_stats);
  if (r) return r;
  if (out) {
    out->gnorm = c->hsc->gnorm;
    out->mass = tf::mass_value(c->hsc->mass);
    out->hmin = c->hsc->hmin;
  }
  return TF_OK;
}

int tf_newton_iteration(tf_ctx* c, const double* h_k, const double* h_old, double dt, double* w,
                        double* v, double* h_next, tf_step_info* info) {
  if (!c || !h_k || !h_old || !h_next || !isfinite(dt)) return TF_ERR_ARG;
  if (h_next == h_k || h_next == h_old) return TF_ERR_ARG;
  TF_CK(c->ops->explicit_part(*c, h_old, dt));
  Scalars s;
  int r = iterate(*c, h_k, dt, h_next, w, v, &s);
  if (r) return r;
  int status = classify(*c, s, 1, 0);
  r = film_stats(*c, h_next, &s);
  if (r) return r;
  fill_info(info, status, 1, s);
  return TF_OK;
}

int tf_newton_adi_step(tf_ctx* c, const double* h_old, double* h_new, double dt, tf_step_info* info) {
  if (!c || !h_old || !h_new || h_old == h_new || !(dt > 0.0) || !isfinite(dt)) return TF_ERR_ARG;
  return step(*c, h_old, h_new, dt, c->p.newton_fixed_iter, info);
}

int tf_advance(tf_ctx* c, double* h, double t0, double t_end, double dt0, int max_attempts,
               const double* dt_replay, const int* iter_replay, tf_step_record* records,
               tf_advance_info* info, int* streak_io) {
  if (!c || !h || !info || max_attempts < 0 || !(dt0 > 0.0) || !isfinite(t0)) return TF_ERR_ARG;
  if (streak_io && *streak_io < 0) return TF_ERR_ARG;
  memset(info, 0, sizeof(*info));
  const tf_params& P = c->p;
  double* cur = h;
  double* nxt = c->ubuf2;
  double t = t0, dt = dt0;
  int streak = streak_io ? *streak_io : 0, a = 0, status = TF_ADV_MAX_ATTEMPTS;
  while (a < max_attempts) {
    if (t >= t_end) {
      status = TF_ADV_DONE;
      break;
    }
    double step_dt;
    int last = 0, fixed = P.newton_fixed_iter;
    if (dt_replay) {
      step_dt = dt_replay[a];
      if (iter_replay) fixed = iter_replay[a];
      if (!(step_dt > 0.0)) return TF_ERR_ARG;
    } else if (t_end - t <= dt) {
      step_dt = t_end - t;
      last = 1;
    } else {
      step_dt = dt;
    }
    tf_step_info si;
    int s = step(*c, cur, nxt, step_dt, fixed, &si);
    if (s < 0) return s;
    if (records) {
      tf_step_record& rec = records[a];
      rec.t = t;
      rec.dt = step_dt;
      rec.accepted = s == TF_STEP_CONVERGED;
      rec.iterations = si.iterations;
      rec.status = s;
      rec.err = si.err;
      rec.gnorm = si.gnorm;
      rec.mass = si.mass;
      rec.hmin = si.hmin;
    }
    ++a;
    info->newton_iterations += si.iterations;
    if (s == TF_STEP_CONVERGED) {
      double* tmp = cur;
      cur = nxt;
      nxt = tmp;
      t = last ? t_end : t + step_dt;
      info->accepted++;
      if (!dt_replay && ++streak >= P.grow_after) {
        dt = fmin(dt * P.dt_grow, P.dt_max);
        streak = 0;
      }
      if (P.rupture_h > 0.0 && si.hmin < P.rupture_h) {
        status = TF_ADV_RUPTURE;
        break;
      }
    } else {
      if (dt_replay) {
        status = TF_ADV_DT_MIN;
        break;
      }
      streak = 0;
      dt = step_dt * P.dt_shrink;
      if (dt < P.dt_min) {
        status = TF_ADV_DT_MIN;
        break;
      }
    }
  }
  if (status == TF_ADV_MAX_ATTEMPTS && t >= t_end) status = TF_ADV_DONE;
  if (cur != h) {
    TF_CK(cudaMemcpyAsync(h, cur, c->N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    TF_CK(cudaStreamSynchronize(c->stream));
  }
  if (streak_io) *streak_io = streak;
  info->status = status;
  info->attempts = a;
  info->t = t;
  info->dt = dt;
  return TF_OK;
}

// ---------------------------------------------------------------------------
// Graph engine: a film's whole run as one launch of its context's graph
// (tf_ensemble_dev.cuh), with the controller state staged through pinned
// memory before and after it.

bool graph_capable(const tf_ctx& c) { return c.ops->ens_graph && c.packed_rhs && !c.part; }

int film_graph_start(tf_ctx& c, double* h, double t0, double t_end, double dt0, int max_att, int streak) {
  if (!c.ens_exec) {  // first use; a failed earlier build keeps its buffers
    if (!c.ens_dev) {
      int r = dalloc((void**)&c.ens_dev, sizeof(tf::EnsDev));
      if (r) return r;
    }
    if (!c.ens_host) TF_CK(cudaMallocHost((void**)&c.ens_host, sizeof(tf::EnsDev)));
    TF_CK(c.ops->ens_graph(c, c.ens_dev, &c.ens_exec));
  }
  tf::EnsDev& e = *c.ens_host;
  memset(&e, 0, sizeof(e));
  const tf_params& P = c.p;
  e.p.cur = h;
  e.p.nxt = c.ubuf2;
  e.ubuf = c.ubuf;
  e.M = c.mk;
  e.theta = P.theta;
  e.tol = P.newton_tol;
  e.dt_max = P.dt_max;
  e.dt_min = P.dt_min;
  e.dt_grow = P.dt_grow;
  e.dt_shrink = P.dt_shrink;
  e.rupture_h = P.rupture_h;
  e.grow_after = P.grow_after;
  e.max_iter = P.newton_max_iter;
  e.fixed_iter = P.newton_fixed_iter;
  e.t = t0;
  e.t_end = t_end;
  e.dt = dt0;
  e.max_att = max_att;
  e.streak = streak;
  e.status = TF_ADV_MAX_ATTEMPTS;
  TF_CK(cudaMemcpyAsync(c.ens_dev, &e, sizeof(e), cudaMemcpyHostToDevice, c.stream));
  TF_CK(cudaGraphLaunch(c.ens_exec, c.stream));
  TF_CK(cudaMemcpyAsync(c.ens_host, c.ens_dev, sizeof(e), cudaMemcpyDeviceToHost, c.stream));
  return TF_OK;
}

// After the graph: what film_finish does, from the staged state.
int film_graph_finish(tf_ctx& c, double* h, tf_advance_info* info, int* streak_io) {
  TF_CK(cudaStreamSynchronize(c.stream));
  const tf::EnsDev& e = *c.ens_host;
  int status = e.status;
  if (status == TF_ADV_MAX_ATTEMPTS && e.t >= e.t_end) status = TF_ADV_DONE;
  if (e.p.cur != h) {
    TF_CK(cudaMemcpyAsync(h, e.p.cur, c.N * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    TF_CK(cudaStreamSynchronize(c.stream));
  }
  memset(info, 0, sizeof(*info));
  info->status = status;
  info->attempts = e.a;
  info->accepted = e.accepted;
  info->newton_iterations = e.newton_iterations;
  info->t = e.t;
  info->dt = e.dt;
  if (streak_io) *streak_io = e.streak;
  if (c.timing.enabled) c.timing.launches += (int)e.kernels;
  return TF_OK;
}

int tf_ensemble_advance(int n, tf_ctx* const* ctx, double* const* h, const double* t0,
                        const double* t_end, const double* dt0, const int* max_attempts,
                        tf_advance_info* info, int* streak, int engine) {
  if (n < 0 || (n > 0 && (!ctx || !h || !t0 || !t_end || !dt0 || !max_attempts || !info)))
    return TF_ERR_ARG;
  if (engine != TF_ENSEMBLE_AUTO && engine != TF_ENSEMBLE_HOST) return TF_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    if (!ctx[i] || !h[i] || max_attempts[i] < 0 || !(dt0[i] > 0.0) || !isfinite(t0[i])) return TF_ERR_ARG;
    if (streak && streak[i] < 0) return TF_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (ctx[j] == ctx[i]) return TF_ERR_ARG;  // one context per film
  }
  // films on the graph engine: launched first, collected at the end
  std::vector<char> on_graph((size_t)n, 0);
  for (int i = 0; i < n; ++i) {
    if (engine != TF_ENSEMBLE_AUTO || !graph_capable(*ctx[i])) continue;
    on_graph[(size_t)i] = 1;
    int r = film_graph_start(*ctx[i], h[i], t0[i], t_end[i], dt0[i], max_attempts[i], streak ? streak[i] : 0);
    if (r) return r;
  }
  std::vector<FilmRun> F((size_t)n);
  int active = 0;
  for (int i = 0; i < n; ++i) {
    FilmRun& f = F[(size_t)i];
    memset(&f, 0, sizeof(f));
    f.c = ctx[i];
    if (on_graph[(size_t)i]) {
      f.done = true;
      continue;
    }
    f.h = h[i];
    f.t = t0[i];
    f.t_end = t_end[i];
    f.dt = dt0[i];
    f.max_att = max_attempts[i];
    f.info = &info[i];
    memset(f.info, 0, sizeof(*f.info));
    f.streak_io = streak ? &streak[i] : nullptr;
    f.streak = streak ? streak[i] : 0;
    f.cur = h[i];
    f.nxt = ctx[i]->ubuf2;
    f.status = TF_ADV_MAX_ATTEMPTS;
    int r = film_start_attempt(f);
    if (r) return r;
    if (!f.done) ++active;
  }
  // Several host threads share the films (film i goes to thread i % T), so
  // that launching the kernels of small films does not become the limit.
  int dev = 0;
  TF_CK(cudaGetDevice(&dev));
  const int T = active < 1 ? 1 : (active < 4 ? active : 4);
  std::vector<int> err((size_t)T, TF_OK);
  auto worker = [&](int w) {
    if (cudaSetDevice(dev) != cudaSuccess) {
      err[(size_t)w] = TF_ERR_CUDA;
      return;
    }
    int left = 0;
    for (int i = w; i < n; i += T) left += F[(size_t)i].done ? 0 : 1;
    while (left > 0) {
      bool progressed = false;
      for (int i = w; i < n; i += T) {
        FilmRun& f = F[(size_t)i];
        if (f.done) continue;
        const cudaError_t q = cudaEventQuery(f.c->ev[7]);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) {
          err[(size_t)w] = cuda_fail(q);
          return;
        }
        progressed = true;
        const int r = f.phase == 1 ? film_on_iteration(f) : film_on_stats(f);
        if (r) {
          err[(size_t)w] = r;
          return;
        }
        if (f.done) --left;
      }
      if (!progressed) std::this_thread::yield();
    }
  };
  std::vector<std::thread> pool;
  for (int w = 1; w < T; ++w) pool.emplace_back(worker, w);
  worker(0);
  for (std::thread& t : pool) t.join();
  for (int e : err)
    if (e) return e;
  for (FilmRun& f : F) TF_CK(cudaStreamSynchronize(f.c->stream));
  for (int i = 0; i < n; ++i) {
    if (!on_graph[(size_t)i]) continue;
    int r = film_graph_finish(*ctx[i], h[i], &info[i], streak ? &streak[i] : nullptr);
    if (r) return r;
  }
  return TF_OK;
}

int tf_line_solver(const tf_ctx* c) {
  if (!c) return -1;
  return c->part ? TF_SOLVER_PARTITIONED : TF_SOLVER_TWISTED;
}

int tf_tuned_line_solver(const tf_params* p) {
  if (!p) return -1;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  const TuneKey k = tune_key(*p);
  for (const auto& e : g_tune)
    if (e.first == k) return e.second;
  return -1;
}

int tf_tune_line_solver(const tf_params* p, void* stream, const double* h, double dt, int iters, int copies,
                        int* best, double* ms) {
  if (!p || !h || !best || iters < 1 || copies < 1 || copies > 256 || !(dt > 0.0) || !isfinite(dt))
    return TF_ERR_ARG;
  double t[2] = {-1.0, -1.0};
  cudaStream_t s0 = (cudaStream_t)stream;
  for (int sv = TF_SOLVER_TWISTED; sv <= TF_SOLVER_PARTITIONED; ++sv) {
    tf_params q = *p;
    q.line_solver = sv;
    // `copies` films on streams of their own, each iterating from h (read
    // only): the throughput a solver gives when many films share the GPU
    std::vector<tf_ctx*> ctx((size_t)copies, nullptr);
    std::vector<cudaStream_t> st((size_t)copies, nullptr);
    int rc = TF_OK;
    for (int k = 0; k < copies && !rc; ++k) {
      if (cudaStreamCreateWithFlags(&st[(size_t)k], cudaStreamNonBlocking) != cudaSuccess) {
        rc = TF_ERR_CUDA;
        break;
      }
      rc = tf_init(&q, st[(size_t)k], &ctx[(size_t)k]);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = TF_ERR_CUDA;
    if (!rc && cudaStreamSynchronize(s0) != cudaSuccess) rc = TF_ERR_CUDA;  // h is ready
    for (int k = 0; k < copies && !rc; ++k)
      if (ctx[(size_t)k]->ops->explicit_part(*ctx[(size_t)k], h, dt) != cudaSuccess) rc = TF_ERR_CUDA;
    // one untimed round, then `iters` timed rounds; each round queues one
    // Newton iteration on every film, then waits for all of them (a
    // round's host round trip is part of an iteration's cost)
    for (int it = 0; it <= iters && !rc; ++it) {
      if (it == 1) {
        if (cudaDeviceSynchronize() != cudaSuccess || cudaEventRecord(e0, s0) != cudaSuccess) rc = TF_ERR_CUDA;
      }
      for (int k = 0; k < copies && !rc; ++k)
        rc = iterate_launch(*ctx[(size_t)k], h, dt, ctx[(size_t)k]->ubuf2, nullptr, nullptr);
      for (int k = 0; k < copies && !rc; ++k)
        if (cudaStreamSynchronize(st[(size_t)k]) != cudaSuccess) rc = TF_ERR_CUDA;
    }
    if (!rc && (cudaEventRecord(e1, s0) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
      rc = TF_ERR_CUDA;
    float el = 0.0f;
    if (!rc && cudaEventElapsedTime(&el, e0, e1) != cudaSuccess) rc = TF_ERR_CUDA;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (int k = 0; k < copies; ++k) {
      tf_destroy(ctx[(size_t)k]);
      if (st[(size_t)k]) cudaStreamDestroy(st[(size_t)k]);
    }
    if (rc == TF_ERR_ARG && sv == TF_SOLVER_PARTITIONED) continue;  // not applicable
    if (rc) return rc;
    t[sv] = (double)el / iters / copies;  // ms per film iteration
  }
  const int choice = (t[1] >= 0.0 && t[1] < t[0]) ? TF_SOLVER_PARTITIONED : TF_SOLVER_TWISTED;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    const TuneKey k = tune_key(*p);
    bool found = false;
    for (auto& e : g_tune)
      if (e.first == k) {
        e.second = choice;
        found = true;
      }
    if (!found) g_tune.emplace_back(k, choice);
  }
  *best = choice;
  if (ms) {
    ms[0] = t[0];
    ms[1] = t[1];
  }
  return TF_OK;
}

int tf_timing_enable(tf_ctx* c, int on) {
  if (!c) return TF_ERR_ARG;
  memset(&c->timing, 0, sizeof(c->timing));
  c->timing.enabled = on ? 1 : 0;
  return TF_OK;
}

int tf_timing_get(const tf_ctx* c, tf_timing* out) {
  if (!c || !out) return TF_ERR_ARG;
  *out = c->timing;
  return TF_OK;
}

}  // extern "C"
