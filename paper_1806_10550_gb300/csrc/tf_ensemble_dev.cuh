// tf_ensemble_dev.cuh -- the device-resident step controller of an ensemble
// film (the graph engine of tf_ensemble_advance).
//
// tf_advance's controller and the Newton loop of a time step (Sec. Adaptive
// Time Stepping, Fig. FlowChartTime; the pseudo-Newton iteration of eqs.
// JacobianSystem1-3) move into device memory and into k_ens_begin and the
// two reduction kernels k_ens_iter and k_ens_step, which finish with the
// controller in their thread 0, so that a film's whole run is one CUDA graph:
// an outer conditional WHILE over attempts and an inner one over the Newton
// iterations after the first, whose conditions these kernels set.  Every decision is the host's, made with the same
// double arithmetic on the same scalars (the reductions' Scalars in device
// memory), so a film advanced here takes the steps, iteration counts and
// bits that tf_advance gives it.  The kernels of the path read the step's
// constants and the iterates' addresses from EnsDev (their optional
// device-pointer arguments).
#pragma once

#include "tf_internal.h"
#include "tf_rhs_packed.cuh"

namespace tf {

// Addresses that change within a run (read by the kernels of the path).
struct EnsPtrs {
  const double* uk;  // iterate of the Newton iteration in flight (u_0 = u^n = cur)
  double* un;        // its result u_k+1
  double* cur;       // the film at time t
  double* nxt;       // the step's result; swapped with cur when the step is accepted
};

struct EnsDev {
  EnsPtrs p;
  double* ubuf;            // second iterate buffer of a step
  // the step in flight: its residual constants (explicit part with the first
  // residual; residual) and band constants, computed here from step_dt
  StripK rk_both, rk_res;
  LineK<float> line;
  ModelK M;
  // parameters (tf_params)
  double theta, tol, dt_max, dt_min, dt_grow, dt_shrink, rupture_h;
  int grow_after, max_iter, fixed_iter;
  // controller state (FilmRun's)
  double t, t_end, dt, step_dt;
  int a, max_att, streak, last, k, kmax, it, sstatus, status, done;
  int accepted, newton_iterations;
  unsigned long long kernels;  // kernel launches the graph ran for this film
};

TF_HD int ens_classify(const Scalars& s, int it, int fixed_iter, double tol) {
  if (s.pivot) return TF_STEP_ZERO_PIVOT;
  if (s.nonfinite) return TF_STEP_NONPOSITIVE;
  if (fixed_iter > 0) return it >= fixed_iter ? TF_STEP_CONVERGED : TF_STEP_NOT_CONVERGED;
  if (s.err < tol) return TF_STEP_CONVERGED;
  return TF_STEP_NOT_CONVERGED;
}

// Start the next attempt: false when the film is done (attempt budget spent
// or t_end reached).  The step's Δt is clipped to land on t_end.
__device__ __forceinline__ bool ens_start_attempt(EnsDev& e) {
  if (e.a >= e.max_att) {
    e.done = 1;
    return false;
  }
  if (e.t >= e.t_end) {
    e.status = TF_ADV_DONE;
    e.done = 1;
    return false;
  }
  e.last = 0;
  if (e.t_end - e.t <= e.dt) {
    e.step_dt = e.t_end - e.t;
    e.last = 1;
  } else {
    e.step_dt = e.dt;
  }
  StepK K;
  K.theta_dt = e.theta * e.step_dt;
  K.expl_dt = (1.0 - e.theta) * e.step_dt;
  e.rk_both = strip_consts(e.M, K, true);
  e.rk_res = strip_consts(e.M, K, false);
  e.line = line_consts<float>(e.M, K);
  e.kmax = e.fixed_iter > 0 ? e.fixed_iter : e.max_iter;
  e.k = 0;
  e.it = 0;
  e.sstatus = TF_STEP_NOT_CONVERGED;
  e.p.uk = e.p.cur;
  e.p.un = e.p.nxt;
  return true;
}

// Before the outer loop: the first attempt.  (The kernel counts below are
// the graph's launches for this film: this kernel; per iteration the x and
// y sweeps and the reductions, and the residual from the second on; per
// attempt the explicit part, the copy, the statistics and their reductions.)
static __global__ void k_ens_begin(EnsDev* __restrict__ e, cudaGraphConditionalHandle outer) {
  e->kernels += 1;
  cudaGraphSetConditional(outer, ens_start_attempt(*e) ? 1u : 0u);
}

// A Newton iteration's reductions (k_finalize's), then in thread 0: classify
// the iteration as step() does, and either run the next iteration (into the
// other iterate buffer) or end the step.
static __global__ void __launch_bounds__(256)
    k_ens_iter(const PartX* __restrict__ px, int nx_part, const PartY* __restrict__ py, int ny_part,
               Scalars* __restrict__ out, EnsDev* __restrict__ e, cudaGraphConditionalHandle inner) {
  if (!finalize_block(px, nx_part, py, ny_part, out)) return;
  EnsDev& E = *e;
  const Scalars s = *out;
  E.kernels += E.k == 0 ? 3 : 4;
  E.it = E.k + 1;
  E.p.uk = E.p.un;
  E.sstatus = ens_classify(s, E.it, E.fixed_iter, E.tol);
  ++E.k;
  const bool more = E.sstatus == TF_STEP_NOT_CONVERGED && E.k < E.kmax;
  if (more) E.p.un = (E.k & 1) ? E.ubuf : E.p.nxt;
  cudaGraphSetConditional(inner, more ? 1u : 0u);
}

// The step's result into nxt when the last iterate is in the other buffer.
static __global__ void __launch_bounds__(256) k_ens_copy(const EnsDev* __restrict__ e, size_t N) {
  const double* src = e->p.uk;
  double* dst = e->p.nxt;
  if (src == dst) return;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x)
    dst[k] = src[k];
}

// The step's film statistics (k_finalize's reduction of k_grid_stats), then
// in thread 0 tf_advance's controller (accept or reject, Δt growth after
// grow_after accepted steps in a row, rupture, Δt floor) and the next
// attempt.
static __global__ void __launch_bounds__(256)
    k_ens_step(const PartY* __restrict__ py, int ny_part, Scalars* __restrict__ out, EnsDev* __restrict__ e,
               cudaGraphConditionalHandle outer) {
  if (!finalize_block(nullptr, 0, py, ny_part, out)) return;
  EnsDev& E = *e;
  const Scalars* s = out;
  E.kernels += 4;
  ++E.a;
  E.newton_iterations += E.it;
  bool go = false;
  if (E.sstatus == TF_STEP_CONVERGED) {
    double* tmp = E.p.cur;
    E.p.cur = E.p.nxt;
    E.p.nxt = tmp;
    E.t = E.last ? E.t_end : E.t + E.step_dt;
    E.accepted++;
    if (++E.streak >= E.grow_after) {
      E.dt = fmin(E.dt * E.dt_grow, E.dt_max);
      E.streak = 0;
    }
    if (E.rupture_h > 0.0 && s->hmin < E.rupture_h) {
      E.status = TF_ADV_RUPTURE;
      E.done = 1;
    } else {
      go = ens_start_attempt(E);
    }
  } else {
    E.streak = 0;
    E.dt = E.step_dt * E.dt_shrink;
    if (E.dt < E.dt_min) {
      E.status = TF_ADV_DT_MIN;
      E.done = 1;
    } else {
      go = ens_start_attempt(E);
    }
  }
  cudaGraphSetConditional(outer, go ? 1u : 0u);
}

}  // namespace tf
