// tf_mode.cuh -- launchers of one precision mode; included once by
// tf_mode_fp64.cu and once by tf_mode_f32b.cu.
#pragma once

#include <type_traits>
#include <vector>

#include "tf_internal.h"
#include "tf_rhs_packed.cuh"
#include "tf_ensemble_dev.cuh"

static_assert(tf::kRhsStripCols == tf::kSW && tf::kRhsStripWarps == tf::kSWarps, "residual strips of the launch grid");

namespace tf {

template <class Mode> struct Launch {
  typedef typename Mode::HP HP;
  typedef typename Mode::LP LP;
  static constexpr size_t smem_stencil = sizeof(StencilSmem<HP, 16, 16>);
  static constexpr size_t smem_rhs = sizeof(RhsSmem<HP, 32>);
  static constexpr bool kF32B = std::is_same<Mode, ModeF32B>::value;
  static constexpr size_t smem_x = sizeof(XSmem<LP>);
  static constexpr size_t smem_y = sizeof(YSmem<LP>);

  static StepK step(const tf_ctx& c, double dt) {
    StepK k;
    k.theta_dt = c.p.theta * dt;
    k.expl_dt = (1.0 - c.p.theta) * dt;
    return k;
  }

  static cudaError_t prepare() {
    cudaError_t e;
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if ((e = cudaFuncSetAttribute(k_stencil<Mode, 0>, A, (int)smem_stencil))) return e;
    if ((e = cudaFuncSetAttribute(k_stencil<Mode, 1>, A, (int)smem_stencil))) return e;
    if ((e = cudaFuncSetAttribute(k_rhs<Mode, kRhsResidual>, A, (int)smem_rhs))) return e;
    if ((e = cudaFuncSetAttribute(k_rhs<Mode, kRhsExplicit>, A, (int)smem_rhs))) return e;
    if ((e = cudaFuncSetAttribute(k_rhs<Mode, kRhsBoth>, A, (int)smem_rhs))) return e;
    if ((e = cudaFuncSetAttribute(k_xsweep<Mode>, A, (int)smem_x))) return e;
    if ((e = cudaFuncSetAttribute(k_ysweep<Mode>, A, (int)smem_y))) return e;
    // the sweeps run two blocks per SM only with the largest shared carveout
    const cudaFuncAttribute C = cudaFuncAttributePreferredSharedMemoryCarveout;
    if ((e = cudaFuncSetAttribute(k_xsweep<Mode>, C, (int)cudaSharedmemCarveoutMaxShared))) return e;
    if ((e = cudaFuncSetAttribute(k_ysweep<Mode>, C, (int)cudaSharedmemCarveoutMaxShared))) return e;
    if ((e = cudaFuncSetAttribute(k_rhs<Mode, kRhsExplicit>, C, (int)cudaSharedmemCarveoutMaxShared))) return e;
    if ((e = cudaFuncSetAttribute(k_rhs<Mode, kRhsBoth>, C, (int)cudaSharedmemCarveoutMaxShared))) return e;
    if constexpr (kF32B) {
      if ((e = part::prepare())) return e;
      // the sweeps of the ensemble graphs (constants from device memory)
      if ((e = cudaFuncSetAttribute(k_xsweep<Mode, true>, A, (int)smem_x))) return e;
      if ((e = cudaFuncSetAttribute(k_ysweep<Mode, true>, A, (int)smem_y))) return e;
      if ((e = cudaFuncSetAttribute(k_xsweep<Mode, true>, C, (int)cudaSharedmemCarveoutMaxShared))) return e;
      if ((e = cudaFuncSetAttribute(k_ysweep<Mode, true>, C, (int)cudaSharedmemCarveoutMaxShared))) return e;
    }
    return cudaFuncSetAttribute(k_rhs<Mode, kRhsResidual>, C, (int)cudaSharedmemCarveoutMaxShared);
  }

  static cudaError_t explicit_part_c(tf_ctx& c, const double* u_old, double dt) {
    c.expl_kernels = 1;
    if constexpr (kF32B) {
      if (c.packed_rhs) {
        k_rhs_strip<kRhsExplicit><<<c.grid_pkx, kST, 0, c.stream>>>(
            c.mk, strip_consts(c.mk, step(c, dt), true), u_old, (HP*)c.bn, nullptr, nullptr, nullptr, c.strip_n, c.strip_rows);
        return cudaGetLastError();
      }
    }
    dim3 grid(c.grid_rx, c.grid_ry);
    k_rhs<Mode, kRhsExplicit><<<grid, 256, smem_rhs, c.stream>>>(c.mk, rhs_consts<HP>(c.mk, step(c, dt), true), u_old,
                                                         (HP*)c.bn, nullptr, nullptr, nullptr);
    return cudaGetLastError();
  }
  static cudaError_t residual_c(tf_ctx& c, const double* u_k, double dt, double* G) {
    dim3 grid(c.grid_st_x, c.grid_st_y), block(16, 16);
    k_stencil<Mode, 1><<<grid, block, smem_stencil, c.stream>>>(c.mk, step(c, dt), u_k, (HP*)c.bn,
                                                                G, c.px);
    return cudaGetLastError();
  }
  static cudaError_t rhs_c(tf_ctx& c, const double* u_k, double dt) {
    if constexpr (kF32B) {
      if (c.packed_rhs) {
        k_rhs_strip<kRhsResidual><<<c.grid_pkx, kST, 0, c.stream>>>(
            c.mk, strip_consts(c.mk, step(c, dt), false), u_k, (HP*)c.bn, (LP*)c.w, (LP*)c.ulp, c.px, c.strip_n, c.strip_rows);
        return cudaGetLastError();
      }
    }
    dim3 grid(c.grid_rx, c.grid_ry);
    k_rhs<Mode, kRhsResidual><<<grid, 256, smem_rhs, c.stream>>>(c.mk, rhs_consts<HP>(c.mk, step(c, dt)), u_k,
                                                   (HP*)c.bn, (LP*)c.w,
                                                   (LP*)c.ulp, c.px);
    return cudaGetLastError();
  }
  // b^n of a step and the right side of its first iteration (u_0 = u^n)
  // from one D(u^n); results equal explicit_part_c then rhs_c.
  static cudaError_t explicit_rhs0_c(tf_ctx& c, const double* u_old, double dt) {
    c.expl_kernels = 1;
    if constexpr (kF32B) {
      if (c.packed_rhs) {
        k_rhs_strip<kRhsBoth><<<c.grid_pkx, kST, 0, c.stream>>>(
            c.mk, strip_consts(c.mk, step(c, dt), true), u_old, (HP*)c.bn, (LP*)c.w, (LP*)c.ulp, c.px, c.strip_n, c.strip_rows);
        return cudaGetLastError();
      }
    }
    c.expl_kernels = 1;
    dim3 grid(c.grid_rx, c.grid_ry);
    k_rhs<Mode, kRhsBoth><<<grid, 256, smem_rhs, c.stream>>>(c.mk, rhs_consts<HP>(c.mk, step(c, dt), true), u_old,
                                                             (HP*)c.bn, (LP*)c.w, (LP*)c.ulp, c.px);
    return cudaGetLastError();
  }
  // film the sweeps stage: u_k itself in FP64, its FP32 copy (written by
  // k_rhs of the same iteration) in FP32-bulk
  static const LP* film_lp(const tf_ctx& c, const double* u_k) {
    return sizeof(LP) == sizeof(double) ? (const LP*)u_k : (const LP*)c.ulp;
  }
  static cudaError_t xsweep_c(tf_ctx& c, double dt, const double* u_k) {
    if constexpr (kF32B) {
      if (c.part) return part::xsweep(c, dt);
    }
    k_xsweep<Mode><<<c.grid_x, kSweepThreads, smem_x, c.stream>>>(c.mk, line_consts<LP>(c.mk, step(c, dt)),
                                                       film_lp(c, u_k), (LP*)c.w,
                                                       (LP*)c.fac_x, c.px + c.n_rhs_parts);
    return cudaGetLastError();
  }
  static cudaError_t ysweep_c(tf_ctx& c, const double* u_k, double dt, double* u_next,
                              double* v_out) {
    if constexpr (kF32B) {
      if (c.part) return part::ysweep(c, u_k, dt, u_next, v_out);
    }
    k_ysweep<Mode><<<c.grid_y, kSweepThreads, smem_y, c.stream>>>(c.mk, line_consts<LP>(c.mk, step(c, dt)),
                                                       u_k, film_lp(c, u_k),
                                                       (const LP*)c.w,
                                                       (LP*)c.fac_y, u_next, v_out, c.py);
    return cudaGetLastError();
  }
  // The whole run of an ensemble film as one graph (FP32-bulk, (3, 2) power
  // law, twisted sweeps): k_ens_begin, then WHILE (attempts) { explicit part
  // with the first residual, x sweep, y sweep, k_ens_iter (reductions and
  // the iteration's classification); WHILE (further iterations) { residual,
  // x sweep, y sweep, k_ens_iter }; copy of the result, film statistics,
  // k_ens_step (their reductions and the step controller) }.  The kernels
  // and their order are those of a tf_advance step, with their constants and
  // grids read from e.
  static cudaError_t ens_graph_c(tf_ctx& c, EnsDev* e, cudaGraphExec_t* out) {
    if constexpr (!kF32B) {
      return cudaErrorNotSupported;
    } else {
      if (!c.packed_rhs || c.part) return cudaErrorNotSupported;
      cudaStream_t s = nullptr;
      cudaGraph_t g = nullptr, B = nullptr, I = nullptr;
      cudaError_t err = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
      if (err) return err;
      const cudaStreamCaptureMode md = cudaStreamCaptureModeRelaxed;
      const StripK rk0 = strip_consts(c.mk, step(c, 1.0), false);  // placeholders: read from e
      const LineK<LP> l0 = line_consts<LP>(c.mk, step(c, 1.0));
      cudaGraphConditionalHandle ho, hi;
      cudaGraphNode_t nb = nullptr, no = nullptr, nx = nullptr, ni = nullptr;
      size_t one = 1;
      auto fail = [&](cudaError_t x) {
        cudaStreamDestroy(s);
        if (g) cudaGraphDestroy(g);
        return x;
      };
      // one Newton iteration's sweeps and reductions
      auto sweeps = [&]() {
        k_xsweep<Mode, true><<<c.grid_x, kSweepThreads, smem_x, s>>>(c.mk, l0, (const LP*)c.ulp, (LP*)c.w,
                                                                     (LP*)c.fac_x, c.px + c.n_rhs_parts, &e->line);
        k_ysweep<Mode, true><<<c.grid_y, kSweepThreads, smem_y, s>>>(c.mk, l0, nullptr, (const LP*)c.ulp,
                                                                     (const LP*)c.w, (LP*)c.fac_y, nullptr, nullptr,
                                                                     c.py, &e->line, &e->p.uk);
        k_ens_iter<<<1, 256, 0, s>>>(c.px, c.n_rhs_parts + c.grid_x, c.py, c.grid_y, c.dsc, e, hi);
      };
      if ((err = cudaGraphCreate(&g, 0))) return fail(err);
      if ((err = cudaGraphConditionalHandleCreate(&ho, g, 0, cudaGraphCondAssignDefault))) return fail(err);
      // top level: the first attempt
      if ((err = cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, md))) return fail(err);
      k_ens_begin<<<1, 1, 0, s>>>(e, ho);
      if ((err = cudaStreamEndCapture(s, &g))) return fail(err);
      if ((err = cudaGraphGetNodes(g, &nb, &one)) || one != 1) return fail(err ? err : cudaErrorUnknown);
      cudaGraphNodeParams po = {};
      po.type = cudaGraphNodeTypeConditional;
      po.conditional.handle = ho;
      po.conditional.type = cudaGraphCondTypeWhile;
      po.conditional.size = 1;
      if ((err = cudaGraphAddNode(&no, g, &nb, nullptr, 1, &po))) return fail(err);
      B = po.conditional.phGraph_out[0];
      // attempt: the explicit part with the first iteration's residual, and
      // the first iteration
      if ((err = cudaGraphConditionalHandleCreate(&hi, B, 0, cudaGraphCondAssignDefault))) return fail(err);
      if ((err = cudaStreamBeginCaptureToGraph(s, B, nullptr, nullptr, 0, md))) return fail(err);
      k_rhs_strip<kRhsBoth, true><<<c.grid_pkx, kST, 0, s>>>(c.mk, rk0, nullptr, (HP*)c.bn, (LP*)c.w, (LP*)c.ulp, c.px,
                                                             c.strip_n, c.strip_rows, &e->rk_both, &e->p.cur);
      sweeps();
      if ((err = cudaStreamEndCapture(s, &B))) return fail(err);
      {  // the last node of the chain: the one no other node depends on
        size_t nn = 0, ne = 0;
        if ((err = cudaGraphGetNodes(B, nullptr, &nn))) return fail(err);
        std::vector<cudaGraphNode_t> nodes(nn);
        if ((err = cudaGraphGetNodes(B, nodes.data(), &nn))) return fail(err);
        for (cudaGraphNode_t n : nodes) {
          if ((err = cudaGraphNodeGetDependentNodes(n, nullptr, nullptr, &ne))) return fail(err);
          if (ne == 0) nx = n;
        }
        if (!nx) return fail(cudaErrorUnknown);
      }
      cudaGraphNodeParams pi = {};
      pi.type = cudaGraphNodeTypeConditional;
      pi.conditional.handle = hi;
      pi.conditional.type = cudaGraphCondTypeWhile;
      pi.conditional.size = 1;
      if ((err = cudaGraphAddNode(&ni, B, &nx, nullptr, 1, &pi))) return fail(err);
      I = pi.conditional.phGraph_out[0];
      // the iterations after the first
      if ((err = cudaStreamBeginCaptureToGraph(s, I, nullptr, nullptr, 0, md))) return fail(err);
      k_rhs_strip<kRhsResidual, true><<<c.grid_pkx, kST, 0, s>>>(c.mk, rk0, nullptr, (HP*)c.bn, (LP*)c.w, (LP*)c.ulp,
                                                                 c.px, c.strip_n, c.strip_rows, &e->rk_res, &e->p.uk);
      sweeps();
      if ((err = cudaStreamEndCapture(s, &I))) return fail(err);
      // end of the attempt: the result into nxt, its statistics, the controller
      if ((err = cudaStreamBeginCaptureToGraph(s, B, &ni, nullptr, 1, md))) return fail(err);
      k_ens_copy<<<1024, 256, 0, s>>>(e, c.N);
      k_grid_stats<<<c.grid_stats, 256, 0, s>>>(nullptr, c.N, c.py, &e->p.nxt);
      k_ens_step<<<1, 256, 0, s>>>(c.py, c.grid_stats, c.dsc, e, ho);
      if ((err = cudaStreamEndCapture(s, &B))) return fail(err);
      cudaGraphExec_t x = nullptr;  // *out only ever holds an instantiated graph
      if ((err = cudaGraphInstantiate(&x, g, 0))) return fail(err);
      *out = x;
      cudaGraphDestroy(g);
      cudaStreamDestroy(s);
      return cudaSuccess;
    }
  }
  static cudaError_t w_to_f64_c(tf_ctx& c, double* out) {
    if (sizeof(LP) == sizeof(double))
      return cudaMemcpyAsync(out, c.w, c.N * sizeof(double), cudaMemcpyDeviceToDevice, c.stream);
    k_to_f64<LP><<<1024, 256, 0, c.stream>>>((const LP*)c.w, out, c.N);
    return cudaGetLastError();
  }
};

template <class Mode> Ops make_ops() {
  typedef Launch<Mode> L;
  Ops o;
  o.hp_bytes = sizeof(typename Mode::HP);
  o.lp_bytes = sizeof(typename Mode::LP);
  o.prepare = &L::prepare;
  o.explicit_part = &L::explicit_part_c;
  o.explicit_rhs0 = &L::explicit_rhs0_c;
  o.residual_g = &L::residual_c;
  o.rhs = &L::rhs_c;
  o.xsweep = &L::xsweep_c;
  o.ysweep = &L::ysweep_c;
  o.w_to_f64 = &L::w_to_f64_c;
  o.ens_graph = L::kF32B ? &L::ens_graph_c : nullptr;
  return o;
}

}  // namespace tf
