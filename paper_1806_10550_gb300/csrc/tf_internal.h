// tf_internal.h -- context and per-mode launch table shared by the C-ABI
// layer (tf_api.cu) and the two precision instantiations (tf_mode_*.cu).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "../../include/tf.h"
#include "tf_line_sweeps.cuh"

namespace tf {

// strips of the packed FP32-bulk residual kernel (k_rhs_strip, tf_rhs_packed.cuh):
// output columns per warp and warps per block
constexpr int kRhsStripCols = 60, kRhsStripWarps = 4;

}  // namespace tf

struct tf_ctx;

namespace tf {

struct EnsDev;

struct Ops {
  size_t hp_bytes, lp_bytes;
  cudaError_t (*prepare)();
  cudaError_t (*explicit_part)(tf_ctx& c, const double* u_old, double dt);
  // explicit part plus the first iteration's right side (u_0 = u_old)
  cudaError_t (*explicit_rhs0)(tf_ctx& c, const double* u_old, double dt);
  cudaError_t (*residual_g)(tf_ctx& c, const double* u_k, double dt, double* G);
  cudaError_t (*rhs)(tf_ctx& c, const double* u_k, double dt);
  cudaError_t (*xsweep)(tf_ctx& c, double dt, const double* u_k);
  cudaError_t (*ysweep)(tf_ctx& c, const double* u_k, double dt, double* u_next, double* v_out);
  cudaError_t (*w_to_f64)(tf_ctx& c, double* out);
  // The graph of a whole ensemble film run (tf_ensemble_dev.cuh) for
  // contexts on the FP32-bulk power-law twisted path; NULL for the others.
  cudaError_t (*ens_graph)(tf_ctx& c, EnsDev* e, cudaGraphExec_t* out);
};

extern const Ops ops_fp64;
extern const Ops ops_f32b;

// Partitioned line solves of the FP32-bulk path (tf_part.cu, kernels in
// tf_partition.cuh).
namespace part {
struct Acc;
constexpr int kRecordValues = 20;  // reduced-system values per separator and line
int nseg_x(int nx);  // segments of an x line
int nseg_y(int ny);  // segments of a y line
size_t acc_bytes();
cudaError_t prepare();
// x phases 1-3 (writes w over the right side in c.w) and y phases 1-2
cudaError_t xsweep(tf_ctx& c, double dt);
// y phase 3, the Newton update and the reductions
cudaError_t ysweep(tf_ctx& c, const double* u_k, double dt, double* u_next, double* v_out);
// the iteration's scalars into c.dsc (clears the accumulators)
cudaError_t finalize(tf_ctx& c);
int launches(const tf_ctx& c);  // kernels of one xsweep + ysweep
}  // namespace part

}  // namespace tf

namespace tf {

// The K iterations of a time step with a fixed iteration count, queued on
// the context's stream without waiting for the GPU: U[0] = u^n, U[1..K]
// receive the iterates (each distinct from the one before), W and V (or
// NULL) w_k and v_k.  The kernels and their order are those of
// tf_newton_adi_step with K fixed iterations (the first fused with the
// explicit part), so the bits are too.  With timing enabled it waits after
// every iteration to read the events.
int fixed_iterates(tf_ctx& c, double dt, int K, double* const* U, double* const* W, double* const* V);

// One time step of exactly K Newton iterations at dt (the step of
// tf_newton_adi_step with its fixed-iteration override), every iteration's
// failure flags checked: TF_OK, a step failure (TF_STEP_NONPOSITIVE,
// TF_STEP_ZERO_PIVOT) or a negative error.
int fixed_step(tf_ctx& c, const double* h_old, double* h_new, double dt, int K);

}  // namespace tf

struct tf_ctx {
  tf_params p;
  tf::ModelK mk;
  double kappa;
  const tf::Ops* ops;
  cudaStream_t stream;
  size_t N;
  int grid_x;      // blocks of the x sweep (32 rows each)
  int grid_y;      // blocks of the y sweep (32 columns each)
  int grid_rx, grid_ry;      // 2-D residual grid (32 x 32 tiles)
  int grid_pkx;              // packed FP32-bulk residual: blocks of kRhsStripWarps strip segments
  int strip_n, strip_rows;   // its strips across x and rows per segment
  bool packed_rhs;           // FP32-bulk with the (3, 2) power law: packed residual kernel
  int n_rhs_parts;           // partial results written by the residual kernel in use
  int grid_st_x, grid_st_y;  // 2-D stencil grid (16 x 16 tiles)
  int grid_stats;  // blocks of k_grid_stats
  void* bn;        // explicit part b^n, HP storage
  void* w;         // right side of the x solve, overwritten by its solution w, LP
  void* ulp;       // FP32 copy of the iterate u_k (FP32-bulk only), written by k_rhs
  void* fac_x;     // x-sweep LU factors, LP
  void* fac_y;     // y-sweep LU factors, LP
  // partitioned line solves (FP32-bulk, (3, 2) power law; tf_partition.cuh)
  bool part;       // this context uses them
  int nsx, nsy;    // segments per x line and per y line
  float* recx;     // x records [nsx-1][20][ny]
  float* recy;     // y records [nsy-1][20][nx]
  float* xsx;      // x separators' values [nsx-1][2][ny]
  float* xsy;      // y separators' values [nsy-1][2][nx]
  tf::part::Acc* acc;  // iteration accumulators (cleared by each finalize)
  double* ubuf;    // iterate buffer
  double* ubuf2;   // state buffer of tf_advance
  tf::PartX* px;
  tf::PartY* py;
  int n_px, n_py;
  tf::Scalars* dsc;
  tf::Scalars* hsc;  // pinned
  tf_timing timing;
  cudaEvent_t ev[8];  // 0-4 iteration timing, 5-6 explicit-part timing, 7 work done (ensembles)
  bool rhs_fused;     // the iteration in flight had its residual formed with b^n
  int expl_kernels;   // kernels the last explicit-part launch queued
  void* adj_ws;       // workspace of tf_adjoint_step (grown on demand)
  size_t adj_bytes;
  // graph engine of tf_ensemble_advance (built on first use)
  tf::EnsDev* ens_dev;        // the film's device-resident controller state
  tf::EnsDev* ens_host;       // pinned staging copy of it
  cudaGraphExec_t ens_exec;   // the instantiated graph of a whole run
};
