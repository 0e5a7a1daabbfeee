// tf_part.cu -- launches of the partitioned line solves (tf_partition.cuh)
// for the FP32-bulk path of a context.
#include "tf_internal.h"
#include "tf_partition.cuh"

namespace tf {
namespace part {

static_assert(kRec == kRecordValues, "record size shared with the workspace allocation");

int nseg_x(int nx) { return seg_count<kLX>(nx); }
int nseg_y(int ny) { return seg_count<kLY>(ny); }
size_t acc_bytes() { return sizeof(Acc); }

cudaError_t prepare() {
  cudaError_t e;
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  const cudaFuncAttribute C = cudaFuncAttributePreferredSharedMemoryCarveout;
  const int maxc = (int)cudaSharedmemCarveoutMaxShared;
  if ((e = cudaFuncSetAttribute(k_part_x1, A, (int)sizeof(X1Smem)))) return e;
  if ((e = cudaFuncSetAttribute(k_part_xy, A, (int)sizeof(XYSmem)))) return e;
  if ((e = cudaFuncSetAttribute(k_part_yc, A, (int)sizeof(YCSmem)))) return e;
  if ((e = cudaFuncSetAttribute(k_part_x1, C, maxc))) return e;
  if ((e = cudaFuncSetAttribute(k_part_xy, C, maxc))) return e;
  return cudaFuncSetAttribute(k_part_yc, C, maxc);
}

static LineK<float> consts(const tf_ctx& c, double dt) {
  StepK k;
  k.theta_dt = c.p.theta * dt;
  k.expl_dt = (1.0 - c.p.theta) * dt;
  return line_consts<float>(c.mk, k);
}

cudaError_t xsweep(tf_ctx& c, double dt) {
  const LineK<float> L = consts(c, dt);
  const float* ul = (const float*)c.ulp;
  float* rw = (float*)c.w;
  const int ny = c.mk.ny, nx = c.mk.nx;
  if (c.nsx > 1) {
    k_part_x1<<<dim3(c.nsx, (ny + kRX - 1) / kRX), kT, sizeof(X1Smem), c.stream>>>(c.mk, L, ul, rw, c.recx,
                                                                                 c.acc);
    k_part_red<<<(ny + 127) / 128, 128, 0, c.stream>>>(c.recx, c.nsx, ny, c.xsx, c.acc);
  }
  k_part_xy<<<dim3(c.nsx, c.nsy), kT, sizeof(XYSmem), c.stream>>>(c.mk, L, ul, rw, c.xsx, c.recy, c.acc);
  if (c.nsy > 1) k_part_red<<<(nx + 127) / 128, 128, 0, c.stream>>>(c.recy, c.nsy, nx, c.xsy, c.acc);
  return cudaGetLastError();
}

cudaError_t ysweep(tf_ctx& c, const double* u_k, double dt, double* u_next, double* v_out) {
  const LineK<float> L = consts(c, dt);
  k_part_yc<<<dim3((c.mk.nx + kCY - 1) / kCY, c.nsy), kT, sizeof(YCSmem), c.stream>>>(
      c.mk, L, u_k, (const float*)c.w, c.xsy, u_next, v_out, c.acc);
  return cudaGetLastError();
}

cudaError_t finalize(tf_ctx& c) {
  k_part_finalize<<<1, 256, 0, c.stream>>>(c.px, c.n_rhs_parts, c.acc, c.dsc);
  return cudaGetLastError();
}

int launches(const tf_ctx& c) { return 2 + (c.nsx > 1 ? 2 : 0) + (c.nsy > 1 ? 1 : 0); }

}  // namespace part
}  // namespace tf
