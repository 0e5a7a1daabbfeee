// tf_noalloc.cu -- residual evaluation that allocates nothing.
//
// Some callers cannot call cudaMalloc: code that runs inside a host
// framework which owns every device allocation and forbids others (fixed
// memory budgets, custom pools), real-time or latency-bounded loops where an
// allocation's unpredictable cost or failure is not acceptable, and plugins
// that are handed device buffers but no right to create a solver context.
// tf_residual_noalloc serves them: it evaluates the same Newton residual as
// tf_residual, with the caller passing the parameters, the stream, the
// inputs and the outputs, and with its scratch (the explicit part b^n and
// the per-block partial results) in one fixed device array defined in this
// file.  It never calls cudaMalloc, cudaFree or an allocating library
// routine.
//
// The fixed array (TF_NOALLOC_MAX_CELLS cells of 8 bytes plus the partial
// results, about 16.3 MiB) exists on every GPU that loads the library and is
// held until the process exits.  In host code the array's name is only a
// host-side stand-in, so its device address is looked up once per device
// with cudaGetSymbolAddress, with that device current, on the first call on
// that device; that first call should therefore come before any stream
// capture.  All calls on a device share the array and it keeps the last
// call's contents; every element a call reads is written earlier by the same
// call, so nothing needs clearing, but calls that overlap on the GPU (two
// streams, or two host threads) race on the array and must be serialised by
// the caller.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "tf_internal.h"

namespace {

constexpr size_t kMaxCells = TF_NOALLOC_MAX_CELLS;
// 16 x 16 tiles of a grid with nx, ny <= 65536 and nx*ny <= kMaxCells:
// ceil(nx/16) ceil(ny/16) <= kMaxCells/256 + (nx + ny)/16 + 1.
constexpr size_t kMaxParts = kMaxCells / 256 + 2 * 65536 / 16 + 1;
constexpr size_t kBnBytes = kMaxCells * 8;
constexpr size_t kPartOff = kBnBytes;
constexpr size_t kScalOff = kPartOff + ((kMaxParts * sizeof(tf::PartX) + 255) / 256) * 256;
constexpr size_t kStatOff = kScalOff + 256;
constexpr int kStatBlocks = 64;
constexpr size_t kScratchBytes = kStatOff + kStatBlocks * sizeof(tf::PartY);

static __device__ __align__(256) unsigned char tf_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_ptr[kMaxDevices];

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
cudaError_t scratch_ptr(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, tf_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_ptr[dev] = p;
  }
  *out = (unsigned char*)g_ptr[dev];
  return cudaSuccess;
}

template <class Mode>
cudaError_t run(const tf::ModelK& mk, double theta, cudaStream_t s, const double* h_k,
                const double* h_old, double dt, double* G, unsigned char* scratch) {
  typedef typename Mode::HP HP;
  tf::StepK K;
  K.theta_dt = theta * dt;
  K.expl_dt = (1.0 - theta) * dt;
  const size_t smem = sizeof(tf::StencilSmem<HP, 16, 16>);
  dim3 grid((mk.nx + 15) / 16, (mk.ny + 15) / 16), block(16, 16);
  HP* bn = (HP*)scratch;
  tf::PartX* px = (tf::PartX*)(scratch + kPartOff);
  tf::k_stencil<Mode, 0><<<grid, block, smem, s>>>(mk, K, h_old, bn, nullptr, nullptr);
  tf::k_stencil<Mode, 1><<<grid, block, smem, s>>>(mk, K, h_k, bn, G, px);
  return cudaGetLastError();
}

}  // namespace

extern "C" int tf_residual_noalloc(const tf_params* p, void* stream, const double* h_k,
                                   const double* h_old, double dt, double* G, tf_norms* out) {
  if (!p || !h_k || !h_old || !G || !isfinite(dt)) return TF_ERR_ARG;
  if (p->nx < 1 || p->ny < 1 || p->nx > 65536 || p->ny > 65536) return TF_ERR_ARG;
  if ((size_t)p->nx * (size_t)p->ny > kMaxCells) return TF_ERR_ARG;
  if (!(p->ds > 0.0) || !isfinite(p->ds) || !(p->theta >= 0.0 && p->theta <= 1.0)) return TF_ERR_ARG;
  if (p->model != TF_MODEL_POWERLAW && p->model != TF_MODEL_LINEAR) return TF_ERR_ARG;
  if (p->precision != TF_FP64 && p->precision != TF_FP32_BULK) return TF_ERR_ARG;
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
  tf::ModelK mk;
  memset(&mk, 0, sizeof(mk));
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
  unsigned char* scratch = nullptr;
  if (scratch_ptr(&scratch) != cudaSuccess) return TF_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = p->precision == TF_FP64
                      ? run<tf::ModeFP64>(mk, p->theta, s, h_k, h_old, dt, G, scratch)
                      : run<tf::ModeF32B>(mk, p->theta, s, h_k, h_old, dt, G, scratch);
  if (e != cudaSuccess) return TF_ERR_CUDA;
  if (out) {
    const int nparts = ((p->nx + 15) / 16) * ((p->ny + 15) / 16);
    tf::PartY* py = (tf::PartY*)(scratch + kStatOff);
    tf::Scalars* sc = (tf::Scalars*)(scratch + kScalOff);
    tf::k_grid_stats<<<kStatBlocks, 256, 0, s>>>(h_k, (size_t)p->nx * p->ny, py);
    tf::k_finalize<<<1, 256, 0, s>>>((const tf::PartX*)(scratch + kPartOff), nparts, py,
                                     kStatBlocks, sc);
    if (cudaGetLastError() != cudaSuccess) return TF_ERR_CUDA;
    tf::Scalars h;
    if (cudaMemcpyAsync(&h, sc, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return TF_ERR_CUDA;
    out->gnorm = h.gnorm;
    out->mass = tf::mass_value(h.mass);
    out->hmin = h.hmin;
  }
  return TF_OK;
}
