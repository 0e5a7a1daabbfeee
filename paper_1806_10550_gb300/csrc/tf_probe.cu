// tf_probe.cu -- arithmetic throughput probes for the roofline denominators
// that the HBM copy and bf16 GEMM measurements do not cover: FP64 and FP32
// fused multiply-add issue rates of the GPU the library runs on.
#include <cuda_runtime.h>

#include "../../include/tf.h"

namespace {

constexpr int kChains = 8;     // independent FMA chains per thread
constexpr int kThreads = 256;

// Every thread runs kChains independent chains a <- a m + c (no
// dependence between chains, so the pipe, not the latency, bounds it);
// the sum is stored so that the chains are not removed.
template <class T>
__global__ void __launch_bounds__(kThreads) k_fma_probe(int iters, T m, T c, T* out) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = T(1) + T(k) * T(1e-3) + T(threadIdx.x) * T(1e-6);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], m, c);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[blockIdx.x * kThreads + threadIdx.x] = s;
}

template <class T>
int run(void* stream, int blocks, int iters, double* tflops) {
  T* out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = TF_OK;
  if (cudaMalloc((void**)&out, (size_t)blocks * kThreads * sizeof(T)) != cudaSuccess) return TF_ERR_NOMEM;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = TF_ERR_CUDA;
  const T m = T(1) - T(1e-7), c = T(1e-7);
  if (!rc) k_fma_probe<T><<<blocks, kThreads, 0, s>>>(iters / 8, m, c, out);  // warm-up
  if (!rc && cudaEventRecord(e0, s) != cudaSuccess) rc = TF_ERR_CUDA;
  if (!rc) k_fma_probe<T><<<blocks, kThreads, 0, s>>>(iters, m, c, out);
  if (!rc && (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
              cudaEventSynchronize(e1) != cudaSuccess))
    rc = TF_ERR_CUDA;
  float ms = 0.0f;
  if (!rc && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = TF_ERR_CUDA;
  if (!rc) *tflops = 2.0 * kChains * (double)iters * blocks * kThreads / (ms * 1e-3) * 1e-12;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return rc;
}

}  // namespace

extern "C" int tf_probe_fma(int precision, void* stream, double* tflops) {
  if (!tflops || (precision != TF_FP64 && precision != TF_FP32_BULK)) return TF_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess)
    return TF_ERR_CUDA;
  // 8 blocks of 256 threads per SM (every warp slot the SM offers them),
  // about 20 ms of work on this GPU in either precision
  return precision == TF_FP64 ? run<double>(stream, 8 * sms, 1 << 13, tflops)
                              : run<float>(stream, 8 * sms, 1 << 18, tflops);
}
