// Measured arithmetic peaks of the device for roofline denominators (not part of the
// method): the FP64 and FP32 fused multiply-add throughput of a kernel that does nothing
// but independent FMA chains, all SMs busy.
#include "kfbi_internal.cuh"

namespace kfbi {
namespace {

constexpr int kChains = 8;      // independent dependency chains per thread
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_probe_kernel(T* out, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == T(-1.2345)) out[0] = s;   // keeps the chains alive; never true for these inputs
}

template <typename T>
kfbi_status run_probe(int iters, double* tflops, cudaStream_t st) {
  int dev = 0, sms = 0, per_sm = 0;
  KFBI_CUDA_TRY(cudaGetDevice(&dev));
  KFBI_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  KFBI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_probe_kernel<T>,
                                                              kThreads, 0));
  const int blocks = sms * (per_sm < 1 ? 1 : per_sm);
  cudaEvent_t e0, e1;
  KFBI_CUDA_TRY(cudaEventCreate(&e0));
  KFBI_CUDA_TRY(cudaEventCreate(&e1));
  // a = 1 - 2^-20, b = 2^-10: the chains stay finite and bounded
  const T a = T(1.0 - 1.0 / 1048576.0), b = T(1.0 / 1024.0);
  fma_probe_kernel<T><<<blocks, kThreads, 0, st>>>(nullptr, iters / 8, a, b);   // warm-up
  KFBI_CUDA_TRY(cudaGetLastError());
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    KFBI_CUDA_TRY(cudaEventRecord(e0, st));
    fma_probe_kernel<T><<<blocks, kThreads, 0, st>>>(nullptr, iters, a, b);
    KFBI_CUDA_TRY(cudaEventRecord(e1, st));
    KFBI_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    KFBI_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    best = ms < best ? ms : best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return KFBI_OK;
}

}  // namespace
}  // namespace kfbi

extern "C" kfbi_status kfbi_measure_fma_peak(int fp64, double* h_tflops, void* stream) {
  if (!h_tflops) {
    kfbi::set_error("kfbi_measure_fma_peak: null output");
    return KFBI_ERR_ARG;
  }
  const cudaStream_t st = (cudaStream_t)stream;
  return fp64 ? kfbi::run_probe<double>(4096, h_tflops, st)
              : kfbi::run_probe<float>(65536, h_tflops, st);
}
