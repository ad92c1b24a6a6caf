// hom_peak.cu -- measured arithmetic peaks of the current GPU: the sustained
// rate of independent fused multiply-adds in the FP32 and FP64 pipes.  These
// are the denominators of the kinetic passes' ALU roofline (the passes are
// bound by FP32 arithmetic and instruction issue, not by HBM).  A measurement
// utility; not a step of the method.
#include <cuda_runtime.h>

#include "../../include/hom.h"

namespace {

constexpr int kChains = 8;     // independent FMA chains per thread (hides the pipe latency)
constexpr int kThreads = 256;

// Each thread runs kChains independent chains acc = acc * a + b.  With
// 0 < a < 1 the values stay near b / (1 - a), never overflow or go subnormal.
// The sink is written only when the sum equals a value it never reaches, so
// the loop is kept and nothing is stored in practice.
template <typename R>
__global__ void __launch_bounds__(kThreads) fma_loop(R a, R b, int iters, R* sink) {
  R acc[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) acc[i] = (R)(threadIdx.x + i) * (R)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc[i] = fma(acc[i], a, b);
  }
  R s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += acc[i];
  if (s == (R)-12345.678) sink[0] = s;
}

template <typename R>
hom_status time_fma(R* sink, cudaStream_t st, int iters, double* flops_per_s) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HOM_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return HOM_ERR_CUDA;
  const unsigned blocks = (unsigned)sms * 8;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess) return HOM_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return HOM_ERR_CUDA;
  }
  hom_status s = HOM_OK;
  double best = 0.0;
  for (int rep = 0; rep < 4 && s == HOM_OK; ++rep) {   // the first run warms up
    cudaEventRecord(e0, st);
    fma_loop<R><<<blocks, kThreads, 0, st>>>((R)0.999999, (R)1e-6, iters, sink);
    cudaEventRecord(e1, st);
    float ms = 0.f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f)) {
      s = HOM_ERR_CUDA;
      break;
    }
    const double flops = 2.0 * blocks * kThreads * kChains * (double)iters;
    if (rep > 0 && flops / (ms * 1e-3) > best) best = flops / (ms * 1e-3);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s == HOM_OK) *flops_per_s = best;
  return s;
}

}  // namespace

extern "C" hom_status hom_alu_peak(int32_t kind, void* d_sink, void* cuda_stream, double* flops_per_s) {
  if (!d_sink || !flops_per_s || (kind != 0 && kind != 1)) return HOM_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // about 10 ms per run at the nominal rates
  if (kind == 0) return time_fma<float>(static_cast<float*>(d_sink), st, 1 << 16, flops_per_s);
  return time_fma<double>(static_cast<double*>(d_sink), st, 1 << 10, flops_per_s);
}
