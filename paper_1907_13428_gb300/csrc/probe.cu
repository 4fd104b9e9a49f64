// Arithmetic peak probe: independent fused multiply-add chains in float or
// double, timed with CUDA events. Used as the denominator of the ALU roofline
// of the double-precision transforms (GB300 runs double at 1/58 of the float
// rate, so those kernels are bound by arithmetic, not by HBM).
#include <algorithm>

#include "internal.h"

namespace fde {

template <typename T>
__global__ void k_fma_chains(T* out, int iters, T a, T b) {
  T x0 = (T)threadIdx.x * (T)1e-3, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  const T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == (T)-12345.678) out[blockIdx.x] = s;  // keeps the chains live; never true
}

}  // namespace fde

extern "C" int fde_alu_peak_probe(int precision, double* tflops, void* stream) {
  if (!tflops || (precision != FDE_FP64 && precision != FDE_FP32)) return FDE_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FDE_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return FDE_ECUDA;
  const int blocks = sms * 8, threads = 256;
  const int iters = precision == FDE_FP64 ? (1 << 13) : (1 << 16);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return FDE_ECUDA;
  double best = 0.0;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, st);
    if (precision == FDE_FP64)
      fde::k_fma_chains<double><<<blocks, threads, 0, st>>>(nullptr, iters, 0.999999, 1e-7);
    else
      fde::k_fma_chains<float><<<blocks, threads, 0, st>>>(nullptr, iters, 0.9999f, 1e-7f);
    fde::note_launches(1);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * 8.0 * iters * (double)blocks * threads;
    if (ms > 0) best = std::max(best, flops / (ms * 1e-3) / 1e12);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaGetLastError() != cudaSuccess) return FDE_ECUDA;
  *tflops = best;
  return FDE_OK;
}
