// ltmp2_alu_peak: the FP64 / FP32 fused multiply-add rate of the current GPU, measured
// with CUDA events on independent FMA chains.  The paper has no counterpart; the roofline
// fractions of the CUDA-core kernels (the FP64 GEMMs and FFTs, the FP32 FFTs) are quoted
// against this measured rate instead of a figure derived from unit counts.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/ltmp2.h"

namespace {

constexpr int kChains = 8;      // independent FMA chains per thread (hide the FMA latency)
constexpr int kThreads = 256;

// Each thread runs kChains chains x = x * b + c for `iters` steps (b < 1 keeps them finite).
// The result is stored only if it is negative, which never happens for these inputs, so
// nothing is folded away and almost nothing reaches memory.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(int iters, T b, T c, T *out) {
  T x[kChains], br[kChains];
  // FP64: both FMA operands in registers (x * 0 is not folded for floating point, so cr is
  // a run-time value), since operands from the constant bank throttle the FP64 pipe.
  // FP32: one register operand and two kernel parameters; three register operands per
  // FFMA collide in the register banks and halve the measured rate.
  const T cr = c + (T)threadIdx.x * (T)0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) {
    x[k] = (T)(threadIdx.x + k) * (T)1e-3;
    br[k] = b - (T)k * (T)1e-9;
  }
#pragma unroll 4
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      if constexpr (sizeof(T) == 8)
        x[k] = fma(x[k], br[k], cr);
      else
        x[k] = fma(x[k], b, c);
    }
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s < (T)0) out[blockIdx.x * kThreads + threadIdx.x] = s;
}

template <typename T> int measure(int iters, double *tflops) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return LTMP2_ERR_CUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains<T>, kThreads, 0) != cudaSuccess)
    return LTMP2_ERR_CUDA;
  const int blocks = sms * std::max(per_sm, 1);
  T *out = nullptr;   // never written (see the kernel); a valid address all the same
  cudaEvent_t a = nullptr, b = nullptr;
  int rc = LTMP2_OK;
  if (cudaMalloc(&out, sizeof(T) * (size_t)blocks * kThreads) != cudaSuccess) return LTMP2_ERR_OOM;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) rc = LTMP2_ERR_CUDA;
  float best = 1e30f;
  for (int rep = 0; rep < 6 && !rc; ++rep) {   // the first launch is a warm-up (and lets the clock settle)
    cudaEventRecord(a);
    k_fma_chains<T><<<blocks, kThreads>>>(iters, (T)0.9999999, (T)1e-7, out);
    cudaEventRecord(b);
    if (cudaEventSynchronize(b) != cudaSuccess) { rc = LTMP2_ERR_CUDA; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (rep > 0) best = std::min(best, ms);
  }
  if (!rc && cudaGetLastError() != cudaSuccess) rc = LTMP2_ERR_CUDA;
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(out);
  if (rc) return rc;
  const double flops = 2.0 * kChains * (double)iters * blocks * kThreads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return LTMP2_OK;
}

}  // namespace

extern "C" int ltmp2_alu_peak(int precision, double *tflops) {
  if (!tflops) return LTMP2_ERR_INVALID_ARG;
  // about 0.1 s per launch at the nominal rates
  if (precision == LTMP2_FP64) return measure<double>(1 << 15, tflops);
  if (precision == LTMP2_FP32) return measure<float>(1 << 20, tflops);
  return LTMP2_ERR_INVALID_ARG;
}
