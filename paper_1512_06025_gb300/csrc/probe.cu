// Measured fused multiply-add rate of the current GPU, the arithmetic roofline denominator of
// the kernels whose bound is the FP64 (or FP32) pipe rather than memory (the roofline study
// of Section 4.4 divides by the peak of the GPU it ran on; here that peak is measured).
//
// Every thread runs kChains independent multiply-add chains (enough independent work to
// keep the pipe busy), the grid is a multiple of the SM count, and the result of every
// chain is stored so that nothing can be optimised away.  Timed with CUDA events around a
// launch sized to run for tens of milliseconds, after a warm-up launch.
#include <algorithm>
#include <string>

#include "bbdg_internal.h"

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) fma_rate_kernel(T* __restrict__ out, int iters, T a, T b) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = T(tid % 7 + c) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = x[c] * a + b;   // contracted to one FMA
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[tid] = s;
}

template <typename T>
int measure(double* tflops, std::string& err) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    err = "cudaGetDevice / attribute query failed";
    return BBDG_ECUDA;
  }
  const int blocks = sms * 8, threads = 256;
  const int64_t nthreads = (int64_t)blocks * threads;
  T* out = nullptr;
  if (cudaMalloc(&out, nthreads * sizeof(T)) != cudaSuccess) {
    err = "cudaMalloc failed";
    return BBDG_ENOMEM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // a, b keep every chain bounded: x -> b / (1 - a) = 1
  const T a = T(0.999999), b = T(1e-6);
  // a short launch to size the timed one (~60 ms), that size once untimed, then once timed
  int iters = 1024;
  float ms = 0.f;
  int rc = BBDG_OK;
  for (int pass = 0; pass < 3; ++pass) {
    cudaEventRecord(e0);
    fma_rate_kernel<T><<<blocks, threads>>>(out, iters, a, b);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      err = "probe kernel failed";
      rc = BBDG_ECUDA;
      break;
    }
    cudaEventElapsedTime(&ms, e0, e1);
    if (pass == 0) iters = (int)std::min<double>(1 << 24, std::max(1024.0, iters * 60.0 / std::max(ms, 0.01f)));
  }
  if (rc == BBDG_OK) {
    const double flop = 2.0 * kChains * (double)iters * (double)nthreads;
    *tflops = flop / (ms * 1e-3) / 1e12;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return rc;
}

}  // namespace

extern "C" {

int bbdg_measure_fma_peak(int precision, double* tflops) {
  if (!tflops || (precision != BBDG_F64 && precision != BBDG_F32)) return BBDG_EINVAL;
  std::string err;
  return precision == BBDG_F64 ? measure<double>(tflops, err) : measure<float>(tflops, err);
}

}  // extern "C"
