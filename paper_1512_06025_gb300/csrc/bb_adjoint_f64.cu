// FP64 instantiations of the adjoint stage kernels (N = 1..10).
#include "bb_adjoint.cuh"

namespace bbdg {
int launch_adjoint_f64(int N, const AdjointArgs<double>& a, cudaStream_t st) {
  switch (N) {
    case 1: return launch_adjoint_n<double, 1>(a, st);
    case 2: return launch_adjoint_n<double, 2>(a, st);
    case 3: return launch_adjoint_n<double, 3>(a, st);
    case 4: return launch_adjoint_n<double, 4>(a, st);
    case 5: return launch_adjoint_n<double, 5>(a, st);
    case 6: return launch_adjoint_n<double, 6>(a, st);
    case 7: return launch_adjoint_n<double, 7>(a, st);
    case 8: return launch_adjoint_n<double, 8>(a, st);
    case 9: return launch_adjoint_n<double, 9>(a, st);
    case 10: return launch_adjoint_n<double, 10>(a, st);
    default: return BBDG_EUNSUPPORTED;
  }
}
int launch_receiver_adjoint_f64(int N, double* lq, int64_t K, int nrec, const int32_t* elem, const double* basis,
                                const double* resid, cudaStream_t st) {
  if (nrec <= 0) return BBDG_OK;
  const int Np = np_of(N);
  const int64_t n = (int64_t)nrec * Np;
  receiver_adjoint_kernel<double><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(lq, K, Np, nrec, elem, basis, resid);
  return cudaGetLastError() == cudaSuccess ? BBDG_OK : BBDG_ECUDA;
}
}  // namespace bbdg

// ---- receiver misfit: r = p - d and J = 1/2 sum r^2 (the objective of the gradient), in
// FP64 with Neumaier's compensated summation in a fixed order (one CTA: every thread sums
// a strided share, thread 0 then adds the 256 partial sums and their compensations in
// thread order), so J is reproducible bit for bit.
namespace {

__device__ __forceinline__ void neumaier_add(double& s, double& c, double y) {
  const double t = s + y;
  c += fabs(s) >= fabs(y) ? (s - t) + y : (y - t) + s;
  s = t;
}

__global__ void __launch_bounds__(256) misfit_kernel(const double* __restrict__ tr, const double* __restrict__ d,
                                                     int64_t n, double* __restrict__ r, double* __restrict__ J) {
  __shared__ double ps[256], pc[256];
  double s = 0.0, c = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double x = tr[i] - d[i];
    r[i] = x;
    neumaier_add(s, c, 0.5 * x * x);
  }
  ps[threadIdx.x] = s;
  pc[threadIdx.x] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    double S = 0.0, C = 0.0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      neumaier_add(S, C, ps[t]);
      C += pc[t];
    }
    J[0] = S + C;
  }
}

}  // namespace

extern "C" int bbdg_misfit(bbdg_ctx* ctx, const void* traces, const void* data, int64_t n, void* resid, void* J,
                           void* stream) {
  if (!ctx) return BBDG_EINVAL;
  if (n < 0 || (n > 0 && (!traces || !data || !resid)) || !J) {
    ctx->err = "bbdg_misfit: bad arguments";
    return BBDG_EINVAL;
  }
  if (cudaSetDevice(ctx->device) != cudaSuccess) {
    ctx->err = "cudaSetDevice failed";
    return BBDG_ECUDA;
  }
  misfit_kernel<<<1, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<const double*>(traces), static_cast<const double*>(data), n, static_cast<double*>(resid),
      static_cast<double*>(J));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ctx->err = std::string("misfit kernel launch failed: ") + cudaGetErrorString(e);
    return BBDG_ECUDA;
  }
  return BBDG_OK;
}
