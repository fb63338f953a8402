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
