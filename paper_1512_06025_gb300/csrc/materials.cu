// The material-dependent words of the element records, formed on the device from the
// material arrays kappa, rho ([mS][K], FP64): kappa and 1/rho of the element (the two factors
// of the acoustic system of Section 2) and, per face, the upwind flux weights
// tau_p = 1/{rho c}, tau_u = {rho c} with {rho c} = (z_k + z_k')/2 and z = rho c =
// sqrt(kappa rho) (the neighbour's own z on the boundary), scaled by |grad lambda_m| as the
// record layouts in bbdg_internal.h state; with the central flux both weights are 0.
// Also d tau / d kappa_k per face for the adjoint's gradient (medium 0 only): with
// d{rho c}/d kappa_k = z_k / (4 kappa_k) (z_k / (2 kappa_k) on the boundary, where both sides
// are the element's own), d tau_p = -tau_p^2 d{rho c} and d tau_u = d{rho c}.
//
// Every value is formed in FP64 with the same operations, in the same order, as the
// element's geometric factors were (|grad lambda_m| comes in precomputed in FP64), and
// rounded once to the state type: the records do not depend on where the materials came
// from (host arrays at set-up or device arrays later).
#include <cmath>

#include "bbdg_internal.h"

namespace bbdg {
namespace {

template <typename T>
__device__ __forceinline__ void put(T* rec, int w, double v) {
  rec[w] = (T)v;
}

template <typename T>
__global__ void __launch_bounds__(256) material_records_kernel(MaterialArgs<T> a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.mS * a.K) return;
  const int64_t s = i / a.K, k = i - s * a.K;
  const double* kap = a.kappa + s * a.K;
  const double* rho = a.rho + s * a.K;
  const double kk = kap[k], rk = rho[k];
  const double zk = sqrt(kk * rk);
  T* g = a.geo ? a.geo + i * kGeoStride : nullptr;
  T* x = a.gext ? a.gext + i * kPipeGeo : nullptr;
  T* d = (a.adg && s == 0) ? a.adg + k * 8 : nullptr;
  const double rinv = 1.0 / rk;
  if (g) {
    put(g, 9, kk);
    put(g, 10, rinv);
  }
  if (x) {
    put(x, 20, kk);
    put(x, 21, rinv);
  }
  for (int m = 0; m < 4; ++m) {
    const int32_t nb = a.nbr[k * 4 + m];
    const double nrm = a.fnrm[k * 4 + m];
    const double zn = nb >= 0 ? sqrt(kap[nb] * rho[nb]) : zk;
    const double avg = 0.5 * (zk + zn);
    const double tau_p = a.central ? 0.0 : 1.0 / avg;
    const double tau_u = a.central ? 0.0 : avg;
    const double tp = nrm * tau_p, tu = tau_u / nrm;
    if (g) {
      put(g, 11 + m, tp);
      put(g, 15 + m, tu);
    }
    if (x) {
      put(x, 4 * m + 3, tp);
      put(x, 16 + m, tu);
    }
    if (d) {
      if (a.central) {
        put(d, m, 0.0);
        put(d, 4 + m, 0.0);
      } else {
        const double davg = nb >= 0 ? zk / (4.0 * kk) : zk / (2.0 * kk);
        put(d, m, -davg / (avg * avg));
        put(d, 4 + m, davg);
      }
    }
  }
}

// counts the entries of kappa and rho that are not finite and > 0
__global__ void __launch_bounds__(256) material_check_kernel(const double* kappa, const double* rho, int64_t n,
                                                             int* bad) {
  int cnt = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double kv = kappa[i], rv = rho[i];
    cnt += !(kv > 0.0 && kv <= 1.7976931348623157e308) + !(rv > 0.0 && rv <= 1.7976931348623157e308);
  }
  if (cnt) atomicAdd(bad, cnt);
}

}  // namespace

template <typename T>
int launch_material_records(const MaterialArgs<T>& a, cudaStream_t st) {
  const int64_t n = a.mS * a.K;
  if (n <= 0) return BBDG_OK;
  const int64_t blocks = (n + 255) / 256;
  if (blocks > INT32_MAX) return BBDG_EINVAL;
  material_records_kernel<T><<<(unsigned)blocks, 256, 0, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? BBDG_OK : BBDG_ECUDA;
}

template int launch_material_records<double>(const MaterialArgs<double>&, cudaStream_t);
template int launch_material_records<float>(const MaterialArgs<float>&, cudaStream_t);

int launch_material_check(const double* kappa, const double* rho, int64_t n, int* bad, cudaStream_t st) {
  if (n <= 0) return BBDG_OK;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return BBDG_ECUDA;
  const int64_t want = (n + 255) / 256;
  const int blocks = (int)(want < 4 * (int64_t)sms ? want : 4 * (int64_t)sms);
  material_check_kernel<<<blocks, 256, 0, st>>>(kappa, rho, n, bad);
  return cudaGetLastError() == cudaSuccess ? BBDG_OK : BBDG_ECUDA;
}

}  // namespace bbdg
