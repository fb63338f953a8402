// bbdg_step_noalloc: LSERK4 steps whose ping-pong buffer lives in a fixed, file-scope
// device array instead of memory the caller (or the library) allocates.
//
// Why: bbdg_step needs a second state-sized buffer because every stage reads the old
// coefficients of neighbouring elements while it writes the new ones.  Some callers cannot
// provide or allocate that buffer: plug-ins that must not touch the device allocator of
// their host application, and real-time loops that forbid allocation after start-up.
// This entry point takes the buffer from a static __device__ array instead.
//
// The array holds kStepScratchBytes on every GPU that loads the library, until the process
// exits.  All calls share it: two calls that overlap on the GPU (different streams, or
// different host threads) race on it.  Nothing in it needs to start at zero: the first
// stage of every step overwrites the whole buffer before any of it is read.
#include <mutex>

#include "bbdg_internal.h"

namespace {

constexpr size_t kStepScratchBytes = size_t(64) << 20;   // 64 MiB

static __device__ __align__(256) unsigned char g_step_scratch[kStepScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_step_scratch on the current device (looked up once per device; in
// host code the symbol itself is only a host-side stand-in, not a device address).
int scratch_address(void** out, std::string& err) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return BBDG_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    err = "device index out of range for the static step buffer";
    return BBDG_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_step_scratch);
    if (e != cudaSuccess || !p) {
      err = std::string("cudaGetSymbolAddress(static step buffer): ") + cudaGetErrorString(e);
      return BBDG_ECUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return BBDG_OK;
}

}  // namespace

extern "C" {

size_t bbdg_step_noalloc_max_bytes(void) { return kStepScratchBytes; }

int bbdg_step_noalloc(bbdg_ctx* ctx, void* q, void* res, int64_t S, double t0, double dt, int nsteps,
                      void* stream) {
  if (!ctx) return BBDG_EINVAL;
  // the same order of checks as bbdg_step: setup state, empty batch, arguments, zero steps
  if (ctx->N == 0) {
    ctx->err = "bbdg_step_noalloc: bbdg_setup_operators has not been called";
    return BBDG_ESTATE;
  }
  if (S == 0) return BBDG_OK;                  // an empty batch: nothing to do
  if (!q || !res || S < 0 || S > 65535 || nsteps < 0) {
    ctx->err = "bbdg_step_noalloc: bad arguments";
    return BBDG_EINVAL;
  }
  if (nsteps == 0) return BBDG_OK;
  const size_t tsize = ctx->precision == BBDG_F64 ? 8 : 4;
  const size_t bytes = (size_t)S * (size_t)ctx->K * 4 * (size_t)bbdg::np_of(ctx->N) * tsize;
  if (bytes > kStepScratchBytes) {
    ctx->err = "bbdg_step_noalloc: the state (" + std::to_string(bytes) + " bytes) exceeds the static step buffer (" +
               std::to_string(kStepScratchBytes) + " bytes); use bbdg_step with a caller-provided scratch buffer";
    return BBDG_EINVAL;
  }
  void* scratch = nullptr;
  int rc = scratch_address(&scratch, ctx->err);
  if (rc != BBDG_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void* cur = q;
  void* nxt = scratch;
  for (int n = 0; n < nsteps; ++n) {
    for (int s = 0; s < 5; ++s) {
      rc = bbdg_rk_stage(ctx, cur, nxt, res, S, s, t0 + n * dt, dt, stream);
      if (rc != BBDG_OK) return rc;
      void* tmp = cur;
      cur = nxt;
      nxt = tmp;
    }
  }
  if (cur != q) {
    const cudaError_t e = cudaMemcpyAsync(q, cur, bytes, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) {
      ctx->err = std::string("bbdg_step_noalloc: cudaMemcpyAsync: ") + cudaGetErrorString(e);
      return BBDG_ECUDA;
    }
  }
  return BBDG_OK;
}

}  // extern "C"
