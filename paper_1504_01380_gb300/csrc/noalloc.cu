// swept_advance_noalloc: the swept advance with no device allocation at all.
//
// Some callers cannot call cudaMalloc: a host that hands a plugin a fixed
// device-memory budget and forbids allocations after start-up, or code that
// must not pay the implicit device synchronisation an allocation can cause.
// For them this entry point runs the same stage kernels as swept_advance but
// keeps the leading-edge buffers in a fixed array in device global memory
// that the library declares at file scope.  The array is part of the loaded
// module, so every GPU that loads the library holds it (kNoallocScratchBytes)
// until the process exits.
//
// Limits and sharing: N <= SWEPT_NOALLOC_MAX_N (the edges of one stage take
// 16 N bytes and there are two stages in flight, 32 N bytes in all).  Every
// call uses the same array, so calls that overlap on the GPU (other streams,
// other host threads) race and corrupt each other's results; order them.
// Nothing in the array has to start at zero: each stage writes the edges
// before the next stage reads them, so a call never reads what an earlier
// call left behind.
//
// Set-up: host code cannot use the array's name as a device address (it is a
// host-side stand-in).  The first call on a device looks the address up with
// cudaGetSymbolAddress with that device current and caches it per device;
// make that first call before any stream capture.  The cache lives as long
// as the process: after cudaDeviceReset (or anything else that destroys the
// device's primary context) the module is loaded again and the array may
// move, so the library must be unloaded and loaded again before the next
// call on that device.
#include <mutex>

#include "swept.h"
#include "swept_internal.h"

namespace {

constexpr int64_t kMaxN = SWEPT_NOALLOC_MAX_N;
constexpr size_t kNoallocScratchBytes = (size_t)32 * kMaxN;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

int status_of(cudaError_t e) {
  return e == cudaSuccess ? SWEPT_OK : SWEPT_ECUDA;
}

}  // namespace

extern "C" int swept_advance_noalloc(int64_t N, int stencil_id, const double* params, int nparams,
                                     int dtype, int B, void* u, int64_t nsteps, void* stream) {
  using swept::StageArgs;
  if (!params || !u || nsteps < 0 || ((uintptr_t)u & 15u)) return SWEPT_EINVAL;
  if (stencil_id != SWEPT_HEAT && stencil_id != SWEPT_KS) return SWEPT_EINVAL;
  if (dtype != SWEPT_F64 && dtype != SWEPT_F32C) return SWEPT_EINVAL;
  const int R = stencil_id == SWEPT_HEAT ? 1 : 2;
  if (N <= 0 || B <= 0 || B % 32) return SWEPT_EINVAL;
  const int K = B / 32;
  if (K != 1 && K != 2 && K != 4 && K != 8 && K != 16 && K != 32) return SWEPT_ENOTSUP;
  if (K % R || N % B) return SWEPT_EINVAL;
  if (N > kMaxN) return SWEPT_ETOOBIG;
  // u and the stream must be on the current device, whose copy of the array
  // the kernels are given
  if (!swept::call_on_device(-1, (cudaStream_t)stream, {u})) return SWEPT_EINVAL;

  // Constants, as swept_plan computes them: heat r; KS a = -(dt/(4 dx)),
  // b = -(dt/dx^2), e = -(dt/(dx^2 dx^2)), FP32 copies rounded to nearest.
  swept::Consts c = {};
  if (stencil_id == SWEPT_HEAT) {
    if (nparams < 1) return SWEPT_EINVAL;
    c.r = params[0];
    c.r32 = (float)c.r;
  } else {
    if (nparams < 2 || !(params[1] > 0.0)) return SWEPT_EINVAL;
    const double dt = params[0], dx = params[1], dx2 = dx * dx;
    c.a = -(dt / (4.0 * dx));
    c.b = -(dt / dx2);
    c.e = -(dt / (dx2 * dx2));
    c.a32 = (float)c.a;
    c.b32 = (float)c.b;
    c.e32 = (float)c.e;
  }
  if (nsteps == 0) return SWEPT_OK;

  void* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) return status_of(e);
  const int nwin = (int)(N / B);
  const size_t half = (size_t)nwin * 2 * B * 8;
  unsigned char* buf[2] = {static_cast<unsigned char*>(scratch),
                           static_cast<unsigned char*>(scratch) + half};

  cudaStream_t s = (cudaStream_t)stream;
  StageArgs a{};
  a.u = u;
  a.N = N;
  a.nwin = nwin;
  a.c = c;
  auto stage = [&](int64_t k, int hv, int ht) -> cudaError_t {
    a.offset = (k & 1) ? B / 2 : 0;
    a.hv = hv;
    a.ht = ht;
    a.ein = buf[(k + 1) & 1];
    a.eout = buf[k & 1];
    if (stencil_id == SWEPT_HEAT)
      return dtype == SWEPT_F64 ? swept::launch_stage_heat_f64(K, a, s)
                                : swept::launch_stage_heat_f32c(K, a, s);
    return dtype == SWEPT_F64 ? swept::launch_stage_ks_f64(K, a, s)
                              : swept::launch_stage_ks_f32c(K, a, s);
  };
  const int64_t H = B / (2 * R);
  const int64_t q = nsteps / H;
  const int rem = (int)(nsteps % H);
  if (q == 0) {
    e = stage(0, 0, rem);
    if (e == cudaSuccess) e = stage(1, rem, 0);
  } else {
    e = stage(0, 0, (int)H);
    for (int64_t k = 1; k < q && e == cudaSuccess; ++k) e = stage(k, (int)H, (int)H);
    if (e == cudaSuccess) e = stage(q, (int)H, rem);
    if (e == cudaSuccess && rem > 0) e = stage(q + 1, rem, 0);
  }
  return status_of(e);
}
