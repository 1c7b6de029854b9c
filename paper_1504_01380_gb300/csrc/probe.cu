// Measured arithmetic peaks of this GPU.
//
// The swept kernels are bound by an arithmetic pipe (FP32 for the compensated
// state, FP64 for the reference precision), not by memory, so their roofline
// denominator is the rate at which the GPU retires independent FP32 or FP64
// operations.  Section 4's model takes the node's speed as a given constant;
// here it is measured: every thread of a grid that fills every SM runs kChains
// independent dependency chains of adds (x <- x + b) or fused multiply-adds
// (x <- x*a + b), enough independent work per scheduler to hide the pipe
// latency, so the launch time is set by the pipe's throughput alone.  One add
// or one fma counts as one operation.  The sum of the chains is stored only
// when it equals a value it never reaches (the store keeps the work alive, and
// nothing is written), into a small array inside the module: the probe
// allocates nothing.
#include "swept.h"
#include "swept_device.cuh"
#include "swept_internal.h"

namespace swept {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;
constexpr int kUnroll = 8;

__device__ double g_probe_sink[kProbeThreads];

template <class T> struct ProbeOps;
template <> struct ProbeOps<float> {
  static __device__ __forceinline__ float add(float x, float y) { return __fadd_rn(x, y); }
  static __device__ __forceinline__ float fma(float x, float y, float z) { return __fmaf_rn(x, y, z); }
};
template <> struct ProbeOps<double> {
  static __device__ __forceinline__ double add(double x, double y) { return __dadd_rn(x, y); }
  static __device__ __forceinline__ double fma(double x, double y, double z) { return __fma_rn(x, y, z); }
};

// a = 1 - 2^-20 and b = 2^-24 keep the fma chains near b / (1 - a) = 1/16
// (no overflow, no subnormals); the add chains grow by b per step and stay
// far from overflow for any iteration count a launch can run.
template <class T, bool FMA>
__global__ void __launch_bounds__(kProbeThreads) alu_probe_kernel(int64_t iters, T a, T b, T never) {
  using O = ProbeOps<T>;
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x & 7) * b + T(c) * b;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = FMA ? O::fma(x[c], a, b) : O::add(x[c], b);
    }
  }
  T s = x[0];
#pragma unroll
  for (int c = 1; c < kChains; ++c) s = O::add(s, x[c]);
  if (s == never) g_probe_sink[threadIdx.x] = (double)s;
}

template <class T, bool FMA>
cudaError_t launch_probe(int64_t iters, double* ops, cudaStream_t s) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, alu_probe_kernel<T, FMA>, kProbeThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int grid = sms * per_sm;          // every SM, at full residency
  *ops = (double)grid * kProbeThreads * (double)iters * kUnroll * kChains;
  const T a = T(1) - T(1.0 / 1048576.0), b = T(1.0 / 16777216.0);
  alu_probe_kernel<T, FMA><<<grid, kProbeThreads, 0, s>>>(iters, a, b, T(-1));
  return cudaGetLastError();
}

// The Euler flux's straight-line binary32 division and square root beside
// CUDA's correctly rounded ones, element by element (see swept_device.cuh).
__global__ void div_sqrt_check_kernel(const float* __restrict__ a, const float* __restrict__ b, int64_t n,
                                      float* __restrict__ out, int* __restrict__ ok) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float x = a[i], y = b[i];
    bool okd = true, oks = true;
    out[i] = div_tested(x, rcp_tested(y), okd);
    out[n + i] = __fdiv_rn(x, y);
    out[2 * n + i] = sqrt_tested(x, oks);
    out[3 * n + i] = __fsqrt_rn(x);
    ok[i] = okd ? 1 : 0;
    ok[n + i] = oks ? 1 : 0;
  }
}

}  // namespace
}  // namespace swept

extern "C" int swept_probe_alu(int kind, int64_t iters, double* ops, void* stream) {
  if (!ops || iters <= 0 || iters > ((int64_t)1 << 40)) return SWEPT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (!swept::call_on_device(-1, s, {})) return SWEPT_EINVAL;
  cudaError_t e;
  switch (kind) {
    case SWEPT_PROBE_F32_ADD: e = swept::launch_probe<float, false>(iters, ops, s); break;
    case SWEPT_PROBE_F32_FMA: e = swept::launch_probe<float, true>(iters, ops, s); break;
    case SWEPT_PROBE_F64_ADD: e = swept::launch_probe<double, false>(iters, ops, s); break;
    case SWEPT_PROBE_F64_FMA: e = swept::launch_probe<double, true>(iters, ops, s); break;
    default: return SWEPT_EINVAL;
  }
  if (e == cudaSuccess) return SWEPT_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? SWEPT_ENOMEM : SWEPT_ECUDA;
}

extern "C" int swept_check_div_sqrt(const float* a, const float* b, int64_t n, float* out, int* ok, void* stream) {
  if (n < 0 || (n > 0 && (!a || !b || !out || !ok))) return SWEPT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (!swept::call_on_device(-1, s, {a, b, out, ok})) return SWEPT_EINVAL;
  if (n == 0) return SWEPT_OK;
  const int64_t blocks = (n + 255) / 256;
  swept::div_sqrt_check_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(a, b, n, out, ok);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SWEPT_OK : SWEPT_ECUDA;
}
