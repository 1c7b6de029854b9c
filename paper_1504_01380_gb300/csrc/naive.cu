// Naive per-step stepper: the "straight" decomposition the swept rule is
// measured against (Section 6 compares the two on the same discretisation).
// One launch per sub-timestep; every launch reads the whole field once and
// writes it once, so the kernel is bound by HBM bandwidth.
//
// Each thread owns V = 4 consecutive points (16-byte vector loads of FP32
// hi/lo, two 16-byte loads of FP64).  The r neighbours beyond a thread's
// points come from the adjacent lanes by shuffle; lanes at a warp's ends (or
// next to the end of the array) read them from global memory, which the
// neighbouring warp's loads have usually brought into L2 already.
#include "swept_internal.h"

namespace swept {

namespace {

constexpr int kV = 4;
constexpr int kNaiveThreads = 256;

template <class DT> __device__ __forceinline__ typename DT::C hi_at(const void* u, int64_t g);
template <> __device__ __forceinline__ double hi_at<F64>(const void* u, int64_t g) {
  return static_cast<const double*>(u)[g];
}
template <> __device__ __forceinline__ float hi_at<F32C>(const void* u, int64_t g) {
  return static_cast<const float*>(u)[g];
}

template <int ST, class DT>
__global__ void __launch_bounds__(kNaiveThreads)
naive_step_kernel(const void* __restrict__ in, void* __restrict__ out, int64_t N, const Consts c) {
  constexpr int R = Radius<ST>::value;
  using Cc = typename DT::C;
  const int lane = threadIdx.x & 31;
  const int64_t i0 = ((int64_t)blockIdx.x * kNaiveThreads + threadIdx.x) * kV;
  const bool valid = i0 < N;
  Tile<DT, kV> t;
  t.zero();
  if (valid) load_points<kV>(t, in, N, i0);
  Cc x[kV + 2 * R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    x[i] = __shfl_sync(kFull, t.hi(kV - R + i), (lane + 31) & 31);
    x[R + kV + i] = __shfl_sync(kFull, t.hi(i), (lane + 1) & 31);
  }
#pragma unroll
  for (int k = 0; k < kV; ++k) x[R + k] = t.hi(k);
  if (!valid) return;
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < R; ++i) {
      int64_t g = i0 - R + i;
      if (g < 0) g += N;
      x[i] = hi_at<DT>(in, g);
    }
  }
  if (lane == 31 || i0 + kV >= N) {
#pragma unroll
    for (int i = 0; i < R; ++i) {
      int64_t g = i0 + kV + i;
      if (g >= N) g -= N;
      x[R + kV + i] = hi_at<DT>(in, g);
    }
  }
  Core<ST, DT, kV>::apply(t, x, c);
  store_points<kV>(t, out, N, i0);
}

template <int ST, class DT>
cudaError_t launch(const void* in, void* out, int64_t N, const Consts& c, cudaStream_t s) {
  const int64_t threads = N / kV;
  const int64_t grid = (threads + kNaiveThreads - 1) / kNaiveThreads;
  naive_step_kernel<ST, DT><<<(unsigned)grid, kNaiveThreads, 0, s>>>(in, out, N, c);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_naive_step(int stencil, int dtype, const void* in, void* out, int64_t N,
                              const Consts& c, cudaStream_t s) {
  if (N % kV) return cudaErrorInvalidValue;
  if (stencil == kHeat) return dtype == 0 ? launch<kHeat, F64>(in, out, N, c, s)
                                          : launch<kHeat, F32C>(in, out, N, c, s);
  return dtype == 0 ? launch<kKS, F64>(in, out, N, c, s) : launch<kKS, F32C>(in, out, N, c, s);
}

}  // namespace swept
