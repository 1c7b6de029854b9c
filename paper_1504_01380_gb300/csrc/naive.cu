// Naive per-step steppers: the "straight" decomposition the swept rule is
// measured against (Section 6 compares the two on the same discretisation).
// One launch per sub-timestep; every launch reads the whole field once and
// writes it once, so the kernel is bound by HBM bandwidth.
//
// Each thread owns V = 4 consecutive points (16-byte vector loads of FP32
// hi/lo, two 16-byte loads of FP64, when aligned).  The r neighbours beyond a
// thread's points come from the adjacent lanes by shuffle; lanes at a warp's
// ends (or within r of the end of the array) read them from global memory,
// which the neighbouring warp's loads have usually brought into L2 already.
// When N is not a multiple of V the last thread owns the N mod V points left,
// loaded and stored one by one, and its right neighbours wrap to the start.
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
template <> __device__ __forceinline__ float hi_at<F32>(const void* u, int64_t g) {
  return static_cast<const float*>(u)[g];
}

template <int ST, class DT>
__global__ void __launch_bounds__(kNaiveThreads)
naive_step_kernel(const void* __restrict__ in, void* __restrict__ out, int64_t N, const Consts c) {
  constexpr int R = Radius<ST>::value;
  griddep_wait();
  using Cc = typename DT::C;
  const int lane = threadIdx.x & 31;
  const int64_t i0 = ((int64_t)blockIdx.x * kNaiveThreads + threadIdx.x) * kV;
  const bool valid = i0 < N;
  // the last thread of a field whose N is not a multiple of V owns fewer points
  const int64_t left = N - i0;
  const bool full = left >= kV;
  Tile<DT, kV> t;
  t.zero();
  if (valid) {
    if (full) {
      load_points<kV>(t, in, N, i0);
    } else {
      Tile<DT, 1> one;
#pragma unroll
      for (int k = 0; k < kV; ++k) {
        if (k < left) {
          load_points<1>(one, in, N, i0 + k);
          t.put(k, one.get(0));
        }
      }
    }
  }
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
  if (!full) {
    // the points after the tail wrap to the start of the field
#pragma unroll
    for (int k = 0; k < kV + R; ++k) {
      if (k >= left && k < left + R) {
        int64_t g = i0 + k;
        if (g >= N) g -= N;
        x[R + k] = hi_at<DT>(in, g);
      }
    }
  } else if (lane == 31 || i0 + kV + R > N) {
#pragma unroll
    for (int i = 0; i < R; ++i) {
      int64_t g = i0 + kV + i;
      if (g >= N) g -= N;
      x[R + kV + i] = hi_at<DT>(in, g);
    }
  }
  Core<ST, DT, kV>::apply(t, x, c);
  if (full) {
    store_points<kV>(t, out, N, i0);
  } else {
#pragma unroll
    for (int k = 0; k < kV; ++k)
      if (k < left) store_point<kV>(t, k, out, N, i0 + k);
  }
}

template <int ST, class DT>
cudaError_t launch(const void* in, void* out, int64_t N, const Consts& c, cudaStream_t s, bool pdl) {
  const int64_t threads = (N + kV - 1) / kV;
  const int64_t grid = (threads + kNaiveThreads - 1) / kNaiveThreads;
  return launch_kernel(pdl, naive_step_kernel<ST, DT>, dim3((unsigned)grid), dim3(kNaiveThreads), 0, s, in, out,
                       N, c);
}

// Runge-Kutta sub-timestep on the whole field: sub 0 writes m = A(u) to out,
// sub 1 writes u' = B(u, m) to out.
template <int ST>
__global__ void __launch_bounds__(kNaiveThreads)
naive_rk2_kernel(int sub, const double* __restrict__ u, const double* __restrict__ m,
                 double* __restrict__ out, int64_t N, const Consts c) {
  constexpr int R = Radius<ST>::value;
  griddep_wait();
  const int lane = threadIdx.x & 31;
  const int64_t i0 = ((int64_t)blockIdx.x * kNaiveThreads + threadIdx.x) * kV;
  const bool valid = i0 < N;
  const int64_t left = N - i0;           // the last thread may own fewer than V points
  const bool full = left >= kV;
  const double* arg = sub == 0 ? u : m;
  Tile<F64P, kV> t;
  t.zero();
  if (valid) {
    if (full) {
      ld_chunk<kV>(u + i0, t.u);
      ld_chunk<kV>(arg + i0, t.m);
    } else {
#pragma unroll
      for (int k = 0; k < kV; ++k) {
        if (k < left) {
          t.u[k] = u[i0 + k];
          t.m[k] = arg[i0 + k];
        }
      }
    }
  }
  double x[kV + 2 * R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    x[i] = __shfl_sync(kFull, t.m[kV - R + i], (lane + 31) & 31);
    x[R + kV + i] = __shfl_sync(kFull, t.m[i], (lane + 1) & 31);
  }
#pragma unroll
  for (int k = 0; k < kV; ++k) x[R + k] = t.m[k];
  if (!valid) return;
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < R; ++i) {
      int64_t g = i0 - R + i;
      if (g < 0) g += N;
      x[i] = arg[g];
    }
  }
  if (!full) {
#pragma unroll
    for (int k = 0; k < kV + R; ++k) {
      if (k >= left && k < left + R) {
        int64_t g = i0 + k;
        if (g >= N) g -= N;
        x[R + k] = arg[g];
      }
    }
  } else if (lane == 31 || i0 + kV + R > N) {
#pragma unroll
    for (int i = 0; i < R; ++i) {
      int64_t g = i0 + kV + i;
      if (g >= N) g -= N;
      x[R + kV + i] = arg[g];
    }
  }
  RK2Core<ST, kV>::apply(t, x, c, sub);
  const double* res = sub == 0 ? t.m : t.u;
  if (full) {
    st_chunk<kV>(out + i0, res);
  } else {
#pragma unroll
    for (int k = 0; k < kV; ++k)
      if (k < left) out[i0 + k] = res[k];
  }
}

// Euler equations, one stage of the midpoint rule per launch (the slopes
// and the flux update fused: radius 2 in the argument).  A block of T
// threads evaluates T consecutive faces, one per thread, and updates the
// T - 1 points between them; it first stages the argument of points
// [b0-2, b0+T+1) in shared memory, then the minmod slopes of [b0-1, b0+T).
// Updates (dF = F_{i+1/2} - F_{i-1/2}):
//   MODE 0 (FP64):              out = fma(-ca, dF, base)
//   MODE 1 (F32C, midpoint):    out = hi + fma(-ca, dF, lo)
//   MODE 2 (F32C, full step):   (out, out_lo) = TwoSum(hi, fma(-ca, dF, lo))
// with base / hi = `base` and lo = `lo`.  Each face is evaluated once, with
// the expressions of the swept kernels, so the results agree bit for bit.
constexpr int kEulerT = 128;

template <class T, int MODE>
__global__ void __launch_bounds__(kEulerT)
naive_euler_kernel(const T* __restrict__ arg, const T* __restrict__ base, const T* __restrict__ lo,
                   T* __restrict__ out, T* __restrict__ out_lo, int64_t N, T ca, T g1) {
  using O = EOps<T>;
  __shared__ T sa[3][kEulerT + 3], ss[3][kEulerT + 1], sf[3][kEulerT];
  griddep_wait();
  const int64_t b0 = (int64_t)blockIdx.x * (kEulerT - 1);
  for (int j = threadIdx.x; j < kEulerT + 3; j += kEulerT) {
    int64_t g = (b0 - 2 + j) % N;
    if (g < 0) g += N;
#pragma unroll
    for (int c = 0; c < 3; ++c) sa[c][j] = arg[c * N + g];
  }
  __syncthreads();
  for (int j = threadIdx.x; j < kEulerT + 1; j += kEulerT) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
      ss[c][j] = minmod<T>(O::sub(sa[c][j + 1], sa[c][j]), O::sub(sa[c][j + 2], sa[c][j + 1]));
  }
  __syncthreads();
  {
    // face f between points b0-1+f (left) and b0+f (right)
    const int f = threadIdx.x;
    T aL[3], sL[3], aR[3], sR[3], F[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      aL[c] = sa[c][f + 1];
      sL[c] = ss[c][f];
      aR[c] = sa[c][f + 2];
      sR[c] = ss[c][f + 1];
    }
    euler_face<T>(aL, sL, aR, sR, g1, F);
#pragma unroll
    for (int c = 0; c < 3; ++c) sf[c][f] = F[c];
  }
  __syncthreads();
  const int j = threadIdx.x;
  const int64_t g = b0 + j;
  if (j < kEulerT - 1 && g < N) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T dF = O::sub(sf[c][j + 1], sf[c][j]);
      const int64_t x = c * N + g;
      if constexpr (MODE == 0) {
        out[x] = O::fma(-ca, dF, base[x]);
      } else if constexpr (MODE == 1) {
        out[x] = O::add(base[x], O::fma(-ca, dF, lo[x]));
      } else {
        float h, l;
        two_sum(base[x], O::fma(-ca, dF, lo[x]), h, l);
        out[x] = h;
        out_lo[x] = l;
      }
    }
  }
}

}  // namespace

cudaError_t launch_naive_euler(const double* arg, const double* base, double* out, int64_t N, double ca,
                               double g1, cudaStream_t s, bool pdl) {
  if (N <= 0) return cudaErrorInvalidValue;
  const int64_t grid = (N + kEulerT - 2) / (kEulerT - 1);
  return launch_kernel(pdl, naive_euler_kernel<double, 0>, dim3((unsigned)grid), dim3(kEulerT), 0, s, arg, base,
                       (const double*)nullptr, out, (double*)nullptr, N, ca, g1);
}

cudaError_t launch_naive_euler_f32c(int full, const float* arg, const float* hi, const float* lo, float* out,
                                    float* out_lo, int64_t N, float ca, float g1, cudaStream_t s, bool pdl) {
  if (N <= 0) return cudaErrorInvalidValue;
  const int64_t grid = (N + kEulerT - 2) / (kEulerT - 1);
  if (full)
    return launch_kernel(pdl, naive_euler_kernel<float, 2>, dim3((unsigned)grid), dim3(kEulerT), 0, s, arg, hi, lo,
                         out, out_lo, N, ca, g1);
  return launch_kernel(pdl, naive_euler_kernel<float, 1>, dim3((unsigned)grid), dim3(kEulerT), 0, s, arg, hi, lo,
                       out, (float*)nullptr, N, ca, g1);
}

cudaError_t launch_naive_rk2(int stencil, int sub, const double* u, const double* m, double* out, int64_t N,
                             const Consts& c, cudaStream_t s, bool pdl) {
  if (N <= 0) return cudaErrorInvalidValue;
  const int64_t grid = ((N + kV - 1) / kV + kNaiveThreads - 1) / kNaiveThreads;
  if (stencil == 2)
    return launch_kernel(pdl, naive_rk2_kernel<kHeatRK2>, dim3((unsigned)grid), dim3(kNaiveThreads), 0, s, sub, u,
                         m, out, N, c);
  return launch_kernel(pdl, naive_rk2_kernel<kKSRK2>, dim3((unsigned)grid), dim3(kNaiveThreads), 0, s, sub, u, m,
                       out, N, c);
}

cudaError_t launch_naive_step(int stencil, int dtype, const void* in, void* out, int64_t N,
                              const Consts& c, cudaStream_t s, bool pdl) {
  if (N <= 0) return cudaErrorInvalidValue;
  if (stencil == kHeat) {
    if (dtype == 2) return launch<kHeat, F32>(in, out, N, c, s, pdl);
    return dtype == 0 ? launch<kHeat, F64>(in, out, N, c, s, pdl) : launch<kHeat, F32C>(in, out, N, c, s, pdl);
  }
  if (dtype == 2) return launch<kKS, F32>(in, out, N, c, s, pdl);
  return dtype == 0 ? launch<kKS, F64>(in, out, N, c, s, pdl) : launch<kKS, F32C>(in, out, N, c, s, pdl);
}

}  // namespace swept
