// Compensated-state conversion and FP64 reductions.
//
// Reductions (conserved sum, objective J = 1/2 sum u^2, directional
// derivative <u, v>) accumulate in FP64 with TwoSum compensation; products
// are split exactly with an FMA (TwoProd).  Pass 1 gives each of a fixed
// number of blocks a fixed grid-stride share and reduces it to a (sum, error)
// pair by a fixed tree; pass 2 combines the pairs in one block.  The order of
// every operation is fixed, so results are bitwise reproducible.
#include "swept_internal.h"

namespace swept {

namespace {

constexpr int kRedThreads = 256;

__global__ void split_kernel(int64_t N, const double* __restrict__ u, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double x = u[i];
  const float h = __double2float_rn(x);
  out[i] = h;
  out[N + i] = __double2float_rn(__dsub_rn(x, (double)h));
}

__global__ void merge_kernel(int64_t N, const float* __restrict__ in, double* __restrict__ u) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  u[i] = __dadd_rn((double)in[i], (double)in[N + i]);
}

__device__ __forceinline__ void two_sum64(double a, double b, double& s, double& e) {
  const double t = __dadd_rn(a, b);
  const double bb = __dsub_rn(t, a);
  e = __dadd_rn(__dsub_rn(a, __dsub_rn(t, bb)), __dsub_rn(b, bb));
  s = t;
}

struct Acc {
  double s, c;
  __device__ __forceinline__ void add(double x) {
    double e;
    two_sum64(s, x, s, e);
    c = __dadd_rn(c, e);
  }
  __device__ __forceinline__ void merge(double s2, double c2) {
    double e;
    two_sum64(s, s2, s, e);
    c = __dadd_rn(__dadd_rn(c, c2), e);
  }
};

template <int DT> __device__ __forceinline__ double value_at(const void* u, int64_t N, int64_t i);
template <> __device__ __forceinline__ double value_at<0>(const void* u, int64_t, int64_t i) {
  return static_cast<const double*>(u)[i];
}
template <> __device__ __forceinline__ double value_at<1>(const void* u, int64_t N, int64_t i) {
  const float* f = static_cast<const float*>(u);
  return __dadd_rn((double)f[i], (double)f[N + i]);
}
template <> __device__ __forceinline__ double value_at<2>(const void* u, int64_t, int64_t i) {
  return (double)static_cast<const float*>(u)[i];
}

__device__ __forceinline__ void block_reduce(Acc& acc, double* sh_s, double* sh_c) {
  const int tid = threadIdx.x;
  sh_s[tid] = acc.s;
  sh_c[tid] = acc.c;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w) {
      Acc a{sh_s[tid], sh_c[tid]};
      a.merge(sh_s[tid + w], sh_c[tid + w]);
      sh_s[tid] = a.s;
      sh_c[tid] = a.c;
    }
    __syncthreads();
  }
  acc.s = sh_s[0];
  acc.c = sh_c[0];
}

template <int DT, int WHAT>
__global__ void __launch_bounds__(kRedThreads)
reduce_pass1(const void* __restrict__ u, const double* __restrict__ v, int64_t N,
             double* __restrict__ scratch) {
  __shared__ double sh_s[kRedThreads], sh_c[kRedThreads];
  Acc acc{0.0, 0.0};
  const int64_t stride = (int64_t)gridDim.x * kRedThreads;
  for (int64_t i = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; i < N; i += stride) {
    const double x = value_at<DT>(u, N, i);
    if (WHAT == 0) {
      acc.add(x);
    } else {
      const double y = (WHAT == 1) ? x : v[i];
      const double p = __dmul_rn(x, y);
      const double e = __fma_rn(x, y, -p);      // x*y = p + e exactly
      acc.add(p);
      acc.add(e);
    }
  }
  block_reduce(acc, sh_s, sh_c);
  if (threadIdx.x == 0) {
    scratch[2 * blockIdx.x] = acc.s;
    scratch[2 * blockIdx.x + 1] = acc.c;
  }
}

__global__ void __launch_bounds__(kRedThreads)
reduce_pass2(const double* __restrict__ scratch, int nblocks, double scale, double* __restrict__ out) {
  __shared__ double sh_s[kRedThreads], sh_c[kRedThreads];
  Acc acc{0.0, 0.0};
  for (int b = threadIdx.x; b < nblocks; b += kRedThreads) acc.merge(scratch[2 * b], scratch[2 * b + 1]);
  block_reduce(acc, sh_s, sh_c);
  if (threadIdx.x == 0) out[0] = __dmul_rn(__dadd_rn(acc.s, acc.c), scale);
}

template <int DT, int WHAT>
cudaError_t reduce_t(const void* u, const double* v, int64_t N, double* scratch, double* out,
                     cudaStream_t s) {
  reduce_pass1<DT, WHAT><<<kReduceBlocks, kRedThreads, 0, s>>>(u, v, N, scratch);
  reduce_pass2<<<1, kRedThreads, 0, s>>>(scratch, kReduceBlocks, WHAT == 1 ? 0.5 : 1.0, out);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_split(int64_t N, const double* u64, float* u32c, cudaStream_t s) {
  split_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, u64, u32c);
  return cudaGetLastError();
}

cudaError_t launch_merge(int64_t N, const float* u32c, double* u64, cudaStream_t s) {
  merge_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, u32c, u64);
  return cudaGetLastError();
}

cudaError_t launch_reduce(int dtype, const void* u, int what, const double* v, int64_t N,
                          double* scratch, double* out, cudaStream_t s) {
  if (dtype == 0) {
    if (what == 0) return reduce_t<0, 0>(u, v, N, scratch, out, s);
    if (what == 1) return reduce_t<0, 1>(u, v, N, scratch, out, s);
    return reduce_t<0, 2>(u, v, N, scratch, out, s);
  }
  if (dtype == 2) {
    if (what == 0) return reduce_t<2, 0>(u, v, N, scratch, out, s);
    if (what == 1) return reduce_t<2, 1>(u, v, N, scratch, out, s);
    return reduce_t<2, 2>(u, v, N, scratch, out, s);
  }
  if (what == 0) return reduce_t<1, 0>(u, v, N, scratch, out, s);
  if (what == 1) return reduce_t<1, 1>(u, v, N, scratch, out, s);
  return reduce_t<1, 2>(u, v, N, scratch, out, s);
}

}  // namespace swept
