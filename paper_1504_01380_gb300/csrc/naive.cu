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
#include <cooperative_groups.h>
#include <type_traits>

#include "swept_internal.h"

namespace cg = cooperative_groups;

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

// One sub-timestep of the kV points of the thread starting at i0 (in, out:
// whole fields, in global or shared memory).  Every lane of the warp calls
// it (the shuffles); lanes past the field's end store nothing.
template <int ST, class DT>
__device__ __forceinline__ void naive_points(const void* __restrict__ in, void* __restrict__ out, int64_t N,
                                             const Consts& c, int64_t i0, int lane) {
  constexpr int R = Radius<ST>::value;
  using Cc = typename DT::C;
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
__global__ void __launch_bounds__(kNaiveThreads)
naive_step_kernel(const void* __restrict__ in, void* __restrict__ out, int64_t N, const Consts c) {
  griddep_wait();
  const int64_t i0 = ((int64_t)blockIdx.x * kNaiveThreads + threadIdx.x) * kV;
  naive_points<ST, DT>(in, out, N, c, i0, threadIdx.x & 31);
}

// Every step of a naive advance in one thread block cluster (the per-step
// counterpart of the cluster-resident swept advance): the field is split over
// the C blocks, M = N / C points each, held in shared memory with R halo
// points per side, [R halo | M own | R halo], in two buffers (hi then lo for
// a compensated field).  Each step steps the padded field (its own points
// need no wrap) into the other buffer, then pushes its first and last R own
// points into the neighbouring blocks' halo inboxes through distributed
// shared memory, and ends with a cluster barrier; the next step starts by
// copying its inbox into its halo.  One barrier per sub-timestep where the
// swept advance needs one per stage.
template <int ST, class DT>
__global__ void __launch_bounds__(1024, 1)
naive_cluster_kernel(void* __restrict__ u, int64_t N, const Consts c, int64_t nsteps, int M) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int R = Radius<ST>::value;
  constexpr int NC = std::is_same<DT, F32C>::value ? 2 : 1;   // components (hi, lo)
  constexpr int NH = 2 * R * NC;                             // halo values per block
  using Cc = typename DT::C;
  cg::cluster_group cl = cg::this_cluster();
  griddep_wait();
  const int L = M + 2 * R;                                   // padded field
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int left = (rank + C - 1) % C, right = (rank + 1) % C;
  Cc* buf[2] = {reinterpret_cast<Cc*>(smem_raw), reinterpret_cast<Cc*>(smem_raw) + NC * L};
  // inbox[p][j * 2R + q]: halo point q of component j (q < R: left halo, else right),
  // written by the neighbours at the end of the step before one of parity p
  Cc* inbox[2] = {buf[1] + NC * L, buf[1] + NC * L + NH};
  const int64_t g0 = (int64_t)rank * M;
  Cc* uc = static_cast<Cc*>(u);
  for (int i = threadIdx.x; i < M; i += blockDim.x)
#pragma unroll
    for (int j = 0; j < NC; ++j) buf[0][j * L + R + i] = uc[j * N + g0 + i];
  cl.sync();                                                 // every block started and loaded
  const int tid = threadIdx.x;
  const int jh = tid / (2 * R), qh = tid % (2 * R);         // this thread's halo value (tid < NH)
  if (tid < NH) {
    // step 0's halo, read from the neighbours once: the left block's own points M - R + q
    // (its buf[0][M + q]), the right block's own points q (its buf[0][R + q])
    Cc* b0 = buf[0];
    if (qh < R) b0[jh * L + qh] = *cl.map_shared_rank(b0 + jh * L + M + qh, (unsigned)left);
    else b0[jh * L + M + qh] = *cl.map_shared_rank(b0 + jh * L + qh, (unsigned)right);
  }
  const int64_t i0 = (int64_t)tid * kV;
  for (int64_t k = 0; k < nsteps; ++k) {
    Cc* cur = buf[k & 1];
    Cc* nxt = buf[(k + 1) & 1];
    if (k > 0 && tid < NH) cur[jh * L + (qh < R ? qh : M + qh)] = inbox[k & 1][tid];
    __syncthreads();
    naive_points<ST, DT>(cur, nxt, L, c, i0, tid & 31);
    __syncthreads();
    if (tid < NH) {
      // my first R own points go to the left block's right halo (its q = R + q'), my last R
      // own points to the right block's left halo (its q = q')
      Cc* box = inbox[(k + 1) & 1];
      if (qh < R) *cl.map_shared_rank(box + jh * 2 * R + R + qh, (unsigned)left) = nxt[jh * L + R + qh];
      else *cl.map_shared_rank(box + jh * 2 * R + qh - R, (unsigned)right) = nxt[jh * L + M + qh - R];
    }
    cl.sync();                                               // the halos are in the inboxes
  }
  const Cc* fin = buf[nsteps & 1];
  for (int i = threadIdx.x; i < M; i += blockDim.x)
#pragma unroll
    for (int j = 0; j < NC; ++j) uc[j * N + g0 + i] = fin[j * L + R + i];
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
    bool ok = true;
    euler_face<T, true>(aL, sL, aR, sR, g1, F, ok);   // straight-line division and square root
    if (!ok) euler_face<T>(aL, sL, aR, sR, g1, F);    // where they could not prove their result
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

namespace {
// Blocks C of a naive cluster: the most (at most 16) that divide N into parts
// of at least 4R points whose padded part (M + 2R points, 4 per thread) fits
// one block of 1024 threads.
int naive_cluster_blocks(int64_t N, int R) {
  for (int C = 16; C >= 1; --C) {
    if (N % C) continue;
    const int64_t M = N / C;
    if (M >= 4 * R && (M + 2 * R + kV - 1) / kV <= 1024) return C;
  }
  return 0;
}

template <int ST, class DT>
cudaError_t launch_res(void* u, int64_t N, const Consts& c, int64_t nsteps, cudaStream_t s, bool pdl, bool query,
                       int* fits) {
  constexpr int R = Radius<ST>::value;
  constexpr int NC = std::is_same<DT, F32C>::value ? 2 : 1;
  if (query) *fits = 0;
  const int C = naive_cluster_blocks(N, R);
  if (C == 0) return query ? cudaSuccess : cudaErrorInvalidValue;
  const int M = (int)(N / C), L = M + 2 * R;
  const size_t smem = (size_t)(2 * NC * L + 2 * 2 * R * NC) * sizeof(typename DT::C);   // fields, inboxes
  const int threads = ((L + kV - 1) / kV + 31) / 32 * 32;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem > (size_t)optin) return query ? cudaSuccess : cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(naive_cluster_kernel<ST, DT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e == cudaSuccess && C > 8)
    e = cudaFuncSetAttribute(naive_cluster_kernel<ST, DT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  return launch_cluster(pdl, naive_cluster_kernel<ST, DT>, dim3(C), dim3(threads), smem, s, query, fits, u, N, c,
                        nsteps, M);
}
}  // namespace

cudaError_t launch_naive_resident(int stencil, int dtype, void* u, int64_t N, const Consts& c, int64_t nsteps,
                                  cudaStream_t s, bool pdl, bool query, int* fits) {
  if (N <= 0) return cudaErrorInvalidValue;
  if (stencil == kHeat) {
    if (dtype == 2) return launch_res<kHeat, F32>(u, N, c, nsteps, s, pdl, query, fits);
    return dtype == 0 ? launch_res<kHeat, F64>(u, N, c, nsteps, s, pdl, query, fits)
                      : launch_res<kHeat, F32C>(u, N, c, nsteps, s, pdl, query, fits);
  }
  if (dtype == 2) return launch_res<kKS, F32>(u, N, c, nsteps, s, pdl, query, fits);
  return dtype == 0 ? launch_res<kKS, F64>(u, N, c, nsteps, s, pdl, query, fits)
                    : launch_res<kKS, F32C>(u, N, c, nsteps, s, pdl, query, fits);
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
