// Cluster-resident swept advance, for problems of at most 64 windows: the
// whole advance in one launch of one thread block cluster (up to 16 blocks
// on 16 SMs, one warp per window).  Each block keeps its windows' stage edges
// in its shared memory; a window's V-fill reads its neighbours' edges through
// distributed shared memory, and the stage boundary is a cluster barrier.  On
// GB300 that barrier (with a remote shared-memory load) takes about 0.27 us,
// where a stage boundary through global memory and a kernel launch costs
// about 2.4 us (the latency tau of Eq. 1 on this GPU), and every window still
// has a warp of its own (one per warp scheduler), as with the per-stage
// launches.  Nothing waits on a flag: the barrier is the only synchronisation.
#include <cooperative_groups.h>
#include <type_traits>

#include "swept.h"
#include "swept_internal.h"
#include "swept_stage.cuh"
#include "swept_sync.cuh"

namespace cg = cooperative_groups;

namespace swept {

namespace {

// Warps per block W (4, 2 or 1: the largest that divides nwin) and blocks C
// = nwin / W of a plan's cluster; false when C would exceed 16.
bool cluster_shape(int nwin, int& W, int& C) {
  for (W = 4; W >= 1; W /= 2) {
    if (nwin % W == 0 && nwin / W <= 16) {
      C = nwin / W;
      return true;
    }
  }
  return false;
}

// Shared memory per block: the edge double buffer of its W windows (2 x W x
// 2B elements), each warp's two arms (3B elements: [B, 2B) left, [2B, 3B)
// right; [0, B) unused) and the stage code's staging area (2B elements).
template <class DT>
size_t cluster_smem(int W, int B) {
  return (size_t)W * 9 * B * sizeof(typename DT::E);
}

template <int ST, class DT, int K>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 1) swept_cluster_kernel(const ResidentArgs p, int W) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using E = typename DT::E;
  constexpr int B = 32 * K;
  constexpr int R = Radius<ST>::value;
  cg::cluster_group cl = cg::this_cluster();
  griddep_wait();
  const int lane = threadIdx.x & 31;
  const int wi = threadIdx.x >> 5;                          // this warp's window in the block
  const int w = (int)cl.block_rank() * W + wi;              // window index
  const int nwin = p.a.nwin;
  E* ebuf = reinterpret_cast<E*>(smem_raw);                 // [2][W][2B]
  E* arms = ebuf + (size_t)4 * W * B + (size_t)wi * 3 * B;
  E* sm = ebuf + (size_t)7 * W * B + (size_t)wi * 2 * B;
  StageArgs a = p.a;
  for (int k = 0; k < p.nstages; ++k) {
    stage_shape(k, p.q, p.rem, p.H, a.hv, a.ht);
    a.offset = (k & 1) ? B / 2 : 0;
    a.lev_fill = k >= 1 ? (int64_t)(k - 1) * p.H : 0;
    a.lev_trap = (int64_t)k * p.H;
    if (a.hv > 0) {
      // the V's arms: the right edges of window wl and the left edges of window wr of
      // stage k - 1, in the blocks that hold them
      const int wl = a.offset ? w : (w == 0 ? nwin - 1 : w - 1);
      const int wr = a.offset ? (w + 1 == nwin ? 0 : w + 1) : w;
      const E* prev = ebuf + (size_t)((k + 1) & 1) * W * 2 * B;
      const uint4* srcL = reinterpret_cast<const uint4*>(
          cl.map_shared_rank(prev + (size_t)(wl % W) * 2 * B + B, (unsigned)(wl / W)));
      const uint4* srcR = reinterpret_cast<const uint4*>(
          cl.map_shared_rank(prev + (size_t)(wr % W) * 2 * B, (unsigned)(wr / W)));
      uint4* dL = reinterpret_cast<uint4*>(arms + B);
      uint4* dR = reinterpret_cast<uint4*>(arms + 2 * B);
      const int n16 = (a.hv * 2 * R * (int)sizeof(E) + 15) / 16;
      for (int i = lane; i < n16; i += 32) {
        dL[i] = srcL[i];
        dR[i] = srcR[i];
      }
      __syncwarp();
    }
    // the stage code reads its arms at windows 0 (right half) and 1 (left half) of
    // a.ein and writes its edges to window 0 of a.eout
    a.ein = arms;
    a.eout = ebuf + (size_t)(k & 1) * W * 2 * B + (size_t)wi * 2 * B;
    StageImpl<ST, DT, K>::run_window_at(a, sm, (int64_t)w * B + a.offset, 0, 1, 0, B, false);
    cl.sync();                                                 // stage k's edges, read by stage k + 1
  }
}

template <int ST, class DT, int K>
cudaError_t launch_k(const ResidentArgs& p, cudaStream_t s, bool pdl, bool query, int* fits) {
  constexpr int B = 32 * K;
  int W = 0, C = 0;
  if (query) *fits = 0;
  if (!cluster_shape(p.a.nwin, W, C)) return query ? cudaSuccess : cudaErrorInvalidValue;
  const size_t smem = cluster_smem<DT>(W, B);
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem > (size_t)optin) return query ? cudaSuccess : cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(swept_cluster_kernel<ST, DT, K>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && C > 8)
    e = cudaFuncSetAttribute(swept_cluster_kernel<ST, DT, K>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  return launch_cluster(pdl, swept_cluster_kernel<ST, DT, K>, dim3(C), dim3(32 * W), smem, s, query, fits, p, W);
}

template <int ST, class DT>
cudaError_t dispatch(int K, const ResidentArgs& p, cudaStream_t s, bool pdl, bool query, int* fits) {
  switch (K) {
    case 1:
      if constexpr (Radius<ST>::value == 1) return launch_k<ST, DT, 1>(p, s, pdl, query, fits);
      else return cudaErrorInvalidValue;
    case 2: return launch_k<ST, DT, 2>(p, s, pdl, query, fits);
    case 4:
      if constexpr (!std::is_same<DT, F64P>::value) return launch_k<ST, DT, 4>(p, s, pdl, query, fits);
      else return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_resident(int stencil, int dtype, int K, const ResidentArgs& p, cudaStream_t s, bool pdl,
                            bool query, int* fits) {
  if (query) *fits = 0;
  if (stencil == kHeatRK2) return dispatch<kHeatRK2, F64P>(K, p, s, pdl, query, fits);
  if (stencil == kKSRK2) return dispatch<kKSRK2, F64P>(K, p, s, pdl, query, fits);
  if (stencil == kHeat) {
    if (dtype == 0) return dispatch<kHeat, F64>(K, p, s, pdl, query, fits);
    if (dtype == 1) return dispatch<kHeat, F32C>(K, p, s, pdl, query, fits);
    return dispatch<kHeat, F32>(K, p, s, pdl, query, fits);
  }
  if (dtype == 0) return dispatch<kKS, F64>(K, p, s, pdl, query, fits);
  if (dtype == 1) return dispatch<kKS, F32C>(K, p, s, pdl, query, fits);
  return dispatch<kKS, F32>(K, p, s, pdl, query, fits);
}

}  // namespace swept
