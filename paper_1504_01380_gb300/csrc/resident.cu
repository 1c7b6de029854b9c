// Cluster-resident swept advance, for problems of at most 64 windows: the
// whole advance in one launch of one thread block cluster (up to 16 blocks
// on 16 SMs, one warp per window).  At the end of a stage each window pushes
// its two edge halves into the shared memory of the two windows of the next
// stage that read them (through distributed shared memory), and the stage
// boundary is a cluster barrier.  On
// GB300 that barrier (with a remote shared-memory load) takes about 0.27 us,
// where a stage boundary through global memory and a kernel launch costs
// about 2.4 us (the latency tau of Eq. 1 on this GPU), and every window still
// has a warp of its own (at most one per warp scheduler), as with the
// per-stage launches.  Nothing waits on a flag: the barrier is the only synchronisation.
#include <cooperative_groups.h>
#include <type_traits>

#include "swept.h"
#include "swept_internal.h"
#include "swept_stage.cuh"
#include "swept_sync.cuh"

namespace cg = cooperative_groups;

namespace swept {

namespace {

// Warps per block W (1, 2 or 4: the smallest that divides nwin and keeps
// C <= 16) and blocks C = nwin / W of a plan's cluster; false when none
// does.  Spreading the windows over more SMs measured faster for FP64 (an
// SM's warp schedulers share its FP64 pipe; heat, N = 1024: 337 -> 318 ns
// per sub-timestep at 32 windows on 16 SMs instead of 8, 582 -> 527 at 16
// windows) and the same for the compensated state.
bool cluster_shape(int nwin, int& W, int& C) {
  for (W = 1; W <= 4; W *= 2) {
    if (nwin % W == 0 && nwin / W <= 16) {
      C = nwin / W;
      return true;
    }
  }
  return false;
}

// Shared memory per block, per warp: the stage's output edges (2B elements:
// the left half, then the right), the arms of the next stage in two parity
// buffers of 3B elements ([B, 2B) the left arm, [2B, 3B) the right; [0, B)
// unused), and the stage code's staging area (2B elements).
template <class DT>
size_t cluster_smem(int W, int B) {
  return (size_t)W * 10 * B * sizeof(typename DT::E);
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
  E* base = reinterpret_cast<E*>(smem_raw);
  E* eout = base + (size_t)wi * 2 * B;                      // [W][2B]
  E* arms0 = base + (size_t)2 * W * B;                      // [2][W][3B]
  E* sm = base + (size_t)8 * W * B + (size_t)wi * 2 * B;    // [W][2B]
  StageArgs a = p.a;
  for (int k = 0; k < p.nstages; ++k) {
    stage_shape(k, p.q, p.rem, p.H, a.hv, a.ht);
    a.offset = (k & 1) ? B / 2 : 0;
    a.lev_fill = k >= 1 ? (int64_t)(k - 1) * p.H : 0;
    a.lev_trap = (int64_t)k * p.H;
    // the stage code reads its arms at windows 0 (right half) and 1 (left half) of a.ein,
    // pushed here by the windows that computed them, and writes its edges to window 0 of
    // a.eout
    a.ein = arms0 + (size_t)(k & 1) * W * 3 * B + (size_t)wi * 3 * B;
    a.eout = eout;
    StageImpl<ST, DT, K>::run_window_at(a, sm, (int64_t)w * B + a.offset, 0, 1, 0, B, false);
    if (a.ht > 0 && k + 1 < p.nstages) {
      // push the edges to the windows of stage k + 1 that read them: at an offset stage
      // window v reads windows v and v + 1 of stage k, at an unshifted one v - 1 and v; so
      // the right edges go to the left arm of window w (next stage offset) or w + 1, the left
      // edges to the right arm of window w - 1 or w
      __syncwarp();
      const bool next_offset = ((k + 1) & 1) != 0;
      const int vr = next_offset ? w : (w + 1 == nwin ? 0 : w + 1);
      const int vl = next_offset ? (w == 0 ? nwin - 1 : w - 1) : w;
      E* nxt = arms0 + (size_t)((k + 1) & 1) * W * 3 * B;
      uint4* dR = reinterpret_cast<uint4*>(
          cl.map_shared_rank(nxt + (size_t)(vr % W) * 3 * B + B, (unsigned)(vr / W)));
      uint4* dL = reinterpret_cast<uint4*>(
          cl.map_shared_rank(nxt + (size_t)(vl % W) * 3 * B + 2 * B, (unsigned)(vl / W)));
      const uint4* sR = reinterpret_cast<const uint4*>(eout + B);
      const uint4* sL = reinterpret_cast<const uint4*>(eout);
      const int n16 = (a.ht * 2 * R * (int)sizeof(E) + 15) / 16;
      for (int i = lane; i < n16; i += 32) {
        dR[i] = sR[i];
        dL[i] = sL[i];
      }
    }
    cl.sync();                                                 // stage k's edges are in the arms
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
