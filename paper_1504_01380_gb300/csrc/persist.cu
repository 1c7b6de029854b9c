// Persistent swept advance for problems small enough that every window gets
// its own warp at once: the latency regime of Sections 4 and 6, where the
// stage boundary itself (on a GPU, a kernel launch: the latency tau of Eq. 1)
// is the cost the swept rule amortises.  One launch runs every stage: warp w
// owns window w at every stage; before stage k it waits until the two
// windows of stage k-1 it reads from (Section 3's neighbours) have published
// their edges, runs the per-window stage, and publishes.  The same wait keeps
// the edge double buffer safe: a window's stage-(k+1) edges overwrite its
// stage-(k-1) edges only after both readers of those have finished stage k.
// Every wait is bounded by a clock budget; a wait that runs out records
// SWEPT_ETIMEOUT in the plan's status word and the launch winds down.
#include "swept.h"
#include "swept_internal.h"
#include "swept_stage.cuh"
#include "swept_sync.cuh"

namespace swept {

namespace {

template <int ST, class DT, int K>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
swept_persistent_kernel(const PersistArgs p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using E = typename DT::E;
  constexpr int B = 32 * K;
  griddep_wait();
  E* sm = reinterpret_cast<E*>(smem_raw) + (threadIdx.x >> 5) * (2 * B);
  const int w = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (w >= p.a.nwin) return;                     // warp-uniform
  const int lane = threadIdx.x & 31;
  StageArgs a = p.a;
  for (int k = 0; k < p.nstages; ++k) {
    stage_shape(k, p.q, p.rem, p.H, a.hv, a.ht);
    a.offset = (k & 1) ? B / 2 : 0;
    a.ein = p.edges + ((k + 1) & 1) * p.edge_half;
    a.eout = p.edges + (k & 1) * p.edge_half;
    a.lev_fill = k >= 1 ? (int64_t)(k - 1) * p.H : 0;
    a.lev_trap = (int64_t)k * p.H;
    if (k >= 1) {
      const int wl = a.offset ? w : (w == 0 ? a.nwin - 1 : w - 1);
      const int wr = a.offset ? (w + 1 == a.nwin ? 0 : w + 1) : w;
      // both flags polled together with relaxed loads (both in flight at once),
      // then one acquire fence; the budget and the status word every 64 polls
      const long long t0 = clock64();
      bool ok = true;
      for (int it = 0;; ++it) {
        const int fl = ld_relaxed(p.flags + wl);
        const int fr = ld_relaxed(p.flags + wr);
        if (fl >= k && fr >= k) break;
        if ((it & 63) == 63 && (clock64() - t0 > p.budget || ld_relaxed(p.status) != 0)) {
          ok = false;
          break;
        }
      }
      fence_acq_rel();
      ok = __all_sync(kFull, ok);
      if (!ok) {
        if (lane == 0) atomicCAS(p.status, 0, SWEPT_ETIMEOUT);
        return;
      }
    }
    StageImpl<ST, DT, K>::run_window(a, sm, w);
    // the warp's edge and state stores, then one fence and the release by lane 0
    __syncwarp();
    if (lane == 0 && w != p.drop_w) {
      __threadfence();
      st_release(p.flags + w, k + 1);
    }
  }
}

template <int ST, class DT, int K>
cudaError_t launch_k(const PersistArgs& p, cudaStream_t s, bool pdl, bool query, int* fits) {
  constexpr int B = 32 * K;
  const size_t smem = stage_smem_bytes(B, (int)sizeof(typename DT::E));
  cudaError_t e = cudaFuncSetAttribute(swept_persistent_kernel<ST, DT, K>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = (p.a.nwin + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (query) {
    // every block must be resident at once: the warps wait on one another
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, swept_persistent_kernel<ST, DT, K>,
                                                      kWarpsPerBlock * 32, smem);
    *fits = (e == cudaSuccess && per_sm * sms >= grid) ? 1 : 0;
    return e;
  }
  return launch_kernel(pdl, swept_persistent_kernel<ST, DT, K>, dim3(grid), dim3(kWarpsPerBlock * 32), smem, s,
                       p);
}

template <int ST, class DT>
cudaError_t dispatch(int K, const PersistArgs& p, cudaStream_t s, bool pdl, bool query, int* fits) {
  switch (K) {
    case 1:
      if constexpr (Radius<ST>::value == 1) return launch_k<ST, DT, 1>(p, s, pdl, query, fits);
      else return cudaErrorInvalidValue;
    case 2: return launch_k<ST, DT, 2>(p, s, pdl, query, fits);
    case 4: return launch_k<ST, DT, 4>(p, s, pdl, query, fits);
    case 8: return launch_k<ST, DT, 8>(p, s, pdl, query, fits);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_persistent(int stencil, int dtype, int K, const PersistArgs& p, cudaStream_t s, bool pdl,
                              bool query, int* fits) {
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
