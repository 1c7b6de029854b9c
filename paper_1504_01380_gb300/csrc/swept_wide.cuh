// Uneven tiles (N not a multiple of the tile width B): the swept stages with
// the last windows wider than B: all B + 32r wide but the very last, which
// takes what is left (B + 1 .. B + 32r points).  Every V between two tiles stays exactly B
// wide (Section 3's V grows by r points per side per level around a tile
// boundary, whatever the tiles' widths), so a wide window of width W = B +
// 32r is its V (a regular B window centred on the previous stage's boundary)
// plus the flat top of the wide trapezoid of the previous stage, W - B points
// already at the stage's base level.  Windows keep their indices from stage
// to stage; their parts alternate sides: at odd stages the window starts B/2
// to the right and its V is at its right end, at even stages its V is at its
// left end.  One warp per wide window: the V part (regular per-window code)
// stores its flat level to the state, then the trapezoid of the full width
// W (per-window code of K + r points per lane) reloads it with the top part
// from the state, writes its edges to the window's slot and stores its own
// flat top for the next stage.
#pragma once

#include "swept_ring.cuh"
#include "swept_stage.cuh"

namespace swept {

// Wide window j = nreg + i of one stage, run by one warp; sm holds 2 x 32 KW
// elements of the warp's shared memory.
template <int ST, class DT, int K, int KW>
__device__ __forceinline__ void wide_window(const StageArgs& a, typename DT::E* sm, int nreg, int i, int odd) {
  constexpr int B = 32 * K, BW = 32 * KW;
  const int j = nreg + i;
  const int64_t N = a.N;
  const int64_t xj = (int64_t)j * B + (int64_t)i * (BW - B);   // start of tile j at stage 0
  const int64_t xj1 = j + 1 == a.nwin ? N : xj + BW;
  if (a.hv > 0) {
    StageArgs av = a;
    av.ht = 0;
    const int64_t vs = odd ? xj1 - B / 2 : xj;
    const int wl = odd ? j : (j == 0 ? a.nwin - 1 : j - 1);
    const int wr = odd ? (j + 1 == a.nwin ? 0 : j + 1) : j;
    StageImpl<ST, DT, K>::run_window_at(av, sm, vs, wl, wr, j, B, false);
    __syncwarp();
  }
  if (a.ht > 0) {
    StageArgs at = a;
    at.hv = 0;
    const int64_t ws = odd ? xj + B / 2 : xj;
    // the last window of a tiling of any N may be narrower than 32 KW points
    StageImpl<ST, DT, KW>::template run_window_at<true>(at, sm, ws, 0, 0, j, B, true, (int)(xj1 - xj));
  }
}

template <int ST, class DT, int K, int KW>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
swept_wide_kernel(const StageArgs a, int nreg, int odd) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using E = typename DT::E;
  constexpr int BW = 32 * KW;
  griddep_wait();
  E* sm = reinterpret_cast<E*>(smem_raw) + (threadIdx.x >> 5) * (2 * BW);
  const int i = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (nreg + i >= a.nwin) return;                            // warp-uniform
  wide_window<ST, DT, K, KW>(a, sm, nreg, i, odd);
}

// A full diamond stage of an uneven tiling in one launch: warps [0, nwarps)
// run the ring over the regular windows [0, nreg) (as swept_ring_kernel),
// the next nwin - nreg warps one wide window each.  The windows of a stage
// are independent, so the wide windows' per-window work overlaps the ring
// runs instead of following them in a launch of its own.
template <int ST, class DT, int K, int KW>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, RingBlocks<DT, KW>::value)
swept_ring_wide_kernel(const StageArgs a, int nwarps, int nreg, int odd) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using E = typename DT::E;
  constexpr int BW = 32 * KW;
  griddep_wait();
  E* sm = reinterpret_cast<E*>(smem_raw) + (threadIdx.x >> 5) * (2 * BW);
  const int gw = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (gw < nwarps) {
    const int w0 = (int)(((int64_t)gw * nreg) / nwarps);
    const int w1 = (int)(((int64_t)(gw + 1) * nreg) / nwarps);
    if (w1 > w0) RingImpl<ST, DT, K>::run(a, sm, w0, w1);
  } else if (nreg + (gw - nwarps) < a.nwin) {
    wide_window<ST, DT, K, KW>(a, sm, nreg, gw - nwarps, odd);
  }
}

// ring < 0: the wide windows alone (swept_wide_kernel).  ring >= 0: a full
// diamond stage, the ring over the nreg = a.nlaunch regular windows with
// `ring` warps (0: the resident warp slots less one per wide window, at most
// nreg / 2, FP64 states at most 4 per SM, as for swept_ring_kernel) and the
// wide windows, in one launch (swept_ring_wide_kernel).
template <int ST, class DT, int K, int KW>
cudaError_t launch_wk(const StageArgs& a, int nreg, int odd, cudaStream_t s, int ring = -1) {
  const size_t smem = stage_smem_bytes(32 * KW, (int)sizeof(typename DT::E));
  const int nwide = a.nwin - nreg;
  if (ring < 0) {
    cudaError_t e = cudaFuncSetAttribute(swept_wide_kernel<ST, DT, K, KW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = (nwide + kWarpsPerBlock - 1) / kWarpsPerBlock;
    return launch_kernel(a.pdl != 0, swept_wide_kernel<ST, DT, K, KW>, dim3(grid), dim3(kWarpsPerBlock * 32),
                         smem, s, a, nreg, odd);
  }
  if (nreg < 1) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(swept_ring_wide_kernel<ST, DT, K, KW>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int nwarps = ring;
  if (nwarps == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, swept_ring_wide_kernel<ST, DT, K, KW>,
                                                      kWarpsPerBlock * 32, smem);
    if (e != cudaSuccess) return e;
    nwarps = sms * (per_sm > 0 ? per_sm : 1) * kWarpsPerBlock - nwide;
    if (FP64Pipe<DT>::value && nwarps > 4 * sms) nwarps = 4 * sms;
    if (nwarps > nreg / 2) nwarps = nreg / 2;
  }
  if (nwarps > nreg) nwarps = nreg;
  if (nwarps < 1) nwarps = 1;
  const int grid = (nwarps + nwide + kWarpsPerBlock - 1) / kWarpsPerBlock;
  return launch_kernel(a.pdl != 0, swept_ring_wide_kernel<ST, DT, K, KW>, dim3(grid), dim3(kWarpsPerBlock * 32),
                       smem, s, a, nwarps, nreg, odd);
}

}  // namespace swept
