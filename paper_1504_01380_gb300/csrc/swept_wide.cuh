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

#include "swept_stage.cuh"

namespace swept {


template <int ST, class DT, int K, int KW>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
swept_wide_kernel(const StageArgs a, int nreg, int odd) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using E = typename DT::E;
  constexpr int B = 32 * K, BW = 32 * KW;
  griddep_wait();
  E* sm = reinterpret_cast<E*>(smem_raw) + (threadIdx.x >> 5) * (2 * BW);
  const int i = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int j = nreg + i;
  if (j >= a.nwin) return;                                   // warp-uniform
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
cudaError_t launch_wk(const StageArgs& a, int nreg, int odd, cudaStream_t s) {
  const size_t smem = stage_smem_bytes(32 * KW, (int)sizeof(typename DT::E));
  cudaError_t e = cudaFuncSetAttribute(swept_wide_kernel<ST, DT, K, KW>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int nwide = a.nwin - nreg;
  const int grid = (nwide + kWarpsPerBlock - 1) / kWarpsPerBlock;
  return launch_kernel(a.pdl != 0, swept_wide_kernel<ST, DT, K, KW>, dim3(grid), dim3(kWarpsPerBlock * 32), smem,
                       s, a, nreg, odd);
}

}  // namespace swept
