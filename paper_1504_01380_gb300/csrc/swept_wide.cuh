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
#include "swept_sync.cuh"

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

// Every full diamond stage of an advance on uneven tiles in one cooperative
// launch (a.nstream stages from the stage a describes).  Warps [0, nwarps)
// stream drifting runs of the regular windows [0, nreg) through the ring, as
// swept_stream_kernel does for even tiles (run indices modulo nreg, so a run
// may step from window nreg - 1 to window 0, whose physical neighbours are
// wide windows); the next nwin - nreg warps take one wide window each through
// every stage.  Windows publish per-window stage counters (a.progress[w] =
// streamed stages done, released after the window's edges are stored), and
// every window waits, bounded, before its fill of stage j until the two
// windows of stage j - 1 it reads from have published j: each wait is on an
// earlier stage, so the waits end.  The same wait keeps the edge buffers
// safe: a window's stage-j edges overwrite its stage-(j-2) edges, whose
// readers at stage j - 1 are the very windows its stage-j fill waited for.

// Bounded wait until window w has published `target` stages; false when the
// budget ran out or another warp recorded a failure.
__device__ __forceinline__ bool wait_window(const StageArgs& a, int w, int target) {
  const long long t0 = clock64();
  bool ok = true;
  for (int it = 0;; ++it) {
    if (ld_relaxed(a.progress + w) >= target) break;
    if ((it & 63) == 63 && (clock64() - t0 > a.budget || ld_relaxed(a.status) != 0)) {
      ok = false;
      break;
    }
    __nanosleep(128);
  }
  fence_acq_rel();
  return __all_sync(kFull, ok);
}

// (window a.drop never publishes: failure injection, a lost message)
__device__ __forceinline__ void publish_window(const StageArgs& a, int w, int stages) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0 && w != a.drop) {
    __threadfence();
    st_release(a.progress + w, stages);
  }
}

template <int ST, class DT, int K>
__device__ bool stream_uneven_ring(const StageArgs& a, typename DT::E* sm, int g, int nwarps, int nreg) {
  using RI = RingImpl<ST, DT, K>;
  using E = typename DT::E;
  constexpr int B = RI::B, H = RI::H;
  const int lane = threadIdx.x & 31;
  const int w0 = (int)(((int64_t)g * nreg) / nwarps);
  const int n = (int)(((int64_t)(g + 1) * nreg) / nwarps) - w0;
  if (n <= 0) return true;
  const int odd0 = a.offset != 0;
  E* s0 = sm;
  E* s1 = sm + B;
  Tile<DT, RI::S> t;
  t.zero();
  const int T = a.nstream * n;
  int jf = 0, i_f = 0, je = 0, ie = 0;
  for (int slot = 0; slot <= T; ++slot) {
    const bool fill = slot < T;
    const bool empty = slot > 0;
    const int cl = (slot & 1) ? 16 : 0;
    const bool offs = ((jf + odd0) & 1) != 0;
    const int wf = (w0 + ((jf + odd0) >> 1) + i_f) % nreg;
    if (fill) {
      const int wl = offs ? wf : (wf == 0 ? a.nwin - 1 : wf - 1);
      const int wr = offs ? (wf + 1 == a.nwin ? 0 : wf + 1) : wf;
      if (jf > 0 && !(wait_window(a, wl, jf) && wait_window(a, wr, jf))) return false;
      const E* ein = static_cast<const E*>((jf & 1) ? a.eout : a.ein);
      RI::warp_copy(s0, ein + (int64_t)wl * (2 * B) + B, B, lane);
      RI::warp_copy(s1, ein + (int64_t)wr * (2 * B), B, lane);
    }
    __syncwarp();
    RI::slot_levels(t, a, s0, s1, lane, cl, fill, empty, a.lev_fill + (int64_t)jf * H, 0);
    __syncwarp();
    if (fill) RI::dump_fill(t, a, lane, cl, a.lev_trap / H + jf, (int64_t)wf * B + (offs ? B / 2 : 0));
    if (empty) {
      const int we = (w0 + ((je + odd0) >> 1) + ie) % nreg;
      E* eout = static_cast<E*>((je & 1) ? const_cast<void*>(a.ein) : a.eout);
      RI::warp_copy(eout + (int64_t)we * (2 * B), s0, B, lane);
      RI::warp_copy(eout + (int64_t)we * (2 * B) + B, s1, B, lane);
      publish_window(a, we, je + 1);
      if (++ie == n) {
        ie = 0;
        ++je;
      }
    }
    __syncwarp();
    if (fill && ++i_f == n) {
      i_f = 0;
      ++jf;
    }
  }
  return true;
}

// Wide window nreg + i through every stage, by one warp.  (A wide window's
// per-window work measured 2.4-2.7 ring slots: one warp per wide window keeps
// it well within a ring run; giving a warp several wide windows to lend the
// freed places to the ring measured slower, and a loop over them cost the
// kernel registers, hence a block per SM.)
template <int ST, class DT, int K, int KW>
__device__ bool stream_uneven_wide(const StageArgs& a, typename DT::E* sm, int nreg, int i) {
  constexpr int H = 32 * K / (2 * Radius<ST>::value);
  const int jw = nreg + i;
  const int odd0 = a.offset != 0;
  for (int j = 0; j < a.nstream; ++j) {
    const int odd = (j + odd0) & 1;
    const int wl = odd ? jw : jw - 1;                          // jw >= nreg >= 1
    const int wr = odd ? (jw + 1 == a.nwin ? 0 : jw + 1) : jw;
    if (j > 0 && !(wait_window(a, wl, j) && wait_window(a, wr, j))) return false;
    StageArgs aj = a;
    aj.ein = (j & 1) ? a.eout : a.ein;
    aj.eout = const_cast<void*>((j & 1) ? a.ein : static_cast<const void*>(a.eout));
    aj.lev_fill = a.lev_fill + (int64_t)j * H;
    aj.lev_trap = a.lev_trap + (int64_t)j * H;
    wide_window<ST, DT, K, KW>(aj, sm, nreg, i, odd);
    publish_window(a, jw, j + 1);
  }
  return true;
}

template <int ST, class DT, int K, int KW>
__global__ void __launch_bounds__(32 * StreamWarps<DT, KW>::value,
                                  StreamWarps<DT, KW>::value == kWarpsPerBlock ? RingBlocks<DT, KW>::value : 1)
swept_stream_wide_kernel(const StageArgs a, int nwarps, int nreg) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using E = typename DT::E;
  constexpr int BW = 32 * KW;
  E* sm = reinterpret_cast<E*>(smem_raw) + (threadIdx.x >> 5) * (2 * BW);
  const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  bool ok = true;
  if (gw < nwarps) ok = stream_uneven_ring<ST, DT, K>(a, sm, gw, nwarps, nreg);
  else if (nreg + (gw - nwarps) < a.nwin) ok = stream_uneven_wide<ST, DT, K, KW>(a, sm, nreg, gw - nwarps);
  if (!ok && (threadIdx.x & 31) == 0) atomicCAS(a.status, 0, SWEPT_ETIMEOUT);
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
  if (a.nstream > 1) {
    // every full diamond in one cooperative launch: every warp resident at once
    cudaError_t e = cudaFuncSetAttribute(swept_stream_wide_kernel<ST, DT, K, KW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, swept_stream_wide_kernel<ST, DT, K, KW>,
                                                      kWarpsPerBlock * 32, smem);
    if (e != cudaSuccess) return e;
    int resident = sms * per_sm * kWarpsPerBlock;
    if (FP64Pipe<DT>::value && resident > 4 * sms) resident = 4 * sms;
    int nwarps = ring > 0 ? ring : resident;
    if (nwarps > nreg / 3) nwarps = nreg / 3;                // runs of at least 3 windows
    if (ring == 0 && nwarps >= sms * kWarpsPerBlock) nwarps -= nwarps % (sms * kWarpsPerBlock);
    if (nwarps < 1) return cudaErrorInvalidValue;
    if (nwarps + nwide > resident) nwarps = resident - nwide;  // one warp per wide window
    if (nwarps < 1) return cudaErrorInvalidValue;
    // every warp of an SM in one block where the kernel allows it (as for swept_stream_kernel)
    const int total = nwarps + nwide;
    int wpb = kWarpsPerBlock;
    if (StreamWarps<DT, KW>::value > kWarpsPerBlock && total % sms == 0 && total / sms > kWarpsPerBlock &&
        total / sms <= StreamWarps<DT, KW>::value)
      wpb = total / sms;
    const size_t smem_b = smem / kWarpsPerBlock * wpb;
    if (wpb != kWarpsPerBlock) {
      e = cudaFuncSetAttribute(swept_stream_wide_kernel<ST, DT, K, KW>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b);
      if (e != cudaSuccess) return e;
    }
    const int grid = (total + wpb - 1) / wpb;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(wpb * 32);
    cfg.dynamicSmemBytes = smem_b;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, swept_stream_wide_kernel<ST, DT, K, KW>, a, nwarps, nreg);
  }
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
