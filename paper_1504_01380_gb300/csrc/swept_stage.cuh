// The swept stage kernel (Section 3): one warp advances one window of
// B = 32*K points whose values live in registers, K consecutive points per
// lane.  Neighbour values inside the window come from the adjacent lanes by
// warp shuffle; the window exchanges only its leading edges, through global
// memory, between launches.
//
// A stage is up to two phases on the same window:
//
//   V-fill (height hv): the window starts from the V formed by the right
//   leading edge of the window on its left and the left leading edge of the
//   window on its right, both written by the previous stage.  Level m
//   (m = 1..hv) computes the gap [B/2 - r m, B/2 + r m) around the window's
//   centre from level m-1: the previous gap plus 2r edge values on each
//   side, placed into the registers that hold those points just before the
//   level.  With hv = h = B/(2r) the gap fills the whole window: a flat level.
//
//   Trapezoid (height ht): from a flat window, level m (m = 1..ht) is
//   computable on [r m, B - r m), the shrinking triangle.  After level m is
//   computed its leading edges are kept: the 2r left-most values
//   [r m, r m + 2r) and the 2r right-most values [B - r m - 2r, B - r m), for
//   m = 0..ht-1 (Section 3: with a 3-point stencil a node sends its two
//   outermost values of each level).  With ht = h the top level is 2r points wide.
//
// Every lane computes all its K points at every level; points outside the
// computable interval get values that nothing reads later (they are either
// overwritten by a placement or never read again).  Placements and captures
// happen at compile-time register offsets: level m = P*(K/r) + j has its
// boundary in lane P (or its mirror) at register r*j + const, so the code for
// the K/r possible j is generated once each and selected by a uniform branch
// tree of depth log2(K/r); the level computation itself is emitted once (an
// unrolled phase of K/r levels overflows the instruction cache for K >= 16).
//
// Layout of one window's edges in global memory (elements of type E):
//   [ L[0][0..2r) L[1][..] ... L[h-1][..] | R[0][0..2r) ... R[h-1][..] ]
// i.e. 2B elements per window, window w at offset w*2B.
#pragma once

#include <type_traits>

#include "swept_internal.h"

namespace swept {

// Kernels that store flat checkpoints when asked (StageArgs::ckpt): the FP64
// KS forward advance, whose states the adjoint's transposed step needs.
template <int ST, class DT> struct DumpsCkpt { static constexpr bool value = false; };
template <> struct DumpsCkpt<kKS, F64> { static constexpr bool value = true; };

template <int ST, class DT, int K>
struct StageImpl {
  using E = typename DT::E;
  using C = typename DT::C;
  static constexpr int R = Radius<ST>::value;
  static constexpr int B = 32 * K;
  static constexpr int H = B / (2 * R);
  static constexpr int L = K / R;      // levels per phase
  static_assert(K % R == 0, "K must be a multiple of the stencil radius");

  // Adjoint sweeps: the forward state at sweep level tau for this lane's K
  // points (window start ws).  Unused (and compiled out) for forward stencils.
  // Runge-Kutta stencils: the sub-timestep of sweep level tau is A when the
  // input level tau - 1 is even, B when it is odd.
  struct Coef {
    double u[K];
    int sub = 0;
  };
  static __device__ __forceinline__ void load_coef(Coef& cf, const StageArgs& a, int64_t ws, int lane,
                                                   int64_t tau) {
    if constexpr (ST == kKSAdj) {
      int64_t g = ws + (int64_t)lane * K;
      if (g >= a.N) g -= a.N;
      const double* lv = tape_level(a, a.tape_len - tau);
      if (g + K <= a.N) {
        ld_chunk<K>(lv + g, cf.u);
      } else {                        // the periodic wrap falls inside this lane's points
#pragma unroll
        for (int k = 0; k < K; ++k) {
          int64_t gk = g + k;
          while (gk >= a.N) gk -= a.N;
          cf.u[k] = lv[gk];
        }
      }
    } else if constexpr (Subs<ST>::value > 1) {
      cf.sub = (int)((tau - 1) & (Subs<ST>::value - 1));
      (void)a; (void)ws; (void)lane;
    } else {
      (void)cf; (void)a; (void)ws; (void)lane; (void)tau;
    }
  }
  // The value a neighbour contributes to the stencil: u (or hi); for the
  // Runge-Kutta pair, u in sub-timestep A and m in B.
  // Euler equations: (q or hi, slopes) for sub-timesteps 0, 1 and (q_mid, slopes) for 2, 3.
  static __device__ __forceinline__ C arg_of(const E& v, int sub) {
    if constexpr (ST == kEuler) {
      return EulerSide<DT>::nb(v, sub);
    } else if constexpr (IsRK2<ST>::value) {
      return sub ? v.y : v.x;
    } else {
      (void)sub;
      return Tile<DT, K>::hi_of(v);
    }
  }

  // Placement for V-fill level mp = P*L + J: left arm at positions
  // 16K - R*mp - 2R + q, right arm at 16K + R*mp + q (level mp values).
  // al / ar: the level's 2r arm values of each side.
  template <int J>
  static __device__ __forceinline__ void place(Tile<DT, K>& t, const E (&al)[2 * R], const E (&ar)[2 * R], int P,
                                               int lane) {
#pragma unroll
    for (int q = 0; q < 2 * R; ++q) {
      const int cc = K - R * J - 2 * R + q;
      const int dl = cc < 0 ? 1 : 0;
      const int k = cc < 0 ? cc + K : cc;
      if (lane == 15 - P - dl) t.put(k, al[q]);
    }
#pragma unroll
    for (int q = 0; q < 2 * R; ++q) {
      const int cc = R * J + q;
      const int dr = cc >= K ? 1 : 0;
      const int k = cc - dr * K;
      if (lane == 16 + P + dr) t.put(k, ar[q]);
    }
  }

  // Capture for trapezoid level m = P*L + J: left edge at positions
  // P*K + R*J + q, right edge (when RIGHT) at (31 - P)*K + K - R*J - 2R + q.
  template <int J, bool RIGHT = true>
  static __device__ __forceinline__ void capture(const Tile<DT, K>& t, E* oL, E* oR, int m, int P,
                                                 int lane) {
#pragma unroll
    for (int q = 0; q < 2 * R; ++q) {
      const int cc = R * J + q;
      const int dl = cc >= K ? 1 : 0;
      const int k = cc - dl * K;
      if (lane == P + dl) oL[m * 2 * R + q] = t.get(k);
    }
    if constexpr (RIGHT) {
#pragma unroll
      for (int q = 0; q < 2 * R; ++q) {
        const int cc = K - R * J - 2 * R + q;
        const int dr = cc < 0 ? 1 : 0;
        const int k = cc + dr * K;
        if (lane == 31 - P - dr) oR[m * 2 * R + q] = t.get(k);
      }
    }
  }

  // Right edge of level m of a trapezoid over `width` points (fewer than the
  // tile's 32K: the last window of a tiling of any N): positions
  // width - r m - 2r + q, whose lane and register are known only at run time.
  static __device__ __forceinline__ void capture_right_at(const Tile<DT, K>& t, E* oR, int m, int width,
                                                          int lane) {
#pragma unroll
    for (int q = 0; q < 2 * R; ++q) {
      const int pos = width - R * m - 2 * R + q;
      const int pl = pos / K;
      const int pk = pos - pl * K;
      E v = t.get(0);
#pragma unroll
      for (int k = 1; k < K; ++k)
        if (pk == k) v = t.get(k);
      if (lane == pl) oR[m * 2 * R + q] = v;
    }
  }

  // Calls f(integral_constant<int, j>) for the runtime j in [LO, HI), with a
  // uniform branch tree.
  template <int LO, int HI, class F>
  static __device__ __forceinline__ void select(int j, F&& f) {
    if constexpr (HI - LO == 1) {
      f(std::integral_constant<int, LO>{});
    } else {
      constexpr int MID = (LO + HI) / 2;
      if (j < MID) select<LO, MID>(j, f);
      else select<MID, HI>(j, f);
    }
  }

  // Levels 1..hv of the V-fill; sL / sR hold the arms (level-major, 2r each).
  static __device__ __forceinline__ void vfill(Tile<DT, K>& t, const E* sL, const E* sR, int hv,
                                               int lane, const StageArgs& a, int64_t ws) {
    const Consts& c = a.c;
    const int hmain = hv < H ? hv : H - 1;
    Coef cf;
    // the arm values of the next level are read one level ahead, off the
    // level's dependence chain (nothing writes the arms during the fill)
    E al[2 * R], ar[2 * R];
#pragma unroll
    for (int q = 0; q < 2 * R; ++q) {
      al[q] = sL[q];
      ar[q] = sR[q];
    }
#pragma unroll 1
    for (int mp = 0; mp < hmain; ++mp) {          // level mp values placed, mp+1 computed
      const int P = mp / L;
      const int j = mp - P * L;
      const int mn = mp + 1 < hv ? mp + 1 : mp;   // inside the hv levels of arms loaded
      E nl[2 * R], nr[2 * R];
#pragma unroll
      for (int q = 0; q < 2 * R; ++q) {
        nl[q] = sL[mn * 2 * R + q];
        nr[q] = sR[mn * 2 * R + q];
      }
      load_coef(cf, a, ws, lane, a.lev_fill + mp + 1);
      select<0, L>(j, [&](auto J) { place<decltype(J)::value>(t, al, ar, P, lane); });
      tile_level<ST, DT, K, false>(t, c, lane, nullptr, nullptr, cf.u, cf.sub);
#pragma unroll
      for (int q = 0; q < 2 * R; ++q) {
        al[q] = nl[q];
        ar[q] = nr[q];
      }
    }
    if (hv == H) {
      // Last level: the arms reach r points beyond the window on each side.
      // Their inner halves go to lanes 0 and 31, their outer halves become
      // the halo of lane 0 (positions -r..-1) and lane 31 (B..B+r-1).
      const int mp = H - 1;
      load_coef(cf, a, ws, lane, a.lev_fill + H);
      C ovl[R], ovr[R];
#pragma unroll
      for (int q = 0; q < R; ++q) {
        ovl[q] = arg_of(sL[mp * 2 * R + q], cf.sub);
        const E vl = sL[mp * 2 * R + R + q];
        if (lane == 0) t.put(q, vl);
        const E vr = sR[mp * 2 * R + q];
        if (lane == 31) t.put(K - R + q, vr);
        ovr[q] = arg_of(sR[mp * 2 * R + R + q], cf.sub);
      }
      tile_level<ST, DT, K, true>(t, c, lane, ovl, ovr, cf.u, cf.sub);
    }
  }

  // Levels 1..ht of the shrinking triangle; edges of levels 0..ht-1 go to
  // oL / oR.  On return the tile holds level ht-1 (the caller computes the
  // top level when ht < h).  GEN: the trapezoid spans `width` points, its
  // right edges found at run time.
  template <bool GEN = false>
  static __device__ __forceinline__ void trapezoid(Tile<DT, K>& t, E* oL, E* oR, int ht, int lane,
                                                   const StageArgs& a, int64_t ws, int width = B) {
    const Consts& c = a.c;
    Coef cf;
#pragma unroll 1
    for (int m = 0; m < ht; ++m) {
      if (m > 0) {
        load_coef(cf, a, ws, lane, a.lev_trap + m);
        tile_level<ST, DT, K, false>(t, c, lane, nullptr, nullptr, cf.u, cf.sub);
      }
      const int P = m / L;
      const int j = m - P * L;
      select<0, L>(j, [&](auto J) { capture<decltype(J)::value, !GEN>(t, oL, oR, m, P, lane); });
      if constexpr (GEN) capture_right_at(t, oR, m, width, lane);
      else (void)width;
    }
  }

  // Copy n elements with the warp in 16-byte units (16-byte aligned; a plain
  // FP32 count is rounded up to 4 elements, which stays inside the B-element slot).
  static __device__ __forceinline__ void warp_copy(E* __restrict__ dst, const E* __restrict__ src,
                                                   int n, int lane) {
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    uint4* d4 = reinterpret_cast<uint4*>(dst);
    const int n16 = (n * (int)sizeof(E) + 15) / 16;   // rounded up: slots hold B elements
    for (int i = lane; i < n16; i += 32) d4[i] = s4[i];
  }

  static __device__ void run(const StageArgs& a, E* sm) {
    const int w = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (w >= (a.nlaunch ? a.nlaunch : a.nwin)) return;     // warp-uniform
    run_window(a, sm, w);
  }

  // The stage on window w (called by one whole warp).
  static __device__ void run_window(const StageArgs& a, E* sm, int w) {
    const int nw = a.nwin;
    const int wl = a.offset ? w : (w == 0 ? nw - 1 : w - 1);
    const int wr = a.offset ? (w + 1 == nw ? 0 : w + 1) : w;
    run_window_at(a, sm, (int64_t)w * B + a.offset, wl, wr, w, B, false);
  }

  // The stage on the window of B points starting at ws (< N): V arms from the
  // right edges of window wl and the left edges of window wr, edges out to
  // window wo's slot; edge slots of 2*eslot elements.  wrap_points: the
  // periodic wrap may fall inside a lane's K points (uneven tiles), so the
  // flat state is loaded point by point.  GEN: a trapezoid of `width` <= B
  // points (the last window of a tiling of any N; the lanes' points past it
  // are loaded but never computable, captured or stored).
  template <bool GEN = false>
  static __device__ void run_window_at(const StageArgs& a, E* sm, int64_t ws, int wl, int wr, int wo, int eslot,
                                       bool wrap_points, int width = B) {
    const int lane = threadIdx.x & 31;
    const int64_t N = a.N;
    E* sL = sm;
    E* sR = sm + B;
    Tile<DT, K> t;
    t.zero();
    if (a.hv == 0) {
      int64_t g = ws + (int64_t)lane * K;
      if (g >= N) g -= N;                        // wrap falls on a lane boundary
      if (!wrap_points || g + K <= N) {
        load_points<K>(t, a.u, N, g);
      } else {
        Tile<DT, 1> one;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          int64_t gk = g + k;
          if (gk >= N) gk -= N;
          load_points<1>(one, a.u, N, gk);
          t.put(k, one.get(0));
        }
      }
      if constexpr (GEN && DumpsCkpt<ST, DT>::value) {
        // the wide window's flat base level (its V part stored the middle,
        // the previous stage its top) is the forward pass's checkpoint when
        // its stage is one; eslot is the regular tile width
        if (double* ck = ckpt_of(a, a.lev_trap / (eslot / (2 * R)))) {
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const int x = lane * K + k;
            if (x < width) {
              int64_t gx = ws + x;
              if (gx >= N) gx -= N;
              ck[gx] = t.get(k);
            }
          }
        }
      }
    } else {
      const E* ein = static_cast<const E*>(a.ein);
      warp_copy(sL, ein + (int64_t)wl * (2 * eslot) + eslot, a.hv * 2 * R, lane);
      warp_copy(sR, ein + (int64_t)wr * (2 * eslot), a.hv * 2 * R, lane);
      __syncwarp();
      vfill(t, sL, sR, a.hv, lane, a, ws);
      __syncwarp();
      if constexpr (DumpsCkpt<ST, DT>::value) {
        // a full fill leaves the window flat: the forward pass's checkpoint
        if (a.hv == H) {
          if (double* ck = ckpt_of(a, a.lev_trap / H)) {
            int64_t g = ws + (int64_t)lane * K;
            if (g >= N) g -= N;
            store_points<K>(t, ck, N, g);
          }
        }
      }
    }
    if (a.ht > 0) {
      trapezoid<GEN>(t, sL, sR, a.ht, lane, a, ws, width);
      __syncwarp();
      E* eout = static_cast<E*>(a.eout) + (int64_t)wo * (2 * eslot);
      warp_copy(eout, sL, a.ht * 2 * R, lane);
      warp_copy(eout + eslot, sR, a.ht * 2 * R, lane);
      if (a.ht < H) {
        // top of the trapezoid: level ht on [r ht, B - r ht)
        Coef cf;
        load_coef(cf, a, ws, lane, a.lev_trap + a.ht);
        tile_level<ST, DT, K, false>(t, a.c, lane, nullptr, nullptr, cf.u, cf.sub);
        const int lo = R * a.ht, hi = (GEN ? width : B) - R * a.ht;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const int x = lane * K + k;
          if (x >= lo && x < hi) {
            int64_t g = ws + x;
            if (g >= N) g -= N;
            store_point<K>(t, k, a.u, N, g);
          }
        }
      }
    } else if (a.hv == H) {
      int64_t g = ws + (int64_t)lane * K;
      if (g >= N) g -= N;
      store_points<K>(t, a.u, N, g);
    } else {
      // partial V-fill: its gap [B/2 - r hv, B/2 + r hv) is at level hv
      const int lo = B / 2 - R * a.hv, hi = B / 2 + R * a.hv;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int x = lane * K + k;
        if (x >= lo && x < hi) {
          int64_t g = ws + x;
          if (g >= N) g -= N;
          store_point<K>(t, k, a.u, N, g);
        }
      }
    }
  }
};

// Small tiles (K <= 4) serve the latency regime, where a stage has a warp per
// window and few warps per SM: declaring one block per SM frees the register
// allocator (88 registers at K = 1 instead of 40 with spills), which shortens
// each level's dependence chain.  Together with reading the V-fill's arm
// values a level ahead, measured on GB300 (heat, N = 1024, per sub-timestep):
// compensated 258 -> 210 ns, FP64 417 -> 374 ns.  Larger tiles keep the
// default, which holds more warps per SM.
template <int K> struct StageBlocks { static constexpr int value = K <= 4 ? 1 : 0; };

template <int ST, class DT, int K>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, StageBlocks<K>::value)
swept_stage_kernel(const StageArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using E = typename DT::E;
  constexpr int B = 32 * K;
  griddep_wait();
  E* sm = reinterpret_cast<E*>(smem_raw) + (threadIdx.x >> 5) * (2 * B);
  StageImpl<ST, DT, K>::run(a, sm);
}

template <int ST, class DT, int K>
cudaError_t launch_stage_k(const StageArgs& a, cudaStream_t s) {
  constexpr int B = 32 * K;
  const size_t smem = stage_smem_bytes(B, (int)sizeof(typename DT::E));
  // set on every launch: the attribute belongs to the current device
  cudaError_t e = cudaFuncSetAttribute(swept_stage_kernel<ST, DT, K>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = ((a.nlaunch ? a.nlaunch : a.nwin) + kWarpsPerBlock - 1) / kWarpsPerBlock;
  return launch_kernel(a.pdl != 0, swept_stage_kernel<ST, DT, K>, dim3(grid), dim3(kWarpsPerBlock * 32), smem, s,
                       a);
}

template <int ST, class DT>
cudaError_t launch_stage_dispatch(int K, const StageArgs& a, cudaStream_t s) {
  switch (K) {
    case 1:
      if constexpr (Radius<ST>::value == 1) return launch_stage_k<ST, DT, 1>(a, s);
      else return cudaErrorInvalidValue;
    case 2: return launch_stage_k<ST, DT, 2>(a, s);
    case 4: return launch_stage_k<ST, DT, 4>(a, s);
    case 8: return launch_stage_k<ST, DT, 8>(a, s);
    case 16: return launch_stage_k<ST, DT, 16>(a, s);
    case 32: return launch_stage_k<ST, DT, 32>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace swept
