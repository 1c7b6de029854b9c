// Ring-pipelined diamond stage (Section 3's diamonds, computed two at a time).
//
// The per-window stage kernel leaves half of its lanes idle: a diamond is a
// V-fill whose computable gap grows by r points per side per level and then a
// triangle that shrinks by r per side, inside a rectangle of B points by 2h
// levels.  Here one warp streams a run of consecutive windows of one stage and
// overlaps the V-fill of window w+1 with the triangle of window w: at level m
// the fill covers 2rm points and the triangle B - 2rm, so together they keep
// every lane busy.
//
// Layout: a register ring of M = 32*S slots, S = K + r per lane, lanes in a
// ring (lane 31's right neighbour is lane 0).  The window being filled sits
// at ring offset c (0 or M/2), the window being emptied at c + M/2; the two
// regions are separated by two gaps of 16r slots.  Each level:
//   1. the V's arm values of the previous level (2r per side, from the
//      previous stage's edges, staged in shared memory at the slot's start)
//      are read, and the triangle's leading edges of the previous level (2r
//      values on each side, adjacent to the gaps) are captured into the same
//      shared-memory slots, which are free once read;
//   2. the arm values are placed into the gaps, where the fill's boundary
//      points read them;
//   3. all M slots are advanced one level.
// At the end of the slot the captured edges go to global memory in one
// coalesced copy.  (Streaming the arms in small cp.async chunks and storing
// captures straight to global memory cuts shared memory to 2 KB per warp, but
// measured 6% slower at K = 32, where registers bind the occupancy anyway.)
// After h levels the filled window is flat and becomes the window being
// emptied in the next slot (same offset), and the next window is filled at
// the other offset.  A run of n windows takes n + 1 slots; the first slot
// only fills and the last only empties.  The streamed form (run_stream,
// swept_stream_kernel) runs every full diamond stage of an advance in one
// launch and joins each stage's last slot to the next stage's first, so a
// run costs n slots per stage.
//
// Every boundary position is r*(level) plus a constant, so with levels in
// phases of S/r the boundary stays in one lane and moves r registers per
// level; the register offsets are compile-time, selected by a uniform branch
// tree as in the per-window kernel (a switch for the compensated KS ring up to
// K = 16, measured faster there).  The values computed are exactly those
// of the per-window kernel (same expression per point, only the order of
// independent updates changes), so results are bit-identical.
#pragma once

#include <type_traits>

#include "swept.h"
#include "swept_internal.h"
#include "swept_stage.cuh"
#include "swept_sync.cuh"

namespace swept {

// How a level's phase step J reaches its compile-time register offsets: a
// binary tree of uniform branches (default) or one switch.  Measured on
// GB300: for the compensated KS ring the switch is faster at K = 16 (N = 2^22,
// B = 512: 1.141 against 1.121e12 cell-updates/s) and the tree at K = 32
// (B = 1024: 1.344 against 1.304e12); the switch is 9% slower for the
// compensated heat ring (N = 2^24); FP64 KS and the compensated Euler
// equations differ by under 1%.
template <int ST, class DT, int K> struct SwitchSelect { static constexpr bool value = false; };
template <int K> struct SwitchSelect<kKS, F32C, K> { static constexpr bool value = K <= 16; };

template <int ST, class DT, int K>
struct RingImpl {
  using E = typename DT::E;
  using C = typename DT::C;
  static constexpr int R = Radius<ST>::value;
  static constexpr int B = 32 * K;          // window width
  static constexpr int S = K + R;           // ring slots per lane
  static constexpr int H = B / (2 * R);     // levels per slot
  static constexpr int L = S / R;           // levels per phase
  static_assert(K % R == 0, "K must be a multiple of the stencil radius");

  // Compile-time parts of the four boundary positions for phase step J.
  //   shrink left edge : p = c + M/2 + R*mp + q           = c + XSL + P*S
  //   shrink right edge: p = c + M/2 + B - R*mp - 2R + q  = c + XSR - P*S
  //   fill left arm    : p = c + B/2 - R*mp - 2R + q      = c + XGL - P*S
  //   fill right arm   : p = c + B/2 + R*mp + q           = c + XGR + P*S
  // with R*mp = P*S + R*J and M/2 = 16S, B = 32K.
  template <int J, int Q> struct Pos {
    static constexpr int XSL = R * J + Q + 16 * S;
    static constexpr int XSR = 48 * S - 34 * R - R * J + Q;
    static constexpr int XGL = 16 * S - 18 * R - R * J + Q;
    static constexpr int XGR = 16 * S - 16 * R + R * J + Q;
  };

  // Lane tests.  A position X (relative to the filled window's start) moving
  // +P lanes per phase is in lane (cl + X/S + P) mod 32, i.e. in the lane
  // whose (lane - cl - P) mod 32 is (X/S) mod 32; one moving -P lanes, in the
  // lane whose (lane - cl + P) mod 32 is.  The run keeps those two residues
  // per phase, set to -1 (no lane) in slots that do not capture (first slot)
  // or do not place (last slot), so each test is one compare with a constant.
  struct Lanes {
    int cap_p, cap_m;   // captures: shrink-left edge (+P), shrink-right edge (-P)
    int put_p, put_m;   // placements: fill-right arm (+P), fill-left arm (-P)
  };
  template <int J, int Q>
  static __device__ __forceinline__ void capture_q(const Tile<DT, S>& t, E* sOL, E* sOR, const Lanes& ln) {
    using Ps = Pos<J, Q>;
    if (ln.cap_p == (Ps::XSL / S) % 32) sOL[Q] = t.get(Ps::XSL % S);
    if (ln.cap_m == (Ps::XSR / S) % 32) sOR[Q] = t.get(Ps::XSR % S);
  }
  template <int J, int Q>
  static __device__ __forceinline__ void place_q(Tile<DT, S>& t, const E (&al)[2 * R], const E (&ar)[2 * R],
                                                 const Lanes& ln) {
    using Ps = Pos<J, Q>;
    if (ln.put_m == (Ps::XGL / S) % 32) t.put(Ps::XGL % S, al[Q]);
    if (ln.put_p == (Ps::XGR / S) % 32) t.put(Ps::XGR % S, ar[Q]);
  }
  template <int J, int... Qs>
  static __device__ __forceinline__ void capture_all(const Tile<DT, S>& t, E* sOL, E* sOR, const Lanes& ln,
                                                     std::integer_sequence<int, Qs...>) {
    (capture_q<J, Qs>(t, sOL, sOR, ln), ...);
  }
  template <int J, int... Qs>
  static __device__ __forceinline__ void place_all(Tile<DT, S>& t, const E (&al)[2 * R], const E (&ar)[2 * R],
                                                   const Lanes& ln, std::integer_sequence<int, Qs...>) {
    (place_q<J, Qs>(t, al, ar, ln), ...);
  }
  static __device__ __forceinline__ Lanes lanes_of(int rel, int P, bool fill, bool empty) {
    const int rp = (rel - P) & 31, rm = (rel + P) & 31;
    return Lanes{empty ? rp : -1, empty ? rm : -1, fill ? rp : -1, fill ? rm : -1};
  }

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
  // The same dispatch as one switch over J (L <= K/R + 1 <= 33 cases).
  template <class F>
  static __device__ __forceinline__ void select_switch(int j, F&& f) {
    static_assert(L <= 33, "at most 33 phase steps");
#define SWEPT_J(n) \
  case n:          \
    if constexpr (n < L) f(std::integral_constant<int, n>{}); \
    break;
    switch (j) {
      SWEPT_J(0) SWEPT_J(1) SWEPT_J(2) SWEPT_J(3) SWEPT_J(4) SWEPT_J(5) SWEPT_J(6) SWEPT_J(7) SWEPT_J(8)
      SWEPT_J(9) SWEPT_J(10) SWEPT_J(11) SWEPT_J(12) SWEPT_J(13) SWEPT_J(14) SWEPT_J(15) SWEPT_J(16)
      SWEPT_J(17) SWEPT_J(18) SWEPT_J(19) SWEPT_J(20) SWEPT_J(21) SWEPT_J(22) SWEPT_J(23) SWEPT_J(24)
      SWEPT_J(25) SWEPT_J(26) SWEPT_J(27) SWEPT_J(28) SWEPT_J(29) SWEPT_J(30) SWEPT_J(31) SWEPT_J(32)
      default: break;
    }
#undef SWEPT_J
  }
  template <class F>
  static __device__ __forceinline__ void select_j(int j, F&& f) {
    if constexpr (SwitchSelect<ST, DT, K>::value) select_switch(j, f);
    else select<0, L>(j, f);
  }

  static __device__ __forceinline__ void warp_copy(E* __restrict__ dst, const E* __restrict__ src, int n,
                                                   int lane) {
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    uint4* d4 = reinterpret_cast<uint4*>(dst);
    const int n16 = (n * (int)sizeof(E) + 15) / 16;   // rounded up: slots hold B elements
    for (int i = lane; i < n16; i += 32) d4[i] = s4[i];
  }

  // Adjoint sweeps: the forward state (the coefficient of the transposed step)
  // at each of this lane's S ring slots for the level being computed
  // (mp + 1 of the slot).  Ring position p (relative to the fill window's
  // start c) is fill-window point p, computed on the V [B/2 - r(mp+1),
  // B/2 + r(mp+1)), and emptied-window point p - M/2 (mod M), computed on
  // [r(mp+1), B - r(mp+1)); the two are disjoint at every level.  Slots
  // outside both get 0 (their values are never read).  Sweep level tau uses
  // forward level tape_len - tau.
  static __device__ __forceinline__ void adjoint_coef(double (&cf)[S], const StageArgs& a, int lane, int cl,
                                                      int wfill, bool fill, bool empty, int mp) {
    constexpr int M = 32 * S;
    const int lo_f = B / 2 - R * (mp + 1), hi_f = B / 2 + R * (mp + 1);
    const int lo_t = R * (mp + 1), hi_t = B - R * (mp + 1);
    const double* rf = tape_level(a, a.tape_len - (a.lev_fill + mp + 1));
    const double* rt = tape_level(a, a.tape_len - (a.lev_trap + mp + 1));
    const int64_t wsf = (int64_t)wfill * B + a.offset;
    const int64_t wst = wsf - B;                       // the emptied window is wfill - 1
#pragma unroll
    for (int k = 0; k < S; ++k) {
      const int p = (((lane - cl) & 31) * S + k) % M;
      const int xt = (p + M / 2) % M;
      double v = 0.0;
      if (fill && p >= lo_f && p < hi_f) {
        int64_t g = wsf + p;
        if (g >= a.N) g -= a.N;
        v = rf[g];
      } else if (empty && xt >= lo_t && xt < hi_t) {
        int64_t g = wst + xt;
        if (g < 0) g += a.N;
        if (g >= a.N) g -= a.N;
        v = rt[g];
      }
      cf[k] = v;
    }
  }

  // After a slot, the filled window sits flat at ring positions [0, B) from
  // the fill offset: ring position p = ((lane - cl) mod 32) * S + k is window
  // point p.  Store it as the forward pass's checkpoint when its stage k is
  // one (StageArgs::ckpt); ws is the window's first global point.
  static __device__ __forceinline__ void dump_fill(const Tile<DT, S>& t, const StageArgs& a, int lane, int cl,
                                                   int64_t k, int64_t ws) {
    if constexpr (DumpsCkpt<ST, DT>::value) {
      double* ck = ckpt_of(a, k);
      if (!ck) return;
      const int rel = (lane - cl) & 31;
#pragma unroll
      for (int j = 0; j < S; ++j) {
        const int p = rel * S + j;
        if (p < B) {
          int64_t g = ws + p;
          if (g >= a.N) g -= a.N;
          ck[g] = t.get(j);
        }
      }
    } else {
      (void)t; (void)a; (void)lane; (void)cl; (void)k; (void)ws;
    }
  }

  // Hooks of a run without dependences (one stage per launch).
  struct NoHooks {
    __device__ __forceinline__ bool ready(int) const { return true; }
    __device__ __forceinline__ void done(int) const {}
  };

  // The h levels of one slot: the window being filled sits at ring offset
  // cl lanes, the one being emptied at cl + 16.  s0/s1 hold the fill's arms
  // on entry and the emptied window's captured edges on return.  `lev` is the
  // absolute level of the fill's first computed level (only its value modulo
  // Subs matters: h is a multiple of Subs, so both windows of the ring are at
  // the same sub-timestep); `wfill` the filled window (adjoint sweeps).
  static __device__ __forceinline__ void slot_levels(Tile<DT, S>& t, const StageArgs& a, E* s0, E* s1, int lane,
                                                     int cl, bool fill, bool empty, int64_t lev, int wfill) {
    int P = 0, j = 0;
    const int rel = (lane - cl) & 31;
    Lanes ln = lanes_of(rel, 0, fill, empty);
#pragma unroll 1
    for (int mp = 0; mp < H; ++mp) {
      E al[2 * R], ar[2 * R];
#pragma unroll
      for (int q = 0; q < 2 * R; ++q) {
        al[q] = s0[mp * 2 * R + q];
        ar[q] = s1[mp * 2 * R + q];
      }
      __syncwarp();
      // (the emptied window sits at offset cl + M/2: the XS* constants include M/2)
      E* const cL = s0 + mp * 2 * R;
      E* const cR = s1 + mp * 2 * R;
      select_j(j, [&](auto JJ) {
        constexpr int J = decltype(JJ)::value;
        capture_all<J>(t, cL, cR, ln, std::make_integer_sequence<int, 2 * R>{});
        place_all<J>(t, al, ar, ln, std::make_integer_sequence<int, 2 * R>{});
      });
      if constexpr (ST == kKSAdj) {
        double cf[S];
        adjoint_coef(cf, a, lane, cl, wfill, fill, empty, mp);
        tile_level<ST, DT, S, false>(t, a.c, lane, nullptr, nullptr, cf, 0);
      } else {
        (void)wfill;
        tile_level<ST, DT, S, false>(t, a.c, lane, nullptr, nullptr, nullptr,
                                     (int)((lev + mp) & (Subs<ST>::value - 1)));
      }
      if (++j == L) {
        j = 0;
        ++P;
        ln = lanes_of(rel, P, fill, empty);
      }
    }
  }

  // One warp: windows [w0, w1) of a full diamond stage (hv = ht = h).
  // sm: 2B elements of shared memory.
  static __device__ void run(const StageArgs& a, E* sm, int w0, int w1) {
    run_hooked(a, sm, w0, w1, NoHooks{});
  }

  // As run(), with hooks for runs whose inputs are produced concurrently:
  // hk.ready(w) is called (by the whole warp) before any arm value of window
  // w is read and returns false when the wait for it gave up; hk.done(w) is
  // called after window w's edges are stored.  Returns false if a wait gave up.
  template <class Hooks>
  static __device__ bool run_hooked(const StageArgs& a, E* sm, int w0, int w1, const Hooks& hk) {
    const int lane = threadIdx.x & 31;
    const E* ein = static_cast<const E*>(a.ein);
    E* eout = static_cast<E*>(a.eout);
    // sm[0, B): fill's left arm in, then the emptied window's left edges out;
    // sm[B, 2B): fill's right arm in, then right edges out.
    E* s0 = sm;
    E* s1 = sm + B;
    Tile<DT, S> t;
    t.zero();
    const int nrun = w1 - w0;
    for (int slot = 0; slot <= nrun; ++slot) {
      const bool fill = slot < nrun;
      const bool empty = slot > 0;
      const int cl = (slot & 1) ? 16 : 0;          // ring offset of the filled window, in lanes
      if (fill) {
        const int w = w0 + slot;
        if (!hk.ready(w)) return false;
        const int wl = a.offset ? w : (w == 0 ? a.nwin - 1 : w - 1);
        const int wr = a.offset ? (w + 1 == a.nwin ? 0 : w + 1) : w;
        warp_copy(s0, ein + (int64_t)wl * (2 * B) + B, B, lane);
        warp_copy(s1, ein + (int64_t)wr * (2 * B), B, lane);
      }
      __syncwarp();
      slot_levels(t, a, s0, s1, lane, cl, fill, empty, a.lev_fill, w0 + slot);
      __syncwarp();
      if (fill) dump_fill(t, a, lane, cl, a.lev_trap / H, (int64_t)(w0 + slot) * B + a.offset);
      if (empty) {
        const int ws = w0 + slot - 1;
        warp_copy(eout + (int64_t)ws * (2 * B), s0, B, lane);
        warp_copy(eout + (int64_t)ws * (2 * B) + B, s1, B, lane);
        hk.done(ws);
      }
      __syncwarp();
    }
    return true;
  }

  // Stages k0 .. k0 + a.nstream - 1 (all full diamonds) streamed by one warp
  // (warp g of nwarps) in one launch: the slot that empties a stage's last
  // window fills the next stage's first, so a run of n windows costs n slots
  // per stage instead of n + 1 (the first slot of a run only fills and the
  // last only empties).
  //
  // Window ownership drifts: at stage k0 + j the warp runs windows
  // w0 + d(j) .. w1 - 1 + d(j) (mod nwin), d(j) = (j + [k0 odd]) / 2, i.e.
  // one window to the right at every step from an offset stage to an
  // unshifted one.  Window w of an offset stage reads windows w and w + 1 of
  // the previous stage, of an unshifted stage windows w - 1 and w; with the
  // drift, every window of the warp reads windows of its own run of the
  // previous stage, except the last, which also reads the first window of
  // warp g + 1's run.  So the first window of a stage reads two windows that
  // were emptied in earlier slots (n >= 3), and the one cross-warp input is
  // waited for on warp g + 1's slot counter (a bounded wait).
  //
  // Edge buffers: stage k0 + j reads a.ein when j is even (else a.eout) and
  // writes the other.  A stage's edges overwrite those of two stages back,
  // read by the stage in between; its readers are this warp's own earlier
  // fills and warp g + 1's first fill of that stage, which the same wait has
  // seen finished; warp g - 1 reads only windows left of this warp's range at
  // every stage (the drift moves the range right), whatever its lag.
  //
  // With a.nstream <= 1 this is the one-stage run of run() (d = 0, no wait).
  // Returns false if a wait gave up (the status word then holds
  // SWEPT_ETIMEOUT).
  static __device__ bool run_stream(const StageArgs& a, E* sm, int g, int nwarps) {
    const int lane = threadIdx.x & 31;
    const int nw = a.nlaunch ? a.nlaunch : a.nwin;   // windows run (uneven tiles: the regular ones)
    const int w0 = (int)(((int64_t)g * nw) / nwarps);
    const int n = (int)(((int64_t)(g + 1) * nw) / nwarps) - w0;
    if (n <= 0) return true;
    const int nst = a.nstream > 1 ? a.nstream : 1;
    const int gr = g + 1 == nwarps ? 0 : g + 1;      // the right neighbour's run length
    const int nr = (int)(((int64_t)(gr + 1) * nw) / nwarps - ((int64_t)gr * nw) / nwarps);
    const int odd0 = a.offset != 0;
    E* s0 = sm;
    E* s1 = sm + B;
    Tile<DT, S> t;
    t.zero();
    const int T = nst * n;                           // windows streamed
    int jf = 0, i_f = 0;                             // next window to fill: stage k0 + jf, run index i_f
    int je = 0, ie = 0;                              // window being emptied
    for (int slot = 0; slot <= T; ++slot) {
      const bool fill = slot < T;
      const bool empty = slot > 0;
      const int cl = (slot & 1) ? 16 : 0;
      if (fill) {
        if (i_f == n - 1 && jf > 0) {
          // warp gr's first window of stage k0 + jf - 1 is emptied in its slot
          // (jf - 1) * nr + 1: wait until its counter has passed that slot
          const int target = (jf - 1) * nr + 2;
          const long long t0 = clock64();
          bool ok = true;
          for (int it = 0;; ++it) {
            if (ld_relaxed(a.progress + gr) >= target) break;
            if ((it & 63) == 63 && (clock64() - t0 > a.budget || ld_relaxed(a.status) != 0)) {
              ok = false;
              break;
            }
            __nanosleep(128);
          }
          fence_acq_rel();
          if (!__all_sync(kFull, ok)) {
            if (lane == 0) atomicCAS(a.status, 0, SWEPT_ETIMEOUT);
            return false;
          }
        }
        const bool offs = ((jf + odd0) & 1) != 0;
        const int w = (w0 + ((jf + odd0) >> 1) + i_f) % a.nwin;
        const int wl = offs ? w : (w == 0 ? a.nwin - 1 : w - 1);
        const int wr = offs ? (w + 1 == a.nwin ? 0 : w + 1) : w;
        const E* ein = static_cast<const E*>((jf & 1) ? a.eout : a.ein);
        warp_copy(s0, ein + (int64_t)wl * (2 * B) + B, B, lane);
        warp_copy(s1, ein + (int64_t)wr * (2 * B), B, lane);
      }
      __syncwarp();
      slot_levels(t, a, s0, s1, lane, cl, fill, empty, a.lev_fill + (int64_t)jf * H, 0);
      __syncwarp();
      if (fill) {
        const bool offs = ((jf + odd0) & 1) != 0;
        const int w = (w0 + ((jf + odd0) >> 1) + i_f) % a.nwin;
        dump_fill(t, a, lane, cl, a.lev_trap / H + jf, (int64_t)w * B + (offs ? B / 2 : 0));
      }
      if (empty) {
        const int w = (w0 + ((je + odd0) >> 1) + ie) % a.nwin;
        E* eout = static_cast<E*>((je & 1) ? const_cast<void*>(a.ein) : a.eout);
        warp_copy(eout + (int64_t)w * (2 * B), s0, B, lane);
        warp_copy(eout + (int64_t)w * (2 * B) + B, s1, B, lane);
        if (++ie == n) {
          ie = 0;
          ++je;
        }
      }
      __syncwarp();
      if (nst > 1 && lane == 0 && g != a.drop) {
        __threadfence();
        st_release(a.progress + g, slot + 1);
      }
      if (fill && ++i_f == n) {
        i_f = 0;
        ++jf;
      }
    }
    return true;
  }
};

// Shared memory of the ring kernel per block: 2B elements per warp.
template <int ST, class DT, int K>
size_t ring_smem_bytes() {
  return stage_smem_bytes(32 * K, (int)sizeof(typename DT::E));
}

// Blocks per SM that the ring's shared memory admits (2B edge elements per
// warp; 228 KB per SM, 1 KB of it reserved per block), at most 16 (64 warps).
// Declared as the kernels' minimum blocks per SM, it tells the register
// allocator the budget it may use without lowering that occupancy
// (65536 / (blocks x 128) registers per thread).
template <class DT, int K> struct RingBlocks {
  static constexpr int smem = kWarpsPerBlock * 2 * 32 * K * (int)sizeof(typename DT::E);
  static constexpr int by_smem = (228 * 1024) / (smem + 1024);
  static constexpr int value = by_smem <= 4 ? (by_smem < 1 ? 1 : by_smem) : 0;
};

template <int ST, class DT, int K>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, RingBlocks<DT, K>::value)
swept_ring_kernel(const StageArgs a, int nwarps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using E = typename DT::E;
  griddep_wait();
  E* sm = reinterpret_cast<E*>(smem_raw) + (threadIdx.x >> 5) * (2 * 32 * K);
  const int gw = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (gw >= nwarps) return;
  // balanced contiguous runs: warp gw takes [gw*n/W, (gw+1)*n/W)
  const int nw = a.nlaunch ? a.nlaunch : a.nwin;    // windows run (uneven tiles: the regular ones)
  const int w0 = (int)(((int64_t)gw * nw) / nwarps);
  const int w1 = (int)(((int64_t)(gw + 1) * nw) / nwarps);
  if (w1 > w0) RingImpl<ST, DT, K>::run(a, sm, w0, w1);
}

// Warps per block of the streamed kernel: every warp an SM holds in one block
// where the shared memory bounds the SM at two to four blocks of four warps
// (the register budget the launch bounds give is then the same as with blocks
// of four); else blocks of four warps.  Measured on GB300: KS, compensated
// FP32, N = 2^22, B = 1024, 1216 warps, two blocks of four per SM: one block
// of eight warps per SM 1.44e12 cell-updates/s against 1.34e12, bit for bit
// the same; the Euler equations, compensated, N = 2^23, B = 128, four blocks
// of four: one block of sixteen 2.72e10 cell-steps/s against 2.61e10; heat
// (three blocks of four, or one of twelve) within 0.3%.  Neither the kernel's
// registers nor the placement of the blocks on the SMs (pinned to two per SM
// by padding their shared memory) made the difference.
template <class DT, int K> struct StreamWarps {
  static constexpr int value =
      RingBlocks<DT, K>::value >= 2 ? kWarpsPerBlock * RingBlocks<DT, K>::value : kWarpsPerBlock;
};

// Several full-diamond stages in one launch (RingImpl::run_stream); a kernel
// of its own so that the one-stage kernel keeps its register budget.
template <int ST, class DT, int K>
__global__ void __launch_bounds__(32 * StreamWarps<DT, K>::value,
                                  StreamWarps<DT, K>::value == kWarpsPerBlock ? RingBlocks<DT, K>::value : 1)
swept_stream_kernel(const StageArgs a, int nwarps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using E = typename DT::E;
  E* sm = reinterpret_cast<E*>(smem_raw) + (threadIdx.x >> 5) * (2 * 32 * K);
  const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (gw >= nwarps) return;
  RingImpl<ST, DT, K>::run_stream(a, sm, gw, nwarps);
}

// Launch with `nwarps` warps; 0 picks min(resident warp slots of the GPU,
// nwin / 2), so that every warp streams at least two windows when it can,
// and for the scalar stencils' FP64 states at most one warp per scheduler
// (4 per SM).
// nwarps < 0 is the automatic choice of kernel.  With at most one window per
// scheduler (nwin <= 4 x SMs) every warp runs alone on its scheduler and the
// stage time is one warp's chain of levels: the per-window kernel (2h levels)
// finishes sooner than ring runs of two windows (3h levels), so that kernel
// is launched instead.  With more windows the pipes are shared and total work
// decides: the ring computes (n+1) h (K+r) slot-levels per n windows against
// 2h K for the per-window kernel, so the ring runs (as for 0).
// FP64 states of the scalar stencils run on GB300's narrow FP64 pipe: one
// warp per scheduler already keeps it busy, and fewer, longer ring runs waste
// fewer fill and drain slots.  Not the Euler equations' FP64 state: its face
// flux is a long chain through divisions and square roots that one warp per
// scheduler leaves the pipe waiting on (measured on GB300, N = 2^23, B = 64:
// 8.5e8 cell-steps/s with one block per SM, 9.4e8 with three).
template <class DT> struct FP64Pipe { static constexpr bool value = false; };
template <> struct FP64Pipe<F64> { static constexpr bool value = true; };
template <> struct FP64Pipe<F64P> { static constexpr bool value = true; };

template <int ST, class DT, int K>
cudaError_t launch_ring_k(const StageArgs& a, int nwarps, cudaStream_t s) {
  const size_t smem = ring_smem_bytes<ST, DT, K>();
  const int nw = a.nlaunch ? a.nlaunch : a.nwin;     // windows run
  cudaError_t e = cudaFuncSetAttribute(swept_ring_kernel<ST, DT, K>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if constexpr (ST != kKSAdj) {
  if (a.nstream > 1) {
    // streamed stages: the warps wait on one another, so every warp must be
    // resident at once (a cooperative launch), with at least 3 windows each
    e = cudaFuncSetAttribute(swept_stream_kernel<ST, DT, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0, per_sm_ring = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, swept_stream_kernel<ST, DT, K>,
                                                      kWarpsPerBlock * 32, smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_ring, swept_ring_kernel<ST, DT, K>,
                                                        kWarpsPerBlock * 32, smem);
    if (e != cudaSuccess) return e;
    int resident = sms * per_sm * kWarpsPerBlock;
    if (FP64Pipe<DT>::value) {                       // one block per SM either way
      if (resident > 4 * sms) resident = 4 * sms;
      per_sm = per_sm_ring = 1;
    }
    const bool automatic = nwarps <= 0;
    if (nwarps <= 0 || nwarps > resident) nwarps = resident;
    if (nwarps > nw / 3) nwarps = nw / 3;
    if (automatic && nwarps >= sms * kWarpsPerBlock) {
      // Every SM gets the same number of blocks.  The warps wait on their
      // neighbours once per stage, so the launch runs at the pace of its most
      // crowded SM: measured on GB300 (KS, compensated FP32, N = 2^22,
      // B = 1024, at most 3 blocks per SM), 1365 warps (342 blocks: some SMs
      // 3, some 2) 1.05e12 cell-updates/s, 912 warps (1.5 blocks per SM)
      // 1.05e12, 1216 warps (2 per SM) 1.30e12.
      nwarps -= nwarps % (sms * kWarpsPerBlock);
    }
    if (nwarps < 1 || a.nlaunch) return cudaErrorInvalidValue;
    if (a.stream_query) {
      // Streaming saves each run's extra slot per stage, 1/n of the work for
      // runs of n windows, and its kernel may hold fewer blocks per SM than
      // the one-stage kernel (it keeps more registers).  Measured on GB300
      // (heat, compensated FP32, N = 2^24): 7-11% faster for runs of 8-12
      // windows; 5-9% slower for runs of 18-27 windows that cost residency.
      const int n = (nw + nwarps - 1) / nwarps;
      return (n <= 16 || per_sm >= per_sm_ring) ? cudaSuccess : cudaErrorNotSupported;
    }
    // one block per SM where the kernel allows it and every SM holds the same number of warps
    int wpb = kWarpsPerBlock;
    if (StreamWarps<DT, K>::value > kWarpsPerBlock && nwarps % sms == 0 && nwarps / sms > kWarpsPerBlock &&
        nwarps / sms <= StreamWarps<DT, K>::value)
      wpb = nwarps / sms;
    const size_t smem_b = smem / kWarpsPerBlock * wpb;
    if (wpb != kWarpsPerBlock) {
      e = cudaFuncSetAttribute(swept_stream_kernel<ST, DT, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem_b);
      if (e != cudaSuccess) return e;
    }
    const int grid = (nwarps + wpb - 1) / wpb;
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
    return cudaLaunchKernelEx(&cfg, swept_stream_kernel<ST, DT, K>, a, nwarps);
  }
  }
  if (nwarps <= 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, swept_ring_kernel<ST, DT, K>,
                                                      kWarpsPerBlock * 32, smem);
    if (e != cudaSuccess) return e;
    const int resident = sms * (per_sm > 0 ? per_sm : 1) * kWarpsPerBlock;
    if (nwarps < 0 && nw <= 4 * sms) return launch_stage_k<ST, DT, K>(a, s);
    nwarps = resident;
    // (the adjoint sweep also waits on its tape loads every level: two warps per scheduler)
    const int cap = (ST == kKSAdj ? 8 : 4) * sms;
    if (FP64Pipe<DT>::value && nwarps > cap) nwarps = cap;
    if (nwarps > nw / 2) nwarps = nw / 2;
    if (nwarps < 1) nwarps = 1;
  }
  if (nwarps > nw) nwarps = nw;
  const int grid = (nwarps + kWarpsPerBlock - 1) / kWarpsPerBlock;
  return launch_kernel(a.pdl != 0, swept_ring_kernel<ST, DT, K>, dim3(grid), dim3(kWarpsPerBlock * 32), smem, s,
                       a, nwarps);
}

template <int ST, class DT>
cudaError_t launch_ring_dispatch(int K, const StageArgs& a, int nwarps, cudaStream_t s) {
  switch (K) {
    case 1:
      if constexpr (Radius<ST>::value == 1) return launch_ring_k<ST, DT, 1>(a, nwarps, s);
      else return cudaErrorInvalidValue;
    case 2: return launch_ring_k<ST, DT, 2>(a, nwarps, s);
    case 4: return launch_ring_k<ST, DT, 4>(a, nwarps, s);
    case 8: return launch_ring_k<ST, DT, 8>(a, nwarps, s);
    case 16: return launch_ring_k<ST, DT, 16>(a, nwarps, s);
    case 32: return launch_ring_k<ST, DT, 32>(a, nwarps, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace swept
