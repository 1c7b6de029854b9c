// Host-side declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <initializer_list>
#include <cuda_runtime.h>

#include "swept_device.cuh"

namespace swept {

// Warps per thread block of the stage kernels.  One warp owns one window.
constexpr int kWarpsPerBlock = 4;

// Where a call runs.  Every device pointer an entry point takes must be
// memory of the current CUDA device (or managed memory), the stream must
// belong to that device, and a plan must have been made on it: a kernel
// launched on one GPU with another GPU's pointer faults.  `plan_dev` < 0
// means "no plan".  Checked before anything is enqueued; a failed query
// leaves no sticky error.  (A stream whose device cannot be queried is
// accepted: the launch itself then reports a foreign stream.)  While `s` is
// being captured into a CUDA graph the pointer and stream queries would end
// the capture, so only the plan's device is checked then; otherwise the
// queries run in relaxed capture mode, so that they cannot disturb a
// capture another thread has open.
inline bool pointer_on_device(const void* p, int dev) {
  if (!p) return true;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}
inline bool call_on_device(int plan_dev, cudaStream_t s, std::initializer_list<const void*> ptrs) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (plan_dev >= 0 && plan_dev != dev) return false;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  if (cap != cudaStreamCaptureStatusNone) return true;
  cudaStreamCaptureMode mode = cudaStreamCaptureModeRelaxed;
  cudaThreadExchangeStreamCaptureMode(&mode);
  bool ok = true;
  int sdev = -1;
  if (cudaStreamGetDevice(s, &sdev) == cudaSuccess) {
    ok = sdev == dev;
  } else {
    cudaGetLastError();
  }
  for (const void* p : ptrs)
    if (ok && !pointer_on_device(p, dev)) ok = false;
  cudaThreadExchangeStreamCaptureMode(&mode);
  return ok;
}

// Arguments of one swept stage launch (one window per warp).
// Every field has a default, so a declared StageArgs is fully defined.
struct StageArgs {
  void* u = nullptr;           // flat state (F64 double[N]; F32C float hi[N], lo[N]; F32 float[N])
  const void* ein = nullptr;   // leading edges of the previous stage: nwin * 2B elements
  void* eout = nullptr;        // leading edges written by this stage
  int64_t N = 0;
  int nwin = 0;                // windows (N / B, or the regular plus the wide ones)
  int offset = 0;              // 0: windows [wB, wB+B); B/2: windows shifted right by B/2
  int hv = 0;                  // V-fill height (0 = load the flat state instead)
  int ht = 0;                  // trapezoid height (0 = none; h = full triangle)
  Consts c{};
  // Adjoint sweeps only: the forward trajectory, tape_len levels; the
  // sweep's level tau uses the forward level tape_len - tau, found by
  // tape_level() below: level n at tape + n*N when tape_ring is
  // 0, else in a ring of tape_ring chunks of tape_h levels (chunk c holds
  // levels tape_rem + c*tape_h ... at slot c mod tape_ring; levels below
  // tape_rem in the last slot).  lev_fill / lev_trap: sweep level of the
  // V-fill's base and of the trapezoid's flat base (also the stage index
  // times h: lev_trap = k*h for stage k).
  const double* tape = nullptr;
  int64_t tape_len = 0;
  int tape_ring = 0, tape_h = 0, tape_rem = 0;
  int64_t lev_fill = 0, lev_trap = 0;
  // Flat checkpoints of a forward FP64 KS advance (the adjoint's forward
  // pass): the V-fill of stage k ends with the window flat at level k*h of
  // the advance; when ckpt is set, 0 < k < ckpt_kmax and k % ckpt_every == 0
  // the kernels also store it to ckpt + (k / ckpt_every) * N.
  double* ckpt = nullptr;
  int ckpt_every = 0;
  int64_t ckpt_kmax = 0;
  int pdl = 0;                 // launch with programmatic dependent launch (host side only)
  int nlaunch = 0;             // windows launched (0: nwin); uneven tiles launch the regular ones only
  // Streamed ring launches: full-diamond stages run by one launch (0 or 1:
  // this stage only), with the per-warp slot counters, the status word and
  // the clock budget of each wait on a neighbouring warp.
  int nstream = 0;
  int stream_query = 0;        // host only: ask whether streaming pays, launch nothing
  int* progress = nullptr;
  int* status = nullptr;
  long long budget = 0;
  int drop = -1;               // failure injection: this warp never publishes its slot counter
};

// Forward level l of an adjoint sweep's tape (see StageArgs::tape).
__device__ __forceinline__ const double* tape_level(const StageArgs& a, int64_t l) {
  if (a.tape_ring == 0) return a.tape + l * a.N;
  const int li = (int)l;
  int slot, off;
  if (li < a.tape_rem) {
    slot = a.tape_ring - 1;
    off = li;
  } else {
    const int c = (li - a.tape_rem) / a.tape_h;
    off = li - a.tape_rem - c * a.tape_h;
    slot = c % a.tape_ring;
  }
  return a.tape + ((int64_t)slot * a.tape_h + off) * a.N;
}

// Where the flat level that ends stage k's V-fill is checkpointed, or nullptr.
__device__ __forceinline__ double* ckpt_of(const StageArgs& a, int64_t k) {
  if (!a.ckpt || k <= 0 || k >= a.ckpt_kmax || k % a.ckpt_every) return nullptr;
  return a.ckpt + (k / a.ckpt_every) * a.N;
}

// Launch `kern` on `s`; with pdl, as a programmatic dependent launch (the
// kernel may be scheduled while the previous kernel on the stream runs, and
// waits for it in griddep_wait_and_release).
template <class... KArgs, class... Args>
inline cudaError_t launch_kernel(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                 cudaStream_t s, Args... args) {
  if (!pdl) {
    kern<<<grid, block, smem, s>>>(args...);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// A launch of `grid` blocks as one thread block cluster (grid.x blocks,
// at most 16; above 8 the kernel must allow non-portable cluster sizes), with
// programmatic dependent launch when pdl.  query = true: *fits = 1 when one
// such cluster can be resident (nothing is launched).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_cluster(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                  cudaStream_t s, bool query, int* fits, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = grid.x;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 2 : 1;
  if (query) {
    int n = 0;
    const cudaError_t e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
    *fits = (e == cudaSuccess && n >= 1) ? 1 : 0;
    return e;
  }
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Launchers, one per (stencil, dtype); K = B / 32.
cudaError_t launch_stage_heat_f64(int K, const StageArgs& a, cudaStream_t s);
cudaError_t launch_stage_heat_f32c(int K, const StageArgs& a, cudaStream_t s);
cudaError_t launch_stage_ks_f64(int K, const StageArgs& a, cudaStream_t s);
cudaError_t launch_stage_ks_f32c(int K, const StageArgs& a, cudaStream_t s);
cudaError_t launch_stage_heat_f32(int K, const StageArgs& a, cudaStream_t s);
cudaError_t launch_stage_ks_f32(int K, const StageArgs& a, cudaStream_t s);

// Ring-pipelined full-diamond stage (hv = ht = h); nwarps <= 0 picks a size.
cudaError_t launch_ring_heat_f64(int K, const StageArgs& a, int nwarps, cudaStream_t s);
cudaError_t launch_ring_heat_f32c(int K, const StageArgs& a, int nwarps, cudaStream_t s);
cudaError_t launch_ring_ks_f64(int K, const StageArgs& a, int nwarps, cudaStream_t s);
cudaError_t launch_ring_ks_f32c(int K, const StageArgs& a, int nwarps, cudaStream_t s);
cudaError_t launch_ring_heat_f32(int K, const StageArgs& a, int nwarps, cudaStream_t s);
cudaError_t launch_ring_ks_f32(int K, const StageArgs& a, int nwarps, cudaStream_t s);

// Adjoint (transposed KS, FP64) stage over a tape; the ring version for full diamonds.
cudaError_t launch_stage_ksadj_f64(int K, const StageArgs& a, cudaStream_t s);
cudaError_t launch_ring_ksadj_f64(int K, const StageArgs& a, int nwarps, cudaStream_t s);

// Two-stage Runge-Kutta stencils (FP64, state pairs (u, m) on chip).
cudaError_t launch_stage_heatrk2_f64(int K, const StageArgs& a, cudaStream_t s);
cudaError_t launch_stage_ksrk2_f64(int K, const StageArgs& a, cudaStream_t s);
cudaError_t launch_ring_heatrk2_f64(int K, const StageArgs& a, int nwarps, cudaStream_t s);
cudaError_t launch_ring_ksrk2_f64(int K, const StageArgs& a, int nwarps, cudaStream_t s);
// Euler equations: FP64 (planar rho/m/E state, 72-byte edge elements, K in
// {1, 2, 4}) and compensated FP32 (hi[3N], lo[3N]; 48-byte edge elements,
// K in {1, 2, 4, 8}).
cudaError_t launch_stage_euler_f64(int K, const StageArgs& a, cudaStream_t s);
cudaError_t launch_ring_euler_f64(int K, const StageArgs& a, int nwarps, cudaStream_t s);
cudaError_t launch_stage_euler_f32c(int K, const StageArgs& a, cudaStream_t s);
cudaError_t launch_ring_euler_f32c(int K, const StageArgs& a, int nwarps, cudaStream_t s);
// Naive Euler stage of the midpoint rule on the planar state: out = base -
// ca (F_{i+1/2} - F_{i-1/2}) with the fluxes of (arg, minmod slopes of arg).
cudaError_t launch_naive_euler(const double* arg, const double* base, double* out, int64_t N, double ca,
                               double g1, cudaStream_t s, bool pdl = false);
// Compensated FP32 version: full = 0: out = hi + fma(-ca, dF, lo) (the
// midpoint, from arg = hi); full = 1: (out, out_lo) = TwoSum(hi, fma(-ca, dF, lo))
// (from arg = the midpoint).  All arrays 3N floats, planar.
cudaError_t launch_naive_euler_f32c(int full, const float* arg, const float* hi, const float* lo, float* out,
                                    float* out_lo, int64_t N, float ca, float g1, cudaStream_t s,
                                    bool pdl = false);
// Naive Runge-Kutta sub-timestep: sub 0: m = A(u); sub 1: out = B(u, m).
cudaError_t launch_naive_rk2(int stencil, int sub, const double* u, const double* m, double* out, int64_t N,
                             const Consts& c, cudaStream_t s, bool pdl = false);

// Uneven tiles (N not a multiple of B): the last nwin - nreg windows are
// B + 32r wide.  One warp per wide window does its V (a regular B window
// centred on the previous stage's boundary, stored flat to u) and then its
// trapezoid of the full width from u.  K in {1, 2, 4, 8, 16, 32} (multiple of r;
// Euler equations: K <= 4 in FP64, K <= 8 compensated).  ring < 0 launches
// the wide windows alone; ring >= 0 a full diamond stage in one launch, the
// ring over the a.nlaunch = nreg regular windows with `ring` warps (0:
// automatic) beside one warp per wide window.
cudaError_t launch_wide_f64(int stencil, int K, const StageArgs& a, int nreg, int odd, cudaStream_t s, int ring);
cudaError_t launch_wide_f32c(int stencil, int K, const StageArgs& a, int nreg, int odd, cudaStream_t s, int ring);
cudaError_t launch_wide_f32(int stencil, int K, const StageArgs& a, int nreg, int odd, cudaStream_t s, int ring);
cudaError_t launch_wide_rk2(int stencil, int K, const StageArgs& a, int nreg, int odd, cudaStream_t s, int ring);
cudaError_t launch_wide_euler(int dtype, int K, const StageArgs& a, int nreg, int odd, cudaStream_t s);
// The transposed KS step (adjoint sweeps) on the wide windows, FP64, K in {2, 4, 8, 16, 32}.
cudaError_t launch_wide_ksadj(int K, const StageArgs& a, int nreg, int odd, cudaStream_t s);

// Persistent advance (every stage in one launch, windows synchronised by
// flags): heat and KS, dtype 0 F64 / 1 F32C / 2 F32, K in {1, 2, 4, 8}.
struct PersistArgs {
  StageArgs a;                  // u, N, nwin, c (the per-stage fields are set on the device)
  unsigned char* edges;         // the edge double buffer
  size_t edge_half;             // bytes per buffer
  int* flags;                   // nwin counters of completed stages (zero before the launch)
  int* status;                  // SWEPT_OK, or SWEPT_ETIMEOUT when a wait ran out
  long long budget;             // clock cycles per wait
  int q, rem, H, nstages;
  int drop_w;                   // window whose publishes are dropped (a lost message; -1: none)
};
// Cluster-resident swept advance: the whole advance in one launch of one
// thread block cluster (at most 16 blocks of 1, 2 or 4 warps, one warp per
// window: nwin <= 64; K <= 4, Runge-Kutta pairs K <= 2), the stage edges in
// the blocks' shared memory (read by the neighbours through distributed shared
// memory), a cluster barrier between stages.
struct ResidentArgs {
  StageArgs a;                  // u, N, nwin, c (the per-stage fields are set on the device)
  int q, rem, H, nstages;
};
// query = true: *fits = 1 when the plan's cluster can be resident.
cudaError_t launch_resident(int stencil, int dtype, int K, const ResidentArgs& p, cudaStream_t s, bool pdl,
                            bool query, int* fits);
// Naive advance of nsteps sub-timesteps in one thread block cluster
// (forward-Euler heat and KS): the field split over the blocks' shared memory,
// each block stepping its part with R halo points from its neighbours, one
// cluster barrier per sub-timestep; query as above.
cudaError_t launch_naive_resident(int stencil, int dtype, void* u, int64_t N, const Consts& c, int64_t nsteps,
                                  cudaStream_t s, bool pdl, bool query, int* fits);

// query = true: *fits = 1 when every block of the launch can be resident at once.
cudaError_t launch_persistent(int stencil, int dtype, int K, const PersistArgs& p, cudaStream_t s, bool pdl,
                              bool query, int* fits);

// Shared-memory bytes per block of the stage kernel for tile width B and
// edge elements of esize bytes (8; 16 for the Runge-Kutta pair; 72 or 48
// for an Euler point state).
inline size_t stage_smem_bytes(int B, int esize = 8) { return (size_t)kWarpsPerBlock * 2 * B * esize; }

// Naive per-step stepper: out = S(in).
cudaError_t launch_naive_step(int stencil, int dtype, const void* in, void* out, int64_t N,
                              const Consts& c, cudaStream_t s, bool pdl = false);

// Conversion and reductions.
cudaError_t launch_split(int64_t N, const double* u64, float* u32c, cudaStream_t s);
cudaError_t launch_merge(int64_t N, const float* u32c, double* u64, cudaStream_t s);
// scratch: at least 2 * kReduceBlocks doubles.
constexpr int kReduceBlocks = 304;
cudaError_t launch_reduce(int dtype, const void* u, int what, const double* v, int64_t N,
                          double* scratch, double* out, cudaStream_t s);

}  // namespace swept
