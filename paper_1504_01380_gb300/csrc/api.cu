// C ABI of the swept-rule library (see include/swept.h for the contract).
//
// The plan owns the device scratch: the leading-edge double buffer (the
// "messages" of Section 3, written by one stage and read by the next) and
// the reduction partials.  swept_advance turns nsteps into the stage
// schedule and enqueues it on the caller's stream: the first triangle, the
// full diamonds (one streamed ring launch, or one launch per stage), the
// last fill and the remainder stage.
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "swept.h"
#include "swept_internal.h"
#include "swept_sync.cuh"

using swept::Consts;
using swept::StageArgs;

struct swept_plan_s {
  int64_t N;
  int radius, stencil, dtype, B, K, H, nwin, device;
  double prm[3];
  Consts c;
  unsigned char* edges;   // two buffers of nwin * 2B edge elements
  size_t edge_half;       // bytes per buffer
  double* red;            // 2 * kReduceBlocks partials
  int diamond;            // SWEPT_DIAMOND_*
  int ring_warps;         // 0 = automatic
  double* adj;            // adjoint scratch: work state, checkpoints, tape
  size_t adj_bytes;
  int rk2;                // two-stage Runge-Kutta: 2 levels per step, pair edges
  int subs;               // sub-timesteps (levels) per time step: 1, 2 or 4
  int use_graph;          // replay the stage sequence as a CUDA graph
  int pdl;                // programmatic dependent launch between consecutive kernels
  int persistent;         // SWEPT_OPT_PERSISTENT: 0 off, 1 when eligible
  int* flags;             // nwin stage counters of the persistent advance
  int* status;            // its device status word
  int drop_w;             // SWEPT_OPT_DROP_WINDOW: a window that never publishes (-1: none)
  int nreg;               // uneven tiles: windows [0, nreg) are B wide, the rest B + 32r (nreg = nwin: even)
  double timeout_s;       // SWEPT_OPT_TIMEOUT_MS / 1000: budget of each persistent or streamed wait
  int stream;             // SWEPT_OPT_STREAM: ring stages of an advance in one launch
  int time_ring;          // SWEPT_OPT_TIME_RING: events around the ring launches of each advance
  int resident;           // SWEPT_OPT_RESIDENT: cluster-resident advance where the problem fits one cluster
  int naive_resident;     // SWEPT_OPT_NAIVE_RESIDENT: the naive stepper's steps in one cluster
  cudaEvent_t ring_ev[2];
  int ring_timed;         // the last advance recorded ring_ev
  int64_t last_launches, last_ring_launches;
  cudaGraphExec_t gexec;  // captured advance (valid for g_u, g_nsteps)
  void* g_u;
  int64_t g_nsteps;
  int g_valid;
};

namespace {

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return SWEPT_OK;
  if (e == cudaErrorMemoryAllocation) return SWEPT_ENOMEM;
  return SWEPT_ECUDA;
}

// Constants of the update.  heat: r.  KS: a = -(dt/(4 dx)), b = -(dt/dx^2),
// e = -(dt/(dx^2 dx^2)), evaluated in FP64 in this order; FP32 copies are
// the FP64 values rounded to nearest.
int make_consts(int stencil, const double* p, int np, Consts& c) {
  std::memset(&c, 0, sizeof c);
  if (stencil == SWEPT_EULER) {
    // dt/dx and gamma - 1, FP64 in this order; params = {dt, dx, gamma}
    if (np < 3 || !(p[1] > 0.0) || !(p[0] >= 0.0) || !(p[2] > 1.0)) return SWEPT_EINVAL;
    c.dtdx = p[0] / p[1];
    c.g1 = p[2] - 1.0;
    c.dtdx32 = (float)c.dtdx;
    c.g132 = (float)c.g1;
    return SWEPT_OK;
  }
  if (stencil == SWEPT_HEAT_RK2 || stencil == SWEPT_KS_RK2) stencil -= 2;   // same constants
  if (stencil == SWEPT_HEAT) {
    if (np < 1) return SWEPT_EINVAL;
    c.r = p[0];
    c.r32 = (float)c.r;
    return SWEPT_OK;
  }
  if (stencil == SWEPT_KS) {
    if (np < 2 || !(p[1] > 0.0)) return SWEPT_EINVAL;
    const double dt = p[0], dx = p[1];
    const double dx2 = dx * dx;
    c.a = -(dt / (4.0 * dx));
    c.b = -(dt / dx2);
    c.e = -(dt / (dx2 * dx2));
    c.a32 = (float)c.a;
    c.b32 = (float)c.b;
    c.e32 = (float)c.e;
    return SWEPT_OK;
  }
  return SWEPT_EINVAL;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int sm_count(const swept_plan_s* p) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
  return sms;
}

cudaError_t launch_stage(const swept_plan_s* p, const StageArgs& a, cudaStream_t s) {
  if (p->stencil == SWEPT_EULER)
    return p->dtype == SWEPT_F64 ? swept::launch_stage_euler_f64(p->K, a, s)
                                 : swept::launch_stage_euler_f32c(p->K, a, s);
  if (p->stencil == SWEPT_HEAT_RK2) return swept::launch_stage_heatrk2_f64(p->K, a, s);
  if (p->stencil == SWEPT_KS_RK2) return swept::launch_stage_ksrk2_f64(p->K, a, s);
  if (p->dtype == SWEPT_F32)
    return p->stencil == SWEPT_HEAT ? swept::launch_stage_heat_f32(p->K, a, s)
                                    : swept::launch_stage_ks_f32(p->K, a, s);
  if (p->stencil == SWEPT_HEAT)
    return p->dtype == SWEPT_F64 ? swept::launch_stage_heat_f64(p->K, a, s)
                                 : swept::launch_stage_heat_f32c(p->K, a, s);
  return p->dtype == SWEPT_F64 ? swept::launch_stage_ks_f64(p->K, a, s)
                               : swept::launch_stage_ks_f32c(p->K, a, s);
}

// Full diamond stage on the ring kernel.  Under SWEPT_DIAMOND_AUTO with
// automatic warps the launcher may pick the per-window kernel instead (when
// every window gets a resident warp at once).
cudaError_t launch_ring(const swept_plan_s* p, const StageArgs& a, cudaStream_t s) {
  const int w = (p->diamond == SWEPT_DIAMOND_AUTO && p->ring_warps == 0) ? -1 : p->ring_warps;
  if (p->stencil == SWEPT_EULER)
    return p->dtype == SWEPT_F64 ? swept::launch_ring_euler_f64(p->K, a, w, s)
                                 : swept::launch_ring_euler_f32c(p->K, a, w, s);
  if (p->stencil == SWEPT_HEAT_RK2) return swept::launch_ring_heatrk2_f64(p->K, a, w, s);
  if (p->stencil == SWEPT_KS_RK2) return swept::launch_ring_ksrk2_f64(p->K, a, w, s);
  if (p->dtype == SWEPT_F32)
    return p->stencil == SWEPT_HEAT ? swept::launch_ring_heat_f32(p->K, a, w, s)
                                    : swept::launch_ring_ks_f32(p->K, a, w, s);
  if (p->stencil == SWEPT_HEAT)
    return p->dtype == SWEPT_F64 ? swept::launch_ring_heat_f64(p->K, a, w, s)
                                 : swept::launch_ring_heat_f32c(p->K, a, w, s);
  return p->dtype == SWEPT_F64 ? swept::launch_ring_ks_f64(p->K, a, w, s)
                               : swept::launch_ring_ks_f32c(p->K, a, w, s);
}

// The ring kernel needs at least two windows per warp to gain over the
// per-window kernel; automatic choice: ring from 8 windows up.
bool use_ring(const swept_plan_s* p) {
  if (p->diamond == SWEPT_DIAMOND_RING) return true;
  if (p->diamond == SWEPT_DIAMOND_WINDOW) return false;
  return p->nwin >= 8;
}

// Default tile width: the largest of 512, 256, ... that keeps K a multiple
// of the radius and divides N, or else tiles it with uneven tiles (Euler
// equations: from 64 in FP64, 128 in F32C).
// Uneven tiles: N = nreg*B + (nwide - 1)*(B + 32r) + W with
// nwide = ceil((N mod B) / (32r)) and the last window W = N - (its start)
// points wide (B + 1 .. B + 32r), nreg >= 0, for every stencil and precision
// the plan takes (K <= 32; Euler equations: K <= 4 in FP64, 8
// compensated).  Any N of at least nwide tiles is tiled so.  Returns nreg, or
// -1 when N cannot be tiled so.
int64_t uneven_nreg(int64_t N, int B, int radius, int stencil, int dtype) {
  if (stencil == SWEPT_EULER) {
    if (B / 32 > (dtype == SWEPT_F64 ? 4 : 8)) return -1;
  } else if (B / 32 > 32) {
    return -1;
  }
  const int64_t extra = N % B;
  const int64_t nwide = (extra + 32 * radius - 1) / (32 * radius);
  const int64_t nreg = N / B - nwide;
  return nreg >= 0 && nreg + nwide >= 1 ? nreg : -1;
}

// The default tile: the widest that divides N or tiles it unevenly, up to
// 1024 points from N = 2^22 on (at least 4096 windows: measured fastest there
// for heat and KS in every precision, e.g. compensated KS at N = 2^22 1.45
// against 1.14e12 cell-updates/s at 512) and 512 below; the Euler equations
// 64 (FP64) or 128 (compensated), their measured best.
int default_B(int64_t N, int radius, int stencil, int dtype) {
  const int kmax = stencil != SWEPT_EULER ? (N >= ((int64_t)1 << 22) ? 32 : 16) : (dtype == SWEPT_F64 ? 2 : 4);
  for (int K = kmax; K >= 1; K /= 2) {
    const int B = 32 * K;
    if (K % radius == 0 && (N % B == 0 || uneven_nreg(N, B, radius, stencil, dtype) >= 0)) return B;
  }
  return 0;
}

}  // namespace

extern "C" {

const char* swept_strerror(int code) {
  switch (code) {
    case SWEPT_OK: return "ok";
    case SWEPT_EINVAL: return "invalid argument";
    case SWEPT_ENOMEM: return "out of device memory";
    case SWEPT_ECUDA: return "CUDA error";
    case SWEPT_ETIMEOUT: return "device-side wait timed out";
    case SWEPT_ENOTSUP: return "not supported by this build";
    case SWEPT_ETOOBIG: return "problem exceeds the fixed scratch of swept_advance_noalloc";
    default: return "unknown status";
  }
}

const char* swept_version(void) { return "swept 0.1 sm_103a"; }

int swept_plan(swept_plan_t* out, int64_t N, int radius, int stencil_id, const double* params,
               int nparams, int dtype, int B) {
  if (!out || !params) return SWEPT_EINVAL;
  *out = nullptr;
  if (stencil_id < SWEPT_HEAT || stencil_id > SWEPT_EULER) return SWEPT_EINVAL;
  const bool euler = stencil_id == SWEPT_EULER;
  const int rad = (stencil_id == SWEPT_HEAT || stencil_id == SWEPT_HEAT_RK2 || euler) ? 1 : 2;
  if (radius != rad) return SWEPT_EINVAL;
  if (dtype != SWEPT_F64 && dtype != SWEPT_F32C && dtype != SWEPT_F32) return SWEPT_EINVAL;
  const bool rk2 = stencil_id == SWEPT_HEAT_RK2 || stencil_id == SWEPT_KS_RK2;
  if (rk2 && dtype != SWEPT_F64) return SWEPT_ENOTSUP;
  if (euler && dtype == SWEPT_F32) return SWEPT_ENOTSUP;
  if (N <= 0) return SWEPT_EINVAL;
  if (B == 0) B = default_B(N, rad, stencil_id, dtype);
  if (B <= 0 || B % 32) return SWEPT_EINVAL;
  const int K = B / 32;
  if (K != 1 && K != 2 && K != 4 && K != 8 && K != 16 && K != 32) return SWEPT_ENOTSUP;
  if (euler && K > (dtype == SWEPT_F64 ? 4 : 8)) return SWEPT_ENOTSUP;
  if (K % rad) return SWEPT_EINVAL;
  int64_t nreg = N / B;
  if (N % B) {
    nreg = uneven_nreg(N, B, rad, stencil_id, dtype);
    if (nreg < 0) return SWEPT_EINVAL;
  }
  if (N / B > (int64_t)0x7fffffff) return SWEPT_EINVAL;
  Consts c;
  int st = make_consts(stencil_id, params, nparams, c);
  if (st) return st;

  swept_plan_s* p = (swept_plan_s*)std::calloc(1, sizeof(swept_plan_s));
  if (!p) return SWEPT_ENOMEM;
  p->N = N;
  p->radius = rad;
  p->stencil = stencil_id;
  p->dtype = dtype;
  p->B = B;
  p->K = K;
  p->H = B / (2 * rad);
  p->nwin = (int)(N / B);                 // nreg regular windows, then the wide ones
  p->nreg = (int)nreg;
  for (int i = 0; i < 3; ++i) p->prm[i] = i < nparams ? params[i] : 0.0;
  p->c = c;
  p->rk2 = rk2 ? 1 : 0;
  p->subs = euler ? 4 : (rk2 ? 2 : 1);
  p->pdl = 1;
  p->drop_w = -1;
  p->timeout_s = 2.0;
  p->stream = 1;
  p->resident = 1;
  cudaGetDevice(&p->device);
  const size_t esize = euler ? (dtype == SWEPT_F64 ? sizeof(swept::EulerE) : sizeof(swept::EulerEF))
                              : (rk2 ? 16 : (dtype == SWEPT_F32 ? 4 : 8));
  p->edge_half = (size_t)p->nwin * 2 * B * esize;
  cudaError_t e = cudaMalloc((void**)&p->edges, 2 * p->edge_half);
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->red, 2 * swept::kReduceBlocks * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->flags, (size_t)p->nwin * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(p->status, 0, sizeof(int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFree(p->edges);
    cudaFree(p->red);
    cudaFree(p->flags);
    cudaFree(p->status);
    std::free(p);
    return cuda_status(e);
  }
  *out = p;
  return SWEPT_OK;
}

void swept_destroy(swept_plan_t p) {
  if (!p) return;
  cudaDeviceSynchronize();
  if (p->g_valid) cudaGraphExecDestroy(p->gexec);
  if (p->time_ring) {
    cudaEventDestroy(p->ring_ev[0]);
    cudaEventDestroy(p->ring_ev[1]);
  }
  if (p->edges) cudaFree(p->edges);
  if (p->red) cudaFree(p->red);
  if (p->adj) cudaFree(p->adj);
  cudaFree(p->flags);
  cudaFree(p->status);
  std::free(p);
}

int swept_plan_info(swept_plan_t p, int64_t* info, int ninfo) {
  if (!p || !info) return SWEPT_EINVAL;
  const int64_t v[6] = {p->B, p->H, p->N, p->dtype, p->stencil, p->radius};
  for (int i = 0; i < ninfo && i < 6; ++i) info[i] = v[i];
  return SWEPT_OK;
}

int swept_plan_set(swept_plan_t p, int option, int64_t value) {
  if (!p) return SWEPT_EINVAL;
  if (option == SWEPT_OPT_DIAMOND) {
    if (value < SWEPT_DIAMOND_AUTO || value > SWEPT_DIAMOND_RING) return SWEPT_EINVAL;
    p->diamond = (int)value;
    return SWEPT_OK;
  }
  if (option == SWEPT_OPT_RING_WARPS) {
    if (value < 0 || value > (int64_t)1 << 30) return SWEPT_EINVAL;
    p->ring_warps = (int)value;
    return SWEPT_OK;
  }
  if (option == SWEPT_OPT_GRAPH) {
    if (value != 0 && value != 1) return SWEPT_EINVAL;
    p->use_graph = (int)value;
    if (p->g_valid) {              // the captured launches carry the old setting
      cudaGraphExecDestroy(p->gexec);
      p->g_valid = 0;
    }
    return SWEPT_OK;
  }
  if (option == SWEPT_OPT_RESIDENT || option == SWEPT_OPT_NAIVE_RESIDENT) {
    if (value != 0 && value != 1) return SWEPT_EINVAL;
    (option == SWEPT_OPT_RESIDENT ? p->resident : p->naive_resident) = (int)value;
    if (p->g_valid) {
      cudaGraphExecDestroy(p->gexec);
      p->g_valid = 0;
    }
    return SWEPT_OK;
  }
  if (option == SWEPT_OPT_PERSISTENT) {
    if (value != 0 && value != 1) return SWEPT_EINVAL;
    p->persistent = (int)value;
    if (p->g_valid) {
      cudaGraphExecDestroy(p->gexec);
      p->g_valid = 0;
    }
    return SWEPT_OK;
  }
  if (option == SWEPT_OPT_DROP_WINDOW) {
    if (value < -1 || value >= p->nwin) return SWEPT_EINVAL;
    p->drop_w = (int)value;
    if (p->g_valid) {
      cudaGraphExecDestroy(p->gexec);
      p->g_valid = 0;
    }
    return SWEPT_OK;
  }
  if (option == SWEPT_OPT_TIMEOUT_MS) {
    if (value < 1 || value > 600000) return SWEPT_EINVAL;
    p->timeout_s = (double)value / 1000.0;
    if (p->g_valid) {
      cudaGraphExecDestroy(p->gexec);
      p->g_valid = 0;
    }
    return SWEPT_OK;
  }
  if (option == SWEPT_OPT_TIME_RING) {
    if (value != 0 && value != 1) return SWEPT_EINVAL;
    if (value == p->time_ring) return SWEPT_OK;
    cudaError_t e = cudaSuccess;
    if (value) {
      e = cudaEventCreate(&p->ring_ev[0]);
      if (e == cudaSuccess) {
        e = cudaEventCreate(&p->ring_ev[1]);
        if (e != cudaSuccess) cudaEventDestroy(p->ring_ev[0]);
      }
    } else {
      cudaEventDestroy(p->ring_ev[0]);
      cudaEventDestroy(p->ring_ev[1]);
    }
    if (e != cudaSuccess) return cuda_status(e);
    p->time_ring = (int)value;
    p->ring_timed = 0;
    return SWEPT_OK;
  }
  if (option == SWEPT_OPT_STREAM) {
    if (value != 0 && value != 1) return SWEPT_EINVAL;
    p->stream = (int)value;
    if (p->g_valid) {
      cudaGraphExecDestroy(p->gexec);
      p->g_valid = 0;
    }
    return SWEPT_OK;
  }
  if (option == SWEPT_OPT_PDL) {
    if (value != 0 && value != 1) return SWEPT_EINVAL;
    p->pdl = (int)value;
    if (p->g_valid) {
      cudaGraphExecDestroy(p->gexec);
      p->g_valid = 0;
    }
    return SWEPT_OK;
  }
  return SWEPT_EINVAL;
}

}  // extern "C"

namespace {

// The persistent advance applies to forward-Euler heat and KS with K <= 8 when
// every window's warp can be resident at once.
bool persistent_ok(const swept_plan_s* p, int64_t levels) {
  if (!p->persistent || p->subs != 1 || p->K > 8 || p->nreg != p->nwin) return false;
  if (p->stencil != SWEPT_HEAT && p->stencil != SWEPT_KS) return false;
  if (levels / p->H > (int64_t)0x3fffffff) return false;
  swept::PersistArgs pa{};
  pa.a.nwin = p->nwin;
  int fits = 0;
  const int st = p->stencil == SWEPT_HEAT ? swept::kHeat : swept::kKS;
  if (swept::launch_persistent(st, p->dtype, p->K, pa, nullptr, false, true, &fits) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return fits != 0;
}

// Internal stencil id of a plan.
int internal_stencil(const swept_plan_s* p) {
  switch (p->stencil) {
    case SWEPT_HEAT: return swept::kHeat;
    case SWEPT_KS: return swept::kKS;
    case SWEPT_HEAT_RK2: return swept::kHeatRK2;
    case SWEPT_KS_RK2: return swept::kKSRK2;
    default: return swept::kEuler;
  }
}

// The cluster-resident advance (SWEPT_OPT_RESIDENT) applies to evenly tiled
// heat and KS plans (forward Euler, K <= 4; Runge-Kutta pairs, K <= 2) of at
// most 64 windows whose cluster fits the GPU, with the automatic kernel
// choice and neither the persistent advance nor failure injection asked for.
bool resident_ok(const swept_plan_s* p, int64_t levels) {
  if (!p->resident || p->persistent || p->drop_w >= 0 || p->nreg != p->nwin || p->nwin > 64) return false;
  if (p->diamond != SWEPT_DIAMOND_AUTO || p->ring_warps != 0) return false;
  if (p->stencil == SWEPT_EULER || p->K > (p->rk2 ? 2 : 4)) return false;
  if (levels / p->H > (int64_t)0x3fffffff) return false;
  swept::ResidentArgs ra{};
  ra.a.nwin = p->nwin;
  int fits = 0;
  if (swept::launch_resident(internal_stencil(p), p->dtype, p->K, ra, nullptr, false, true, &fits) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return fits != 0;
}

// Clock cycles of one bounded wait (SWEPT_OPT_TIMEOUT_MS at the SM clock).
long long wait_budget(const swept_plan_s* p) {
  int dev = 0, khz = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
  if (khz <= 0) khz = 2000000;
  return (long long)(p->timeout_s * (double)khz * 1000.0);
}

// The ring stages of an advance (q - 1 full diamonds) run as one streamed
// launch when there are at least two of them, the tiles are even, and the
// ring is the kernel for them (with the automatic choice: more windows than
// four per SM, where the per-window kernel is not picked instead).
// Uneven tiles stream too (swept_stream_wide_kernel: the wide windows beside
// the regular windows' runs), except for the Euler equations, whose wide
// windows' shared memory would cost their ring a block per SM.
bool stream_ok(const swept_plan_s* p, int64_t q) {
  if (!p->stream || q < 3 || p->nreg < 3 || !use_ring(p)) return false;
  if (p->nreg != p->nwin && p->stencil == SWEPT_EULER) return false;
  if (q - 1 > (int64_t)0x7fffffff / p->nwin) return false;    // slot counters stay in int
  if (p->diamond == SWEPT_DIAMOND_AUTO && p->ring_warps == 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (p->nreg <= 4 * sms) return false;
    // and only where it pays (run length against residency; the ring launcher decides)
    StageArgs a{};
    a.nwin = p->nreg;
    a.nstream = (int)(q - 1);
    a.stream_query = 1;
    return launch_ring(p, a, nullptr) == cudaSuccess;
  }
  return true;
}

// The wide windows of an uneven tiling (swept_wide.cuh): alone (ring < 0),
// beside the ring over the a.nlaunch regular windows in one launch (ring >= 0
// warps, 0 automatic), or, with a.nstream > 1, every full diamond stage of the
// advance in one streamed launch.
cudaError_t launch_wide(const swept_plan_s* p, const StageArgs& a, int odd, cudaStream_t s, int ring) {
  if (p->stencil == SWEPT_EULER) return swept::launch_wide_euler(p->dtype, p->K, a, p->nreg, odd, s);
  if (p->stencil == SWEPT_HEAT_RK2) return swept::launch_wide_rk2(swept::kHeatRK2, p->K, a, p->nreg, odd, s, ring);
  if (p->stencil == SWEPT_KS_RK2) return swept::launch_wide_rk2(swept::kKSRK2, p->K, a, p->nreg, odd, s, ring);
  const int st = p->stencil == SWEPT_HEAT ? swept::kHeat : swept::kKS;
  if (p->dtype == SWEPT_F64) return swept::launch_wide_f64(st, p->K, a, p->nreg, odd, s, ring);
  if (p->dtype == SWEPT_F32C) return swept::launch_wide_f32c(st, p->K, a, p->nreg, odd, s, ring);
  return swept::launch_wide_f32(st, p->K, a, p->nreg, odd, s, ring);
}

// Flat checkpoints an advance stores on the way (the adjoint's forward pass):
// the level that ends stage k's V-fill goes to ckpt + (k / every) * N for
// 0 < k < kmax, k % every == 0 (StageArgs::ckpt).
struct Dumps {
  double* ckpt;
  int every;
  int64_t kmax;
};

// Enqueue the stage sequence of one advance (Section 3's stages, A5's schedule).
int enqueue_advance(swept_plan_s* p, void* u, int64_t nsteps, cudaStream_t s, const Dumps* dumps = nullptr) {
  const int64_t levels = p->subs * nsteps;                // sub-timesteps
  const int64_t H = p->H;
  const int64_t q = levels / H;
  const int rem = (int)(levels % H);
  if (!dumps && levels > 0 && resident_ok(p, levels)) {
    swept::ResidentArgs ra{};
    ra.a.u = u;
    ra.a.N = p->N;
    ra.a.nwin = p->nwin;
    ra.a.c = p->c;
    ra.q = (int)q;
    ra.rem = rem;
    ra.H = (int)H;
    ra.nstages = q == 0 ? 2 : (rem ? (int)q + 2 : (int)q + 1);
    p->last_launches = 1;
    p->last_ring_launches = 0;
    p->ring_timed = 0;
    return cuda_status(swept::launch_resident(internal_stencil(p), p->dtype, p->K, ra, s, p->pdl != 0, false, nullptr));
  }
  if (!dumps && persistent_ok(p, levels)) {
    swept::PersistArgs pa{};
    pa.a.u = u;
    pa.a.N = p->N;
    pa.a.nwin = p->nwin;
    pa.a.c = p->c;
    pa.edges = p->edges;
    pa.edge_half = p->edge_half;
    pa.flags = p->flags;
    pa.status = p->status;
    pa.budget = wait_budget(p);                       // per wait
    pa.drop_w = p->drop_w;
    pa.q = (int)q;
    pa.rem = rem;
    pa.H = (int)H;
    pa.nstages = q == 0 ? 2 : (rem ? (int)q + 2 : (int)q + 1);
    cudaError_t e = cudaMemsetAsync(p->flags, 0, (size_t)p->nwin * sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->status, 0, sizeof(int), s);
    const int st = p->stencil == SWEPT_HEAT ? swept::kHeat : swept::kKS;
    if (e == cudaSuccess) e = swept::launch_persistent(st, p->dtype, p->K, pa, s, false, false, nullptr);
    return cuda_status(e);
  }
  unsigned char* buf[2] = {p->edges, p->edges + p->edge_half};
  // launch counts of this advance, and events around its ring launches
  // (SWEPT_OPT_TIME_RING; not while the stream is being captured)
  int64_t nlaunch = 0, nring = 0;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  const bool timing = p->time_ring && cudaStreamIsCapturing(s, &cap) == cudaSuccess &&
                      cap == cudaStreamCaptureStatusNone;
  p->ring_timed = 0;
  StageArgs a{};
  a.u = u;
  a.N = p->N;
  a.nwin = p->nwin;
  a.c = p->c;
  a.pdl = p->pdl;
  if (dumps) {
    a.ckpt = dumps->ckpt;
    a.ckpt_every = dumps->every;
    a.ckpt_kmax = dumps->kmax;
  }
  // stage k: windows shifted by B/2 when k is odd (the alternating point
  // sets of Section 3); reads the edges of stage k-1, writes its own.
  const bool uneven = p->nreg != p->nwin;
  const bool ring = use_ring(p) && p->nreg > 0;
  auto setup = [&](int64_t k, int hv, int ht) {
    a.offset = (k & 1) ? p->B / 2 : 0;
    a.hv = hv;
    a.ht = ht;
    a.ein = buf[(k + 1) & 1];
    a.eout = buf[k & 1];
    a.lev_fill = k >= 1 ? (k - 1) * H : 0;      // absolute levels (Runge-Kutta parity)
    a.lev_trap = k * H;
  };
  auto stage = [&](int64_t k, int hv, int ht) -> cudaError_t {
    setup(k, hv, ht);
    const bool full = ring && hv == p->H && ht == p->H;
    ++nlaunch;
    if (full) ++nring;
    if (!uneven) return full ? launch_ring(p, a, s) : launch_stage(p, a, s);
    // uneven tiles: the B-wide windows (ring or per window) and the wide ones;
    // a full diamond stage on the ring runs both in one launch (except for the
    // Euler equations, whose ring would lose a block per SM to the wide
    // windows' larger shared memory)
    const int odd = (int)(k & 1);
    const int w = (p->diamond == SWEPT_DIAMOND_AUTO && p->ring_warps == 0) ? -1 : p->ring_warps;
    const bool joint = full && p->stencil != SWEPT_EULER &&
                       (w >= 0 || (int64_t)p->nreg > 4 * (int64_t)sm_count(p));
    cudaError_t e = cudaSuccess;
    if (p->nreg > 0 && !joint) {
      a.nlaunch = p->nreg;
      e = full ? launch_ring(p, a, s) : launch_stage(p, a, s);
      a.nlaunch = 0;
      ++nlaunch;
    }
    if (e != cudaSuccess) return e;
    a.nlaunch = joint ? p->nreg : 0;
    e = launch_wide(p, a, odd, s, joint ? (w > 0 ? w : 0) : -1);
    a.nlaunch = 0;
    return e;
  };
  cudaError_t e = cudaSuccess;
  if (q == 0) {
    e = stage(0, 0, rem);                              // trapezoid of height rem
    if (e == cudaSuccess) e = stage(1, rem, 0);       // its V-fill
  } else {
    e = stage(0, 0, (int)H);                           // shrinking triangles
    const bool stream = stream_ok(p, q);
    if (e == cudaSuccess && stream) {
      // diamonds 1 .. q-1 in one streamed ring launch; its slot counters and
      // the status word start from 0
      setup(1, (int)H, (int)H);
      a.nstream = (int)(q - 1);
      a.progress = p->flags;
      a.status = p->status;
      a.budget = wait_budget(p);
      a.drop = p->drop_w;
      e = cudaMemsetAsync(p->flags, 0, (size_t)p->nwin * sizeof(int), s);
      if (e == cudaSuccess) e = cudaMemsetAsync(p->status, 0, sizeof(int), s);
      if (e == cudaSuccess && timing) e = cudaEventRecord(p->ring_ev[0], s);
      if (e == cudaSuccess) {
        if (!uneven) {
          e = launch_ring(p, a, s);
        } else {
          // the regular windows' runs and the wide windows in one launch; the
          // counters are per window
          const int w = (p->diamond == SWEPT_DIAMOND_AUTO && p->ring_warps == 0) ? 0 : p->ring_warps;
          e = launch_wide(p, a, 1, s, w);
        }
      }
      if (e == cudaSuccess && timing) e = cudaEventRecord(p->ring_ev[1], s);
      a.nstream = 0;
      ++nlaunch;
      ++nring;
    } else {
      const bool timed = timing && ring && !uneven && q >= 2;
      if (e == cudaSuccess && timed) e = cudaEventRecord(p->ring_ev[0], s);
      for (int64_t k = 1; k < q && e == cudaSuccess; ++k) e = stage(k, (int)H, (int)H);   // diamonds
      if (e == cudaSuccess && timed) e = cudaEventRecord(p->ring_ev[1], s);
    }
    p->ring_timed = timing && nring > 0 && e == cudaSuccess;
    if (e == cudaSuccess) e = stage(q, (int)H, rem);  // last V-fill (+ trapezoid)
    if (e == cudaSuccess && rem > 0) e = stage(q + 1, rem, 0);
  }
  p->last_launches = nlaunch;
  p->last_ring_launches = nring;
  return cuda_status(e);
}

}  // namespace

extern "C" {

int swept_advance(swept_plan_t p, void* u, int64_t nsteps, void* stream) {
  if (!p || !u || nsteps < 0 || !aligned16(u)) return SWEPT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (!swept::call_on_device(p->device, s, {u})) return SWEPT_EINVAL;
  if (nsteps == 0) return SWEPT_OK;
  if (!p->use_graph) return enqueue_advance(p, u, nsteps, s);
  // graph replay: capture the stage sequence once per (u, nsteps)
  if (!p->g_valid || p->g_u != u || p->g_nsteps != nsteps) {
    if (p->g_valid) {
      cudaGraphExecDestroy(p->gexec);
      p->g_valid = 0;
    }
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_status(e);
    cudaGraph_t g;
    int rc = SWEPT_OK;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      rc = enqueue_advance(p, u, nsteps, cs);
      e = cudaStreamEndCapture(cs, &g);
      if (e == cudaSuccess) {
        if (rc == SWEPT_OK) e = cudaGraphInstantiate(&p->gexec, g, 0);
        cudaGraphDestroy(g);
      }
    }
    cudaStreamDestroy(cs);
    if (rc != SWEPT_OK) return rc;
    if (e != cudaSuccess) return cuda_status(e);
    p->g_valid = 1;
    p->g_u = u;
    p->g_nsteps = nsteps;
  }
  return cuda_status(cudaGraphLaunch(p->gexec, s));
}

}  // extern "C"

namespace {

// Scratch of the KS adjoint.  The forward pass is one swept advance that
// also stores the flat level ending every m-th stage (a flat checkpoint every
// m*h levels, m = `every`); the reverse pass recomputes the forward levels
// from those checkpoints, m*h at a time, with the naive stepper (every level
// is computed once more, as in any checkpointed adjoint) into a ring of m + 1
// chunks of h levels, and sweeps the cotangent back one stage at a time,
// each stage reading at most two chunks.  nsteps = q*h + rem is advanced as
// rem levels first, so that the long advance's stage boundaries are the
// sweep's (forward level rem + k*h = sweep level (q - k)*h).  Scratch, in
// states of 8N bytes: the level-0 state (when rem > 0) + ceil(q/m)
// checkpoints + (m + 1)*h tape levels; m (at most 2*K_cycles stages, K_cycles
// swept cycles of two stages) is the one that minimises it.
struct AdjLayout {
  int64_t q = 0, rem = 0, every = 1, nckpt = 0, ring = 0, states = 0;
};

AdjLayout adjoint_layout(const swept_plan_s* p, int64_t nsteps, int K_cycles) {
  AdjLayout L;
  const int64_t H = p->H;
  L.q = nsteps / H;
  L.rem = nsteps % H;
  if (K_cycles <= 0) K_cycles = 64;
  const int64_t mmax = 2 * (int64_t)K_cycles;
  int64_t best = -1;
  for (int64_t m = 1; m <= mmax && m <= (L.q > 1 ? L.q : 1); ++m) {
    const int64_t states = (L.q + m - 1) / m + (m + 1) * H;
    if (best < 0 || states < best) {
      best = states;
      L.every = m;
    }
  }
  L.nckpt = L.q > 0 ? (L.q + L.every - 1) / L.every : 0;
  L.ring = L.every + 1;
  L.states = (L.rem > 0 ? 1 : 0) + L.nckpt + L.ring * H;
  return L;
}

// Host mirror of tape_level(): the ring slot of forward level l.
double* tape_at(double* ring, const AdjLayout& L, int64_t H, int64_t N, int64_t l) {
  int64_t slot, off;
  if (l < L.rem) {
    slot = L.ring - 1;
    off = l;
  } else {
    const int64_t c = (l - L.rem) / H;
    off = l - L.rem - c * H;
    slot = c % L.ring;
  }
  return ring + (slot * H + off) * N;
}

int adjoint_ks(swept_plan_s* p, const double* u0, double* lam, int64_t F, const AdjLayout& L, double* scratch,
               cudaStream_t s) {
  const int64_t N = p->N, H = p->H;
  const size_t bytes = (size_t)N * sizeof(double);
  double* pre = scratch;                                   // level 0 (rem > 0)
  double* ckpt = pre + (L.rem > 0 ? N : 0);                // level rem + g*every*H, g < nckpt
  double* ring = ckpt + L.nckpt * N;                       // the tape ring
  cudaError_t e = cudaSuccess;
  // ---- forward pass: checkpoints
  if (L.rem > 0) e = cudaMemcpyAsync(pre, u0, bytes, cudaMemcpyDeviceToDevice, s);
  if (L.q > 0) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(ckpt, u0, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && L.rem > 0) {
      const int rc = enqueue_advance(p, ckpt, L.rem, s);     // level rem
      if (rc != SWEPT_OK) return rc;
    }
    // the long advance runs in the ring's memory (free until the reverse pass)
    if (e == cudaSuccess) e = cudaMemcpyAsync(ring, ckpt, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && L.nckpt > 1) {
      const Dumps d{ckpt, (int)L.every, L.q};
      const int rc = enqueue_advance(p, ring, L.q * H, s, &d);
      if (rc != SWEPT_OK) return rc;
    }
  }
  if (e != cudaSuccess) return cuda_status(e);
  // ---- reverse pass.  Chunk c >= 0 holds forward levels rem + c*H .. + H - 1,
  // chunk -1 levels 0 .. rem - 1; chunks >= `lowest` are in the ring.
  int64_t lowest = L.q;
  auto recompute_down_to = [&](int64_t need) -> cudaError_t {
    cudaError_t r = cudaSuccess;
    while (lowest > need && r == cudaSuccess) {
      const int64_t top = lowest - 1;
      int64_t l0, count;
      const double* from;
      if (top >= 0) {                                     // the checkpoint group holding chunk top
        const int64_t g = top / L.every;
        l0 = L.rem + g * L.every * H;
        count = (lowest - g * L.every) * H;
        from = ckpt + g * N;
        lowest = g * L.every;
      } else {
        l0 = 0;
        count = L.rem;
        from = pre;
        lowest = -1;
      }
      r = cudaMemcpyAsync(tape_at(ring, L, H, N, l0), from, bytes, cudaMemcpyDeviceToDevice, s);
      for (int64_t l = l0 + 1; l < l0 + count && r == cudaSuccess; ++l)
        r = swept::launch_naive_step(p->stencil, p->dtype, tape_at(ring, L, H, N, l - 1),
                                     tape_at(ring, L, H, N, l), N, p->c, s, p->pdl != 0);
    }
    return r;
  };
  // the sweep: swept_advance's stage schedule on lam, transposed stencil;
  // sweep level tau reads forward level F - tau
  unsigned char* buf[2] = {p->edges, p->edges + p->edge_half};
  StageArgs a{};
  a.u = lam;
  a.N = N;
  a.nwin = p->nwin;
  a.c = p->c;
  a.tape = ring;
  a.tape_len = F;
  a.tape_ring = (int)L.ring;
  a.tape_h = (int)H;
  a.tape_rem = (int)L.rem;
  a.pdl = p->pdl;
  auto stage = [&](int64_t k, int hv, int ht, int64_t need) -> cudaError_t {
    cudaError_t r = recompute_down_to(need);
    if (r != cudaSuccess) return r;
    a.offset = (k & 1) ? p->B / 2 : 0;
    a.hv = hv;
    a.ht = ht;
    a.ein = buf[(k + 1) & 1];
    a.eout = buf[k & 1];
    a.lev_fill = k >= 1 ? (k - 1) * H : 0;
    a.lev_trap = k * H;
    const bool full = use_ring(p) && p->nreg > 0 && hv == p->H && ht == p->H;
    const int w = (p->diamond == SWEPT_DIAMOND_AUTO && p->ring_warps == 0) ? -1 : p->ring_warps;
    if (p->nreg == p->nwin)
      return full ? swept::launch_ring_ksadj_f64(p->K, a, w, s) : swept::launch_stage_ksadj_f64(p->K, a, s);
    // uneven tiles: the regular windows, then the wide ones
    if (p->nreg > 0) {
      a.nlaunch = p->nreg;
      r = full ? swept::launch_ring_ksadj_f64(p->K, a, w, s) : swept::launch_stage_ksadj_f64(p->K, a, s);
      a.nlaunch = 0;
    }
    if (r == cudaSuccess) r = swept::launch_wide_ksadj(p->K, a, p->nreg, (int)(k & 1), s);
    return r;
  };
  const int64_t q = L.q;
  const int rem = (int)L.rem;
  if (q == 0) {
    e = stage(0, 0, rem, -1);
    if (e == cudaSuccess) e = stage(1, rem, 0, -1);
  } else {
    e = stage(0, 0, (int)H, q - 1);
    for (int64_t k = 1; k < q && e == cudaSuccess; ++k) e = stage(k, (int)H, (int)H, q - k - 1);
    if (e == cudaSuccess) e = stage(q, (int)H, rem, rem > 0 ? -1 : 0);
    if (e == cudaSuccess && rem > 0) e = stage(q + 1, rem, 0, -1);
  }
  return cuda_status(e);
}

}  // namespace

extern "C" {

int swept_adjoint_scratch(swept_plan_t p, int64_t nsteps, int K_cycles, int64_t* bytes) {
  if (!p || !bytes || nsteps < 0) return SWEPT_EINVAL;
  if (p->dtype != SWEPT_F64 || p->subs > 1) return SWEPT_ENOTSUP;
  *bytes = 0;
  if (p->stencil == SWEPT_KS && nsteps > 0)
    *bytes = adjoint_layout(p, nsteps, K_cycles).states * p->N * (int64_t)sizeof(double);
  return SWEPT_OK;
}

int swept_adjoint(swept_plan_t p, const void* u0, const void* lam_T, void* grad, int64_t nsteps,
                  int K_cycles, void* stream) {
  if (!p || !u0 || !lam_T || !grad || nsteps < 0) return SWEPT_EINVAL;
  if (!aligned16(u0) || !aligned16(lam_T) || !aligned16(grad)) return SWEPT_EINVAL;
  if (p->dtype != SWEPT_F64 || p->subs > 1) return SWEPT_ENOTSUP;
  cudaStream_t s = (cudaStream_t)stream;
  if (!swept::call_on_device(p->device, s, {u0, lam_T, grad})) return SWEPT_EINVAL;
  if (u0 == grad) return SWEPT_EINVAL;
  const size_t bytes = (size_t)p->N * sizeof(double);
  cudaError_t e = cudaMemcpyAsync(grad, lam_T, bytes, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess || nsteps == 0) return cuda_status(e);
  if (p->stencil == SWEPT_HEAT) {
    // dPhi = I + r L2 is symmetric and its transpose applied to lam is the
    // same update with the same rounding: the adjoint is the forward sweep.
    return swept_advance(p, grad, nsteps, stream);
  }
  if (nsteps > 0x7fffffff) return SWEPT_EINVAL;     // tape levels are 32-bit indices
  const AdjLayout L = adjoint_layout(p, nsteps, K_cycles);
  const size_t need = (size_t)L.states * bytes;
  if (p->adj_bytes < need) {
    cudaStreamSynchronize(s);
    if (p->adj) cudaFree(p->adj);
    p->adj = nullptr;
    p->adj_bytes = 0;
    e = cudaMalloc((void**)&p->adj, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_status(e);
    }
    p->adj_bytes = need;
  }
  return adjoint_ks(p, static_cast<const double*>(u0), static_cast<double*>(grad), nsteps, L, p->adj, s);
}

int swept_naive_advance(swept_plan_t p, void* u, int64_t nsteps, void* stream) {
  if (!p || !u || nsteps < 0 || !aligned16(u)) return SWEPT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (!swept::call_on_device(p->device, s, {u})) return SWEPT_EINVAL;
  if (p->stencil == SWEPT_EULER && p->dtype == SWEPT_F32C) {
    // per time step: q_mid = hi + (lo - dt/(2dx) dF(hi)) into scratch, then
    // (hi', lo') = TwoSum(hi, lo - dt/dx dF(q_mid)) into scratch, swap
    const int64_t N = p->N;
    float* qm = reinterpret_cast<float*>(p->edges);
    float* bufs[2] = {static_cast<float*>(u), qm + 3 * N};
    const float cf = p->c.dtdx32, ch = 0.5f * p->c.dtdx32, g1 = p->c.g132;
    cudaError_t e = cudaSuccess;
    int cur = 0;
    for (int64_t k = 0; k < nsteps && e == cudaSuccess; ++k) {
      const float* hi = bufs[cur];
      const float* lo = bufs[cur] + 3 * N;
      e = swept::launch_naive_euler_f32c(0, hi, hi, lo, qm, nullptr, N, ch, g1, s, p->pdl != 0);
      if (e == cudaSuccess)
        e = swept::launch_naive_euler_f32c(1, qm, hi, lo, bufs[cur ^ 1], bufs[cur ^ 1] + 3 * N, N, cf, g1, s,
                                           p->pdl != 0);
      cur ^= 1;
    }
    if (e == cudaSuccess && cur == 1)
      e = cudaMemcpyAsync(u, bufs[1], (size_t)N * 6 * sizeof(float), cudaMemcpyDeviceToDevice, s);
    return cuda_status(e);
  }
  if (p->stencil == SWEPT_EULER) {
    // per time step: q_mid = q - dt/(2dx) dF(q) into scratch, then
    // q' = q - dt/dx dF(q_mid) into scratch, swap
    const int64_t N = p->N;
    double* qm = reinterpret_cast<double*>(p->edges);
    double* bufs[2] = {static_cast<double*>(u), qm + 3 * N};
    const double half = 0.5 * p->c.dtdx;
    cudaError_t e = cudaSuccess;
    int cur = 0;
    for (int64_t k = 0; k < nsteps && e == cudaSuccess; ++k) {
      e = swept::launch_naive_euler(bufs[cur], bufs[cur], qm, N, half, p->c.g1, s, p->pdl != 0);
      if (e == cudaSuccess)
        e = swept::launch_naive_euler(qm, bufs[cur], bufs[cur ^ 1], N, p->c.dtdx, p->c.g1, s, p->pdl != 0);
      cur ^= 1;
    }
    if (e == cudaSuccess && cur == 1)
      e = cudaMemcpyAsync(u, bufs[1], (size_t)N * 3 * sizeof(double), cudaMemcpyDeviceToDevice, s);
    return cuda_status(e);
  }
  if (p->rk2) {
    // per time step: m = A(u) into scratch, then u' = B(u, m) into scratch, swap
    double* m = reinterpret_cast<double*>(p->edges);
    double* bufs[2] = {static_cast<double*>(u), m + p->N};
    cudaError_t e = cudaSuccess;
    int cur = 0;
    for (int64_t k = 0; k < nsteps && e == cudaSuccess; ++k) {
      e = swept::launch_naive_rk2(p->stencil, 0, bufs[cur], nullptr, m, p->N, p->c, s, p->pdl != 0);
      if (e == cudaSuccess)
        e = swept::launch_naive_rk2(p->stencil, 1, bufs[cur], m, bufs[cur ^ 1], p->N, p->c, s, p->pdl != 0);
      cur ^= 1;
    }
    if (e == cudaSuccess && cur == 1)
      e = cudaMemcpyAsync(u, bufs[1], (size_t)p->N * 8, cudaMemcpyDeviceToDevice, s);
    return cuda_status(e);
  }
  if (p->naive_resident && nsteps > 0) {
    const int st = p->stencil == SWEPT_HEAT ? swept::kHeat : swept::kKS;
    int fits = 0;
    cudaError_t e = swept::launch_naive_resident(st, p->dtype, u, p->N, p->c, nsteps, s, false, true, &fits);
    if (e != cudaSuccess) return cuda_status(e);
    if (fits) return cuda_status(swept::launch_naive_resident(st, p->dtype, u, p->N, p->c, nsteps, s, p->pdl != 0,
                                                               false, nullptr));
  }
  void* bufs[2] = {u, p->edges};
  cudaError_t e = cudaSuccess;
  int cur = 0;
  for (int64_t k = 0; k < nsteps && e == cudaSuccess; ++k) {
    e = swept::launch_naive_step(p->stencil, p->dtype, bufs[cur], bufs[cur ^ 1], p->N, p->c, s, p->pdl != 0);
    cur ^= 1;
  }
  if (e == cudaSuccess && cur == 1) {
    const size_t bytes = (size_t)p->N * (p->dtype == SWEPT_F32 ? 4 : 8);   // F64, F32C: 8 B per point
    e = cudaMemcpyAsync(u, p->edges, bytes, cudaMemcpyDeviceToDevice, s);
  }
  return cuda_status(e);
}

int swept_stage(swept_plan_t p, void* u, int64_t k, int hv, int ht, void* stream) {
  if (!p || !u || k < 0 || !aligned16(u)) return SWEPT_EINVAL;
  if (hv < 0 || ht < 0 || hv > p->H || ht > p->H || (hv == 0 && ht == 0)) return SWEPT_EINVAL;
  if (p->nreg != p->nwin) return SWEPT_ENOTSUP;
  cudaStream_t s = (cudaStream_t)stream;
  if (!swept::call_on_device(p->device, s, {u})) return SWEPT_EINVAL;
  // the same stage as swept_advance's stage k: windows shifted by B/2 when k
  // is odd, edges of stage k-1 in buffer (k+1) & 1, its own in buffer k & 1
  unsigned char* buf[2] = {p->edges, p->edges + p->edge_half};
  StageArgs a{};
  a.u = u;
  a.N = p->N;
  a.nwin = p->nwin;
  a.c = p->c;
  a.pdl = p->pdl;
  a.offset = (k & 1) ? p->B / 2 : 0;
  a.hv = hv;
  a.ht = ht;
  a.ein = buf[(k + 1) & 1];
  a.eout = buf[k & 1];
  a.lev_fill = k >= 1 ? (k - 1) * p->H : 0;
  a.lev_trap = k * p->H;
  const bool full = use_ring(p) && hv == p->H && ht == p->H;
  return cuda_status(full ? launch_ring(p, a, s) : launch_stage(p, a, s));
}

int swept_edge_copy(swept_plan_t p, int64_t k, int window, int side, void* buf, int dir, void* stream) {
  if (!p || !buf || k < 0 || window < 0 || window >= p->nwin || (side != 0 && side != 1)) return SWEPT_EINVAL;
  if ((dir != 0 && dir != 1) || p->nreg != p->nwin) return SWEPT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (!swept::call_on_device(p->device, s, {buf})) return SWEPT_EINVAL;
  // one window's slot is 2B elements: B of left edges (h levels x 2r), then B of right edges
  const size_t half = p->edge_half / ((size_t)p->nwin * 2);
  unsigned char* e = p->edges + (size_t)(k & 1) * p->edge_half + ((size_t)window * 2 + side) * half;
  cudaError_t r = dir == 0 ? cudaMemcpyAsync(buf, e, half, cudaMemcpyDeviceToDevice, s)
                           : cudaMemcpyAsync(e, buf, half, cudaMemcpyDeviceToDevice, s);
  return cuda_status(r);
}

int swept_plan_last_advance(swept_plan_t p, int64_t* launches, int64_t* ring_launches, double* ring_ms) {
  if (!p || !launches || !ring_launches || !ring_ms) return SWEPT_EINVAL;
  *launches = p->last_launches;
  *ring_launches = p->last_ring_launches;
  *ring_ms = -1.0;
  if (p->time_ring && p->ring_timed) {
    float ms = 0.0f;
    cudaError_t e = cudaEventSynchronize(p->ring_ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p->ring_ev[0], p->ring_ev[1]);
    if (e != cudaSuccess) return cuda_status(e);
    *ring_ms = ms;
  }
  return SWEPT_OK;
}

int swept_plan_status(swept_plan_t p, void* stream) {
  if (!p) return SWEPT_EINVAL;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return SWEPT_ECUDA;
  int st = 0;
  if (cudaMemcpy(&st, p->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SWEPT_ECUDA;
  return st;
}

int swept_f32c_split(int64_t N, const double* u64, void* u32c, void* stream) {
  if (N <= 0 || !u64 || !u32c) return SWEPT_EINVAL;
  if (!swept::call_on_device(-1, (cudaStream_t)stream, {u64, u32c})) return SWEPT_EINVAL;
  return cuda_status(swept::launch_split(N, u64, (float*)u32c, (cudaStream_t)stream));
}

int swept_f32c_merge(int64_t N, const void* u32c, double* u64, void* stream) {
  if (N <= 0 || !u64 || !u32c) return SWEPT_EINVAL;
  if (!swept::call_on_device(-1, (cudaStream_t)stream, {u64, u32c})) return SWEPT_EINVAL;
  return cuda_status(swept::launch_merge(N, (const float*)u32c, u64, (cudaStream_t)stream));
}

int swept_reduce(swept_plan_t p, const void* u, int what, const void* v, double* out, void* stream) {
  if (!p || !u || !out) return SWEPT_EINVAL;
  if (what < SWEPT_SUM || what > SWEPT_DOT) return SWEPT_EINVAL;
  if (what == SWEPT_DOT && !v) return SWEPT_EINVAL;
  if (!swept::call_on_device(p->device, (cudaStream_t)stream, {u, what == SWEPT_DOT ? v : nullptr, out}))
    return SWEPT_EINVAL;
  return cuda_status(swept::launch_reduce(p->dtype, u, what, (const double*)v, p->N, p->red, out,
                                          (cudaStream_t)stream));
}

}  // extern "C"
