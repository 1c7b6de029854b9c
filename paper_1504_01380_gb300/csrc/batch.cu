// Batched persistent swept launch: many independent periodic problems of
// uneven length and step count advanced by one kernel launch.
//
// Work items are (problem, run of up to RL consecutive windows, stage), one
// swept stage of those windows (Section 3's per-node stage), processed by one
// warp: full diamond stages stream the run through the ring-pipelined kernel
// code (fill of one window overlapped with the triangle of the previous);
// other stages (first triangle, last fill, remainder) go window by window with
// the per-window stage code.  Items are handed out by one atomic
// counter in stage-major order over the whole batch: every stage-s item of
// every problem precedes every stage-(s+1) item.  A stage-s item (s >= 1)
// reads the leading edges of the two stage-(s-1) windows it straddles, so it
// waits until both have published: each window has a counter of completed
// stages, written with release semantics after its edges, and read with
// acquire semantics.  Items are only waited on by later items and the queue
// order puts every dependency before its dependant, and warps take items
// only while running, so the waits always end unless something is lost; as a
// guard every wait has a clock budget after which the warp records
// SWEPT_ETIMEOUT in a status word and stops, and the other warps stop taking
// work once the status is set.  No wait is unbounded.
//
// The same wait also protects the edge double buffer from being overwritten
// early: window w's stage-(s+2) edges go where its stage-s edges were, and
// the windows that read those (stage s+1, straddling w) are exactly the ones
// w's stage-(s+2) item waits for.
//
// Problems are sorted by stage count (descending) so that the problems still
// active at stage s are a prefix; an item index decodes to (stage, problem,
// window) by two binary searches over small tables.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>

#include "swept.h"
#include "swept_internal.h"
#include "swept_ring.cuh"
#include "swept_stage.cuh"
#include "swept_sync.cuh"

namespace swept {

struct BatchProblem {
  int64_t u_off;          // byte offset of the state in the pool
  int64_t e_off;          // byte offset of the edge double buffer in the plan's edge pool
  int64_t f_off;          // index of the first window counter
  int64_t N;
  int nwin, B, H, stencil, q, rem, nstages, nruns;
  Consts c;
};

struct BatchArgs {
  unsigned char* pool;
  unsigned char* edges;
  int* flags;
  const BatchProblem* probs;    // sorted by nstages, descending
  const int64_t* cum;           // nprob + 1: runs before problem i (sorted order)
  const int* nactive;           // per stage: problems still active (a prefix)
  const int64_t* stage_start;   // nstage_max + 1: first item of each stage
  int nstage_max;
  int64_t nitems;
  unsigned long long* counter;
  int* status;
  long long timeout_cycles;
  int64_t drop_item;            // item whose first window never publishes (-1: none)
  int run_len;                  // windows per item
};

namespace {

template <class T>
__device__ __forceinline__ int upper_index(const T* a, int n, T x) {
  // largest i in [0, n) with a[i] <= x (a ascending, a[0] <= x)
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}


// Dependence hooks of one item: wait (bounded) for the two windows of the
// previous stage a window reads from; publish a window after its edges.
struct BatchHooks {
  int* flags;
  int* status;
  long long budget;
  int s, nwin, offset, lane;
  int drop_w;                   // window that must not publish (-1: none)
  __device__ __forceinline__ bool ready(int w) const {
    if (s == 0) return true;
    const int wl = offset ? w : (w == 0 ? nwin - 1 : w - 1);
    const int wr = offset ? (w + 1 == nwin ? 0 : w + 1) : w;
    const long long t0 = clock64();
    bool ok = wait_ge(flags + wl, s, t0, budget);
    if (ok) ok = wait_ge(flags + wr, s, t0, budget);
    ok = __all_sync(kFull, ok);
    if (!ok && lane == 0) atomicCAS(status, 0, SWEPT_ETIMEOUT);
    return ok;
  }
  __device__ __forceinline__ void done(int w) const {
    __threadfence();
    __syncwarp();
    if (lane == 0 && w != drop_w) st_release(flags + w, s + 1);
  }
};

template <int ST, class DT, int K>
__device__ __forceinline__ bool batch_item(const StageArgs& a, typename DT::E* sm, int w0, int w1,
                                           const BatchHooks& hk, int H) {
  if (a.hv == H && a.ht == H) return RingImpl<ST, DT, K>::run_hooked(a, sm, w0, w1, hk);
  for (int w = w0; w < w1; ++w) {
    if (!hk.ready(w)) return false;
    StageImpl<ST, DT, K>::run_window(a, sm, w);
    hk.done(w);
  }
  return true;
}

// Blocks per SM the batch kernel declares for the compensated state: 5 (a
// budget of 102 registers, of which it uses 96 with a few spills; the
// allocator would otherwise take 120 and leave 4 blocks).  Measured on GB300, 4096 problems, B = 256 / 512: 4 blocks
// 1.53e12, 5 blocks 1.58e12, 6 blocks (80 registers) 1.39e12 cell-updates/s.
template <class DT> struct BatchBlocks { static constexpr int value = 0; };
template <> struct BatchBlocks<F32C> { static constexpr int value = 5; };

template <class DT, int KH, int KK>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, BatchBlocks<DT>::value)
swept_batch_kernel(const BatchArgs ba) {
  using E = typename DT::E;
  constexpr int BMAX = 32 * (KH > KK ? KH : KK);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  E* sm = reinterpret_cast<E*>(smem_raw) + (threadIdx.x >> 5) * (2 * BMAX);
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long idx = 0;
    if (lane == 0) idx = atomicAdd(ba.counter, 1ull);
    idx = __shfl_sync(kFull, idx, 0);
    if ((int64_t)idx >= ba.nitems) return;
    if (ld_acquire(ba.status) != 0) return;
    const int s = upper_index<int64_t>(ba.stage_start, ba.nstage_max, (int64_t)idx);
    const int64_t k = (int64_t)idx - ba.stage_start[s];
    const int i = upper_index<int64_t>(ba.cum, ba.nactive[s], k);
    const int run = (int)(k - ba.cum[i]);
    const BatchProblem P = ba.probs[i];
    const int w0 = run * ba.run_len;
    const int w1 = min(w0 + ba.run_len, P.nwin);
    StageArgs a{};
    a.u = ba.pool + P.u_off;
    a.N = P.N;
    a.nwin = P.nwin;
    a.offset = (s & 1) ? P.B / 2 : 0;
    stage_shape(s, P.q, P.rem, P.H, a.hv, a.ht);
    const int64_t half = (int64_t)P.nwin * 2 * P.B * 8;
    unsigned char* eb = ba.edges + P.e_off;
    a.ein = eb + ((s + 1) & 1) * half;
    a.eout = eb + (s & 1) * half;
    a.c = P.c;
    BatchHooks hk;
    hk.flags = ba.flags + P.f_off;
    hk.status = ba.status;
    hk.budget = ba.timeout_cycles;
    hk.s = s;
    hk.nwin = P.nwin;
    hk.offset = a.offset;
    hk.lane = lane;
    hk.drop_w = (int64_t)idx == ba.drop_item ? w0 : -1;
    const bool ok = P.stencil == kHeat ? batch_item<kHeat, DT, KH>(a, sm, w0, w1, hk, P.H)
                                       : batch_item<kKS, DT, KK>(a, sm, w0, w1, hk, P.H);
    if (!ok) return;
  }
}

template <class DT, int KH, int KK>
cudaError_t launch_batch_t(const BatchArgs& ba, int grid, cudaStream_t s, bool query, int* capacity) {
  constexpr int BMAX = 32 * (KH > KK ? KH : KK);
  const size_t smem = stage_smem_bytes(BMAX);
  cudaError_t e = cudaFuncSetAttribute(swept_batch_kernel<DT, KH, KK>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (query) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, swept_batch_kernel<DT, KH, KK>,
                                                      kWarpsPerBlock * 32, smem);
    *capacity = sms * (per_sm > 0 ? per_sm : 1);
    return e;
  }
  swept_batch_kernel<DT, KH, KK><<<grid, kWarpsPerBlock * 32, smem, s>>>(ba);
  return cudaGetLastError();
}

// Tile widths built for the batch: heat and KS each B in {256, 512}.
template <class DT>
cudaError_t launch_batch_dt(int KH, int KK, const BatchArgs& ba, int grid, cudaStream_t s, bool query,
                            int* cap) {
  if (KH == 8 && KK == 8) return launch_batch_t<DT, 8, 8>(ba, grid, s, query, cap);
  if (KH == 8 && KK == 16) return launch_batch_t<DT, 8, 16>(ba, grid, s, query, cap);
  if (KH == 16 && KK == 8) return launch_batch_t<DT, 16, 8>(ba, grid, s, query, cap);
  if (KH == 16 && KK == 16) return launch_batch_t<DT, 16, 16>(ba, grid, s, query, cap);
  return cudaErrorInvalidValue;
}

cudaError_t launch_batch(int dtype, int KH, int KK, const BatchArgs& ba, int grid, cudaStream_t s,
                         bool query, int* cap) {
  return dtype == SWEPT_F64 ? launch_batch_dt<F64>(KH, KK, ba, grid, s, query, cap)
                            : launch_batch_dt<F32C>(KH, KK, ba, grid, s, query, cap);
}

// ---------------------------------------------------------------------------
// Naive batched stepper: the stronger per-step baseline for a batch.  One
// launch per time step covers every problem that still has steps left (the
// problems sorted by step count, descending, so the active ones are a
// prefix); each thread advances 4 consecutive points of one problem with the
// same Core as the swept kernels, reading its halo straight from global
// memory (periodic within its problem).  The state ping-pongs between the
// pool and a scratch pool of the same layout.
struct NaiveProb {
  int64_t u_off, N, nsteps;
  int stencil;
  Consts c;
};

constexpr int kNaiveV = 4;
constexpr int kNaiveBT = 256;

template <class DT> __device__ __forceinline__ typename DT::C hi_point(const unsigned char* u, int64_t g);
template <> __device__ __forceinline__ double hi_point<F64>(const unsigned char* u, int64_t g) {
  return reinterpret_cast<const double*>(u)[g];
}
template <> __device__ __forceinline__ float hi_point<F32C>(const unsigned char* u, int64_t g) {
  return reinterpret_cast<const float*>(u)[g];
}

// Problem of chunk c: the i with cstart[i] <= c < cstart[i + 1].
__device__ __forceinline__ int chunk_problem(const int64_t* cstart, int n, int64_t c) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (cstart[mid] <= c) lo = mid;
    else hi = mid;
  }
  return lo;
}

template <int ST, class DT>
__device__ __forceinline__ void naive_points(const NaiveProb& P, const unsigned char* src, unsigned char* dst,
                                             int64_t g) {
  constexpr int R = Radius<ST>::value;
  using Cc = typename DT::C;
  const unsigned char* u = src + P.u_off;
  Tile<DT, kNaiveV> t;
  load_points<kNaiveV>(t, u, P.N, g);
  Cc x[kNaiveV + 2 * R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    int64_t gl = g - R + i;
    if (gl < 0) gl += P.N;
    int64_t gr = g + kNaiveV + i;
    if (gr >= P.N) gr -= P.N;
    x[i] = hi_point<DT>(u, gl);
    x[R + kNaiveV + i] = hi_point<DT>(u, gr);
  }
#pragma unroll
  for (int k = 0; k < kNaiveV; ++k) x[R + k] = t.hi(k);
  Core<ST, DT, kNaiveV>::apply(t, x, P.c);
  store_points<kNaiveV>(t, dst + P.u_off, P.N, g);
}

template <class DT>
__global__ void __launch_bounds__(kNaiveBT)
batch_naive_kernel(const NaiveProb* __restrict__ probs, const int64_t* __restrict__ cstart, int nact,
                   const unsigned char* __restrict__ src, unsigned char* __restrict__ dst) {
  const int64_t c = (int64_t)blockIdx.x * kNaiveBT + threadIdx.x;
  if (c >= cstart[nact]) return;
  const int i = chunk_problem(cstart, nact + 1, c);
  const NaiveProb& P = probs[i];
  const int64_t g = (c - cstart[i]) * kNaiveV;
  if (P.stencil == kHeat) naive_points<kHeat, DT>(P, src, dst, g);
  else naive_points<kKS, DT>(P, src, dst, g);
}

// Problems whose step count is odd end in the scratch pool: copy their
// 8N bytes back (one thread per 4 points = 32 bytes).
__global__ void __launch_bounds__(kNaiveBT)
batch_copy_odd_kernel(const NaiveProb* __restrict__ probs, const int64_t* __restrict__ cstart, int nprob,
                      const unsigned char* __restrict__ scratch, unsigned char* __restrict__ pool) {
  const int64_t c = (int64_t)blockIdx.x * kNaiveBT + threadIdx.x;
  if (c >= cstart[nprob]) return;
  const int i = chunk_problem(cstart, nprob + 1, c);
  const NaiveProb& P = probs[i];
  if ((P.nsteps & 1) == 0) return;
  const int64_t byte = P.u_off + (c - cstart[i]) * 32;
  const uint4* s4 = reinterpret_cast<const uint4*>(scratch + byte);
  uint4* d4 = reinterpret_cast<uint4*>(pool + byte);
  d4[0] = s4[0];
  d4[1] = s4[1];
}

cudaError_t launch_batch_naive_step(int dtype, const NaiveProb* probs, const int64_t* cstart, int nact,
                                    int64_t nchunks, const unsigned char* src, unsigned char* dst,
                                    cudaStream_t s) {
  const int64_t grid = (nchunks + kNaiveBT - 1) / kNaiveBT;
  if (grid == 0) return cudaSuccess;
  if (dtype == SWEPT_F64)
    batch_naive_kernel<F64><<<(unsigned)grid, kNaiveBT, 0, s>>>(probs, cstart, nact, src, dst);
  else
    batch_naive_kernel<F32C><<<(unsigned)grid, kNaiveBT, 0, s>>>(probs, cstart, nact, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_batch_copy_odd(const NaiveProb* probs, const int64_t* cstart, int nprob, int64_t nchunks,
                                  const unsigned char* scratch, unsigned char* pool, cudaStream_t s) {
  const int64_t grid = (nchunks + kNaiveBT - 1) / kNaiveBT;
  if (grid == 0) return cudaSuccess;
  batch_copy_odd_kernel<<<(unsigned)grid, kNaiveBT, 0, s>>>(probs, cstart, nprob, scratch, pool);
  return cudaGetLastError();
}

}  // namespace
}  // namespace swept

using swept::BatchArgs;
using swept::BatchProblem;

struct swept_batch_s {
  int nprob, dtype, B_heat, B_ks, nstage_max, grid;
  int run_len;                  // windows per work item
  int device;                   // the CUDA device the batch was planned on
  int64_t nitems, total_windows, pool_bytes;
  BatchProblem* h_probs;        // host copy, sorted by stage count (descending)
  unsigned char* edges;
  int* flags;
  BatchProblem* d_probs;
  int64_t* d_cum;
  int* d_nactive;
  int64_t* d_stage_start;
  unsigned long long* d_counter;
  int* d_status;
  double timeout_s;
  int64_t drop_item;
  int use_graph;                // 1 (default): replay a captured graph
  // graph of one advance (memsets + the launch), rebuilt when the pool changes
  cudaGraphExec_t exec;
  void* graph_pool;
  bool graph_valid;
  // naive batched stepper: problems by step count (descending), chunk
  // prefix (4 points per chunk), host copy of the sorted step counts and
  // of the prefix, scratch pool (allocated on first use)
  swept::NaiveProb* d_nv;
  int64_t* d_nv_cstart;
  int64_t* h_nv_steps;
  int64_t* h_nv_cstart;
  unsigned char* nv_scratch;
};

namespace {

// Windows per work item: the ring pays one extra slot per item, so an item of
// n windows keeps 1/(n + 1) of its slots partly idle; longer items leave fewer
// items per stage to spread over the warps and to hide the waits at stage
// transitions.  The plan takes the longest of 32, 16 and 8 that leaves at
// least 8 items per resident warp in stage 0 (measured on GB300, 4096 ragged
// problems, 2432 warps: runs of 8 1.45e12, 16 1.53e12 (13 items per warp),
// 32 1.45e12 cell-updates/s).
constexpr int kRunLens[3] = {32, 16, 8};
constexpr int kItemsPerWarp = 8;

int cuda_status_b(cudaError_t e) {
  if (e == cudaSuccess) return SWEPT_OK;
  if (e == cudaErrorMemoryAllocation) return SWEPT_ENOMEM;
  return SWEPT_ECUDA;
}

int batch_consts(int stencil, const double* p, swept::Consts& c) {
  std::memset(&c, 0, sizeof c);
  if (stencil == SWEPT_HEAT) {
    c.r = p[0];
    c.r32 = (float)c.r;
    return SWEPT_OK;
  }
  if (!(p[1] > 0.0)) return SWEPT_EINVAL;
  const double dt = p[0], dx = p[1], dx2 = dx * dx;
  c.a = -(dt / (4.0 * dx));
  c.b = -(dt / dx2);
  c.e = -(dt / (dx2 * dx2));
  c.a32 = (float)c.a;
  c.b32 = (float)c.b;
  c.e32 = (float)c.e;
  return SWEPT_OK;
}

void free_batch(swept_batch_s* b) {
  if (!b) return;
  if (b->graph_valid) cudaGraphExecDestroy(b->exec);
  cudaFree(b->edges);
  cudaFree(b->flags);
  cudaFree(b->d_probs);
  cudaFree(b->d_cum);
  cudaFree(b->d_nactive);
  cudaFree(b->d_stage_start);
  cudaFree(b->d_counter);
  cudaFree(b->d_status);
  cudaFree(b->d_nv);
  cudaFree(b->d_nv_cstart);
  cudaFree(b->nv_scratch);
  std::free(b->h_nv_steps);
  std::free(b->h_nv_cstart);
  std::free(b->h_probs);
  std::free(b);
}

BatchArgs make_args(const swept_batch_s* b, void* pool) {
  BatchArgs a;
  a.pool = static_cast<unsigned char*>(pool);
  a.edges = b->edges;
  a.flags = b->flags;
  a.probs = b->d_probs;
  a.cum = b->d_cum;
  a.nactive = b->d_nactive;
  a.stage_start = b->d_stage_start;
  a.nstage_max = b->nstage_max;
  a.nitems = b->nitems;
  a.counter = b->d_counter;
  a.status = b->d_status;
  int dev = 0, khz = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
  if (khz <= 0) khz = 2000000;
  a.timeout_cycles = (long long)(b->timeout_s * (double)khz * 1000.0);
  a.drop_item = b->drop_item;
  a.run_len = b->run_len;
  return a;
}

// Item tables for the plan's run length: runs per problem, their prefix over
// the sorted problems, the active prefix of each stage and the first item of
// each stage; uploaded over the device copies.
cudaError_t upload_tables(swept_batch_s* b) {
  const int nprob = b->nprob, nstage_max = b->nstage_max;
  for (int i = 0; i < nprob; ++i)
    b->h_probs[i].nruns = (b->h_probs[i].nwin + b->run_len - 1) / b->run_len;
  std::vector<int64_t> cum(nprob + 1, 0);
  for (int i = 0; i < nprob; ++i) cum[i + 1] = cum[i] + b->h_probs[i].nruns;
  std::vector<int> nactive(std::max(nstage_max, 1), 0);
  std::vector<int64_t> stage_start(nstage_max + 1, 0);
  for (int s = 0; s < nstage_max; ++s) {
    int n = 0;
    while (n < nprob && b->h_probs[n].nstages > s) ++n;
    nactive[s] = n;
    stage_start[s + 1] = stage_start[s] + cum[n];
  }
  b->nitems = stage_start[nstage_max];
  cudaError_t e = cudaMemcpy(b->d_probs, b->h_probs, sizeof(BatchProblem) * nprob, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_cum, cum.data(), sizeof(int64_t) * (nprob + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_nactive, nactive.data(), sizeof(int) * nactive.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_stage_start, stage_start.data(), sizeof(int64_t) * (nstage_max + 1),
                   cudaMemcpyHostToDevice);
  return e;
}

cudaError_t enqueue(swept_batch_s* b, void* pool, cudaStream_t s) {
  BatchArgs a = make_args(b, pool);
  cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_status, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->flags, 0, (size_t)b->total_windows * sizeof(int), s);
  if (e == cudaSuccess && b->nitems > 0)
    e = swept::launch_batch(b->dtype, b->B_heat / 32, b->B_ks / 32, a, b->grid, s, false, nullptr);
  return e;
}

}  // namespace

extern "C" {

int swept_batch_plan(swept_batch_t* out, int nprob, const swept_problem_t* probs, int dtype, int B_heat,
                     int B_ks) {
  if (!out || nprob <= 0 || !probs) return SWEPT_EINVAL;
  *out = nullptr;
  if (dtype != SWEPT_F64 && dtype != SWEPT_F32C) return SWEPT_EINVAL;
  if (B_heat == 0) B_heat = 512;
  if (B_ks == 0) B_ks = 512;
  if ((B_heat != 256 && B_heat != 512) || (B_ks != 256 && B_ks != 512)) return SWEPT_ENOTSUP;
  std::vector<BatchProblem> h(nprob);
  std::vector<swept::NaiveProb> nv(nprob);
  // resident blocks of the batch kernel (the default grid) and the run length
  int cap = 0;
  {
    BatchArgs none{};
    cudaError_t e = swept::launch_batch(dtype, B_heat / 32, B_ks / 32, none, 0, nullptr, true, &cap);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_status_b(e);
    }
  }
  int64_t windows = 0;
  for (int i = 0; i < nprob; ++i) {
    const int B = probs[i].stencil == SWEPT_HEAT ? B_heat : B_ks;
    if (B > 0 && probs[i].N > 0) windows += probs[i].N / B;
  }
  int run_len = kRunLens[2];
  for (int rl : kRunLens) {
    if (windows / rl >= (int64_t)kItemsPerWarp * swept::kWarpsPerBlock * (cap > 0 ? cap : 1)) {
      run_len = rl;
      break;
    }
  }
  int64_t e_off = 0, f_off = 0, extent = 16;
  for (int i = 0; i < nprob; ++i) {
    const swept_problem_t& p = probs[i];
    if (p.stencil != SWEPT_HEAT && p.stencil != SWEPT_KS) return SWEPT_EINVAL;
    const int B = p.stencil == SWEPT_HEAT ? B_heat : B_ks;
    const int R = p.stencil == SWEPT_HEAT ? 1 : 2;
    if (p.N <= 0 || p.N % B || p.nsteps < 0 || p.offset < 0 || (p.offset & 15)) return SWEPT_EINVAL;
    if (p.N / B > (int64_t)0x7fffffff) return SWEPT_EINVAL;
    BatchProblem& d = h[i];
    std::memset(&d, 0, sizeof d);
    if (batch_consts(p.stencil, p.params, d.c) != SWEPT_OK) return SWEPT_EINVAL;
    d.u_off = p.offset;
    d.N = p.N;
    d.nwin = (int)(p.N / B);
    d.B = B;
    d.H = B / (2 * R);
    d.stencil = p.stencil;
    d.q = (int)(p.nsteps / d.H);
    d.rem = (int)(p.nsteps % d.H);
    d.nstages = p.nsteps == 0 ? 0 : (d.q == 0 ? 2 : (d.rem ? d.q + 2 : d.q + 1));
    d.e_off = e_off;
    d.f_off = f_off;
    e_off += (int64_t)d.nwin * 2 * B * 8 * 2;
    f_off += d.nwin;
    nv[i].u_off = p.offset;
    nv[i].N = p.N;
    nv[i].nsteps = p.nsteps;
    nv[i].stencil = p.stencil;
    nv[i].c = d.c;
    extent = std::max<int64_t>(extent, p.offset + 8 * p.N);
  }
  std::stable_sort(nv.begin(), nv.end(),
                   [](const swept::NaiveProb& x, const swept::NaiveProb& y) { return x.nsteps > y.nsteps; });
  std::stable_sort(h.begin(), h.end(),
                   [](const BatchProblem& x, const BatchProblem& y) { return x.nstages > y.nstages; });
  const int nstage_max = h[0].nstages;
  swept_batch_s* b = (swept_batch_s*)std::calloc(1, sizeof(swept_batch_s));
  if (!b) return SWEPT_ENOMEM;
  b->nprob = nprob;
  cudaGetDevice(&b->device);
  b->dtype = dtype;
  b->B_heat = B_heat;
  b->B_ks = B_ks;
  b->nstage_max = nstage_max;
  b->total_windows = f_off;
  b->timeout_s = 2.0;
  b->drop_item = -1;
  b->use_graph = 1;
  b->run_len = run_len;
  b->pool_bytes = extent;
  b->h_nv_steps = (int64_t*)std::malloc(sizeof(int64_t) * nprob);
  b->h_nv_cstart = (int64_t*)std::malloc(sizeof(int64_t) * (nprob + 1));
  b->h_probs = (BatchProblem*)std::malloc(sizeof(BatchProblem) * nprob);
  if (!b->h_nv_steps || !b->h_nv_cstart || !b->h_probs) {
    free_batch(b);
    return SWEPT_ENOMEM;
  }
  b->h_nv_cstart[0] = 0;
  for (int i = 0; i < nprob; ++i) {
    b->h_nv_steps[i] = nv[i].nsteps;
    b->h_nv_cstart[i + 1] = b->h_nv_cstart[i] + nv[i].N / 4;
  }
  cudaError_t e = cudaMalloc((void**)&b->edges, (size_t)std::max<int64_t>(e_off, 16));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_nv, sizeof(swept::NaiveProb) * nprob);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_nv_cstart, sizeof(int64_t) * (nprob + 1));
  if (e == cudaSuccess) e = cudaMemcpy(b->d_nv, nv.data(), sizeof(swept::NaiveProb) * nprob, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_nv_cstart, b->h_nv_cstart, sizeof(int64_t) * (nprob + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->flags, (size_t)std::max<int64_t>(f_off, 1) * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_probs, sizeof(BatchProblem) * nprob);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_cum, sizeof(int64_t) * (nprob + 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_nactive, sizeof(int) * std::max(nstage_max, 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_stage_start, sizeof(int64_t) * (nstage_max + 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_counter, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_status, sizeof(int));
  if (e == cudaSuccess) {
    std::copy(h.begin(), h.end(), b->h_probs);
    e = upload_tables(b);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_batch(b);
    return cuda_status_b(e);
  }
  b->grid = cap > 0 ? cap : 1;
  *out = b;
  return SWEPT_OK;
}

int swept_batch_set(swept_batch_t b, int option, double value) {
  if (!b) return SWEPT_EINVAL;
  if (option == SWEPT_BOPT_TIMEOUT_S) {
    if (!(value > 0.0) || value > 600.0) return SWEPT_EINVAL;
    b->timeout_s = value;
  } else if (option == SWEPT_BOPT_DROP_ITEM) {
    b->drop_item = (int64_t)value;
  } else if (option == SWEPT_BOPT_GRID) {
    if (value < 1 || value > 1e6) return SWEPT_EINVAL;
    b->grid = (int)value;
  } else if (option == SWEPT_BOPT_GRAPH) {
    if (value != 0 && value != 1) return SWEPT_EINVAL;
    b->use_graph = (int)value;
  } else if (option == SWEPT_BOPT_RUN_LEN) {
    if (value < 1 || value > 1024 || value != (double)(int)value) return SWEPT_EINVAL;
    cudaDeviceSynchronize();       // the tables may be in use by a launch in flight
    b->run_len = (int)value;
    const cudaError_t e = upload_tables(b);
    if (e != cudaSuccess) return cuda_status_b(e);
  } else {
    return SWEPT_EINVAL;
  }
  if (b->graph_valid) {            // the captured launch carries the old settings
    cudaGraphExecDestroy(b->exec);
    b->graph_valid = false;
  }
  return SWEPT_OK;
}

int swept_batch_info(swept_batch_t b, int64_t* info, int ninfo) {
  if (!b || !info) return SWEPT_EINVAL;
  const int64_t v[6] = {b->nitems, b->nstage_max, b->total_windows, b->grid, b->nprob, b->run_len};
  for (int i = 0; i < ninfo && i < 6; ++i) info[i] = v[i];
  return SWEPT_OK;
}

int swept_advance_batch(swept_batch_t b, void* pool, void* stream) {
  if (!b || !pool || ((uintptr_t)pool & 15u)) return SWEPT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (!swept::call_on_device(b->device, s, {pool})) return SWEPT_EINVAL;
  if (!b->use_graph) return cuda_status_b(enqueue(b, pool, s));
  if (!b->graph_valid || b->graph_pool != pool) {
    if (b->graph_valid) {
      cudaGraphExecDestroy(b->exec);
      b->graph_valid = false;
    }
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_status_b(e);
    cudaGraph_t g;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e2 = enqueue(b, pool, cs);
      e = cudaStreamEndCapture(cs, &g);
      if (e == cudaSuccess) e = e2;
      if (e == cudaSuccess) {
        e = cudaGraphInstantiate(&b->exec, g, 0);
        cudaGraphDestroy(g);
      }
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return cuda_status_b(e);
    b->graph_valid = true;
    b->graph_pool = pool;
  }
  return cuda_status_b(cudaGraphLaunch(b->exec, s));
}

int swept_batch_naive_advance(swept_batch_t b, void* pool, void* stream) {
  if (!b || !pool || ((uintptr_t)pool & 15u)) return SWEPT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (!swept::call_on_device(b->device, s, {pool})) return SWEPT_EINVAL;
  cudaError_t e = cudaSuccess;
  if (!b->nv_scratch) {
    e = cudaMalloc((void**)&b->nv_scratch, (size_t)b->pool_bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      b->nv_scratch = nullptr;
      return cuda_status_b(e);
    }
  }
  unsigned char* buf[2] = {static_cast<unsigned char*>(pool), b->nv_scratch};
  int nact = b->nprob;
  for (int64_t k = 0; e == cudaSuccess; ++k) {
    while (nact > 0 && b->h_nv_steps[nact - 1] <= k) --nact;    // active problems: a prefix
    if (nact == 0) break;
    e = swept::launch_batch_naive_step(b->dtype, b->d_nv, b->d_nv_cstart, nact, b->h_nv_cstart[nact],
                                       buf[k & 1], buf[(k + 1) & 1], s);
  }
  if (e == cudaSuccess)
    e = swept::launch_batch_copy_odd(b->d_nv, b->d_nv_cstart, b->nprob, b->h_nv_cstart[b->nprob],
                                     b->nv_scratch, static_cast<unsigned char*>(pool), s);
  return cuda_status_b(e);
}

int swept_batch_status(swept_batch_t b, void* stream) {
  if (!b) return SWEPT_EINVAL;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return SWEPT_ECUDA;
  int st = 0;
  e = cudaMemcpy(&st, b->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return SWEPT_ECUDA;
  return st;
}

void swept_batch_destroy(swept_batch_t b) {
  if (!b) return;
  cudaDeviceSynchronize();
  free_batch(b);
}

}  // extern "C"
