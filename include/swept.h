/*
 * swept.h -- C ABI of the swept-rule library for one NVIDIA GB300 (sm_103a).
 *
 * The library advances a 1D periodic field u by nsteps explicit sub-timesteps
 * of a local stencil.  The swept rule (Sections 3-4 of Alhubail & Wang,
 * "The swept rule for breaking the latency barrier in time advancing PDEs")
 * tiles space-time into shrinking triangles and diamonds so that each tile of
 * B points advances B/(2r) sub-timesteps on chip between exchanges of its
 * leading edges.  The result equals per-step stepping exactly.
 *
 * Conventions for every entry point
 *   - Return value: SWEPT_OK (0) or a negative SWEPT_E* code; nothing is
 *     thrown or aborted across the ABI.  swept_strerror() names a code.
 *   - Pointers documented as "device" must point to memory of the current
 *     CUDA device (or managed memory), 16-byte aligned; the caller owns
 *     them.  A plan or batch is used on the device it was made on, with a
 *     stream of that device.  Each entry point checks this before it
 *     enqueues anything and returns SWEPT_EINVAL otherwise (a kernel given
 *     another GPU's pointer would fault).  While the stream is being captured
 *     into a CUDA graph only the plan's device is checked (the pointer
 *     queries would end the capture): the caller vouches for the pointers.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls enqueue work on it and return without synchronising
 *     unless stated otherwise.
 *   - A plan is not thread-safe: concurrent calls on one plan, or calls on
 *     one plan from different streams without ordering, race on its scratch.
 *
 * State layout in device memory
 *   SWEPT_F64  : double u[N].
 *   SWEPT_F32C : float hi[N] followed by float lo[N] (8N bytes); the value
 *                of point i is hi[i] + lo[i] (compensated FP32).
 *   SWEPT_F32  : float u[N] (4N bytes).
 *   SWEPT_EULER plans: the conserved variables density, momentum, energy.
 *                FP64: double rho[N], m[N], E[N] (24N bytes).  F32C: float
 *                hi of rho, m, E (3N), then lo of rho, m, E (3N) (24N bytes):
 *                the F32C layout of the 3N values rho, m, E.
 */
#ifndef SWEPT_H
#define SWEPT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- enums ------------------------------------------------------------ */

/* Arithmetic of the state (Section 2 leaves precision open). */
#define SWEPT_F64   0   /* IEEE binary64 */
#define SWEPT_F32C  1   /* binary32 pair (hi, lo), TwoSum-compensated update */
#define SWEPT_F32   2   /* plain binary32, the FP64 expressions in binary32: a
                           diagnostic precision (forward-Euler heat and KS)   */

/* Stencils (the sub-timestep of Section 2, one per time level).
 *   SWEPT_HEAT: u_t = u_xx, 3-point forward Euler; radius 1;
 *               params[0] = r = dt/dx^2.
 *   SWEPT_KS  : u_t = -u u_x - u_xx - u_xxxx (Section 6), central
 *               differences with flux u^2/2 and the 3-point second
 *               difference applied twice, forward Euler; radius 2;
 *               params[0] = dt, params[1] = dx.                            */
#define SWEPT_HEAT  0
#define SWEPT_KS    1
/* Two-stage Runge-Kutta (midpoint) versions, FP64 only: one time step is two
 * sub-timesteps (Section 2), A: m = u + dt/2 f(u) (u is forwarded) and
 * B: u' = u + dt f(m), each of the stencil's radius; nsteps counts time
 * steps.  The state in memory is u (double[N]); (u, m) pairs exist on chip
 * and in the edge buffers.  Same parameters as the forward-Euler stencils. */
#define SWEPT_HEAT_RK2  2
#define SWEPT_KS_RK2    3
/* Euler equations of gas dynamics (Section 7), FP64 or SWEPT_F32C, radius 1:
 * q = (rho, m, E), p = (gamma - 1)(E - m^2/(2 rho)); second-order finite
 * volumes with minmod-limited slopes, interface flux = mean physical flux
 * minus the spectral radius of the Roe matrix times the jump, midpoint rule.
 * One time step is four sub-timesteps (Section 2): slopes of q, half-step
 * flux update into q_mid, slopes of q_mid, full-step flux update of q with
 * q_mid's fluxes.  nsteps counts time steps.  params = {dt, dx, gamma}
 * (nparams = 3, dx > 0, dt >= 0, gamma > 1).  FP64: B in {32, 64, 128},
 * 9-value point states (72 bytes) on chip and in the edge buffers.  F32C:
 * fluxes and slopes in binary32 from hi (and from a binary32 midpoint), the
 * full-step increment added to lo and renormalised by TwoSum, as in the
 * compensated heat and KS updates; B in {32, 64, 128, 256}, 12-float point
 * states (48 bytes). */
#define SWEPT_EULER     4

/* Status codes. */
#define SWEPT_OK         0
#define SWEPT_EINVAL    -1   /* bad argument: sizes, radius, null pointer   */
#define SWEPT_ENOMEM    -2   /* device allocation failed                    */
#define SWEPT_ECUDA     -3   /* a CUDA call or kernel launch failed         */
#define SWEPT_ETIMEOUT  -4   /* a device-side wait ran out (batched,
                                persistent or streamed launch)              */
#define SWEPT_ENOTSUP   -5   /* combination not built into this library     */
#define SWEPT_ETOOBIG   -6   /* problem larger than swept_advance_noalloc's
                                fixed scratch (N > SWEPT_NOALLOC_MAX_N)     */

/* Reductions for swept_reduce. */
#define SWEPT_SUM         0  /* sum_i u_i                 (Section 6 check) */
#define SWEPT_HALF_SUMSQ  1  /* J = 1/2 sum_i u_i^2                         */
#define SWEPT_DOT         2  /* sum_i u_i v_i                               */

typedef struct swept_plan_s *swept_plan_t;

/* ---- plan ------------------------------------------------------------- */

/*
 * swept_plan -- validate a problem and allocate its scratch.
 *
 * Defines the problem of Section 3: a periodic 1D grid of N points split
 * into N/B tiles of B points, each advanced by the stencil `stencil_id`
 * (radius `radius`, parameters `params[0..nparams)`) in arithmetic `dtype`.
 *   N       >= B, N % B == 0; or (Euler equations K <= 4 in FP64,
 *           8 compensated) any N at least nwide = ceil((N mod B)/(32 radius))
 *           tiles long: the last nwide windows are then wider than B (uneven
 *           tiles: their trapezoids keep the height h, their Vs stay B wide),
 *           all B + 32 radius points but the last, which takes the rest
 *           (B + 1 .. B + 32 radius points).  With B = 0 any N >= 32 (heat,
 *           Euler equations) or >= 64 (KS) is tiled.
 *   radius  must equal the stencil's radius (1 heat, 2 KS, either time
 *           integrator; 1 Euler equations).
 *   B       tile width: 32*K points with K in {1,2,4,8,16,32}, K % radius
 *           == 0 (Section 3 gives each node an even count of points; in
 *           general B % (2*radius) == 0).  B = 0 picks the measured
 *           default: the widest tile that divides N or tiles it unevenly, up
 *           to 1024 points from N = 2^22 on and 512 below (Euler equations:
 *           64 in FP64, 128 compensated).
 *   params  host pointer; copied.
 * Allocates the edge double-buffer (2 * 2N values, 32N bytes; 64N for the
 * Runge-Kutta pairs; 288N / 192N for FP64 / F32C Euler point states) on
 * the current device.
 * *out is set on success.
 * Errors: SWEPT_EINVAL, SWEPT_ENOTSUP, SWEPT_ENOMEM, SWEPT_ECUDA.
 */
int swept_plan(swept_plan_t *out, int64_t N, int radius, int stencil_id,
               const double *params, int nparams, int dtype, int B);

/* Release the plan and its device scratch (synchronises the device). */
void swept_destroy(swept_plan_t plan);

/* Query: B, h = B/(2 radius), N, dtype, stencil, radius in info[0..6). */
int swept_plan_info(swept_plan_t plan, int64_t *info, int ninfo);

/*
 * swept_plan_set -- tuning options of a plan (used by the autotuner and the
 * tests; results do not depend on them, only speed does).
 *   SWEPT_OPT_DIAMOND    kernel for full diamond stages:
 *                        SWEPT_DIAMOND_AUTO (default: the ring from 8
 *                        windows up, except that with automatic ring warps
 *                        the per-window kernel runs when there is at most one
 *                        window per warp scheduler, 4 per SM), SWEPT_DIAMOND_WINDOW
 *                        (one warp per window), SWEPT_DIAMOND_RING (one warp
 *                        streams a run of windows, overlapping the V-fill of
 *                        one with the triangle of the previous).
 *   SWEPT_OPT_RING_WARPS warps of a ring launch; 0 = min(resident warp slots,
 *                        N/B/2), and at most 4 per SM for heat and KS FP64 states.  A
 *                        streamed launch takes at most the resident warps and
 *                        at most N/B/3 (3 windows per warp or more).
 *   SWEPT_OPT_GRAPH      1: swept_advance captures its stage sequence into a
 *                        CUDA graph on the first call for a given (u, nsteps)
 *                        and replays it afterwards (fewer host launches: the
 *                        GPU's counterpart of the latency tau of Section 4);
 *                        0 (default): launch the stages directly.
 *   SWEPT_OPT_PDL        1 (default): consecutive kernels of an advance (stages;
 *                        the naive stepper's steps) are programmatic dependent
 *                        launches: the next kernel is prepared while the
 *                        previous one drains and waits for its results on the
 *                        device, hiding part of the launch gap; 0: plain launches.
 *   SWEPT_OPT_PERSISTENT 1: forward-Euler heat and KS advances with K <= 8 whose
 *                        windows can all be resident at once run every stage
 *                        in one launch, each warp waiting (bounded by
 *                        SWEPT_OPT_TIMEOUT_MS, default 2 s) on
 *                        device flags for the two windows it reads from before
 *                        each stage: no stage boundary at all (the latency
 *                        regime); other plans ignore it.  0 (default): off.
 *                        A wait that runs out ends the launch with the status
 *                        SWEPT_ETIMEOUT, read by swept_plan_status.
 *   SWEPT_OPT_STREAM     1 (default): an advance whose ring stages (full
 *                        diamonds, forward schemes; uneven tiles but for the
 *                        Euler equations, with one warp per wide window beside
 *                        the regular windows' runs and per-window counters)
 *                        number two or more runs them all in one cooperative
 *                        launch, where each warp's last slot of a stage is the
 *                        first slot of its next stage; warps then wait (bounded,
 *                        SWEPT_OPT_TIMEOUT_MS) on their right neighbour's slot
 *                        counter once per stage.  With the automatic kernel
 *                        choice (SWEPT_DIAMOND_AUTO, automatic warps) only where
 *                        it pays: runs of at most 16 windows per warp, or no
 *                        loss of resident blocks.  0: one ring launch per stage.
 *                        A wait that runs out records SWEPT_ETIMEOUT, read by
 *                        swept_plan_status.  Results do not depend on it.
 *   SWEPT_OPT_TIME_RING  1: each advance records CUDA events around its ring
 *                        launches (not while the stream is being captured),
 *                        read by swept_plan_last_advance.  0 (default): none.
 *   SWEPT_OPT_TIMEOUT_MS budget of each persistent or streamed wait,
 *                        1..600000 ms (2000).
 *   SWEPT_OPT_RESIDENT   1 (default): an advance of an evenly tiled heat or KS
 *                        plan (forward Euler with K <= 4, Runge-Kutta pairs
 *                        with K <= 2) of at most 64 windows, with the automatic
 *                        kernel choice (SWEPT_DIAMOND_AUTO, automatic warps) and
 *                        neither SWEPT_OPT_PERSISTENT nor SWEPT_OPT_DROP_WINDOW,
 *                        runs in one launch of one thread block cluster (at most
 *                        16 blocks of 4, 2 or 1 warps, one warp per window) when
 *                        the GPU can hold it: at the end of a stage each window
 *                        pushes its edges into the shared memory of the windows
 *                        that read them (distributed shared memory), and a
 *                        cluster barrier separates the stages (the latency
 *                        regime of Section 4, without a kernel launch or a
 *                        global-memory round trip per stage).  0: the per-stage
 *                        launches.
 *   SWEPT_OPT_NAIVE_RESIDENT 1: swept_naive_advance of a forward-Euler heat or
 *                        KS plan runs every step in one thread block cluster
 *                        when N splits into at most 16 parts of 4r to 4094
 *                        points (each block steps its part in shared memory
 *                        with r halo points its neighbours push to it, one cluster
 *                        barrier per step: the per-step counterpart of
 *                        SWEPT_OPT_RESIDENT); 0 (default): one launch per step.
 *   SWEPT_OPT_DROP_WINDOW failure injection: in the persistent advance window
 *                        `value`, in a streamed ring launch warp `value` (of
 *                        uneven tiles: window `value`), never publishes its
 *                        progress (a lost message), so the waits on it run
 *                        out; -1 (default) none.
 * Errors: SWEPT_EINVAL for an unknown option or value.
 */
#define SWEPT_OPT_DIAMOND     0
#define SWEPT_OPT_RING_WARPS  1
#define SWEPT_OPT_GRAPH       2
#define SWEPT_OPT_PDL         3
#define SWEPT_OPT_PERSISTENT  4
#define SWEPT_OPT_DROP_WINDOW 5
#define SWEPT_OPT_TIMEOUT_MS  6
#define SWEPT_OPT_STREAM      7
#define SWEPT_OPT_TIME_RING   8
#define SWEPT_OPT_RESIDENT    9
#define SWEPT_OPT_NAIVE_RESIDENT 10
#define SWEPT_DIAMOND_AUTO    0
#define SWEPT_DIAMOND_WINDOW  1
#define SWEPT_DIAMOND_RING    2
int swept_plan_set(swept_plan_t plan, int option, int64_t value);

/* ---- advance ---------------------------------------------------------- */

/*
 * swept_advance -- u <- u after nsteps sub-timesteps, by the swept rule.
 *
 * Stage 0 is the shrinking triangle of Section 3 on the tiles [jB, jB+B);
 * every later stage is a diamond on the windows shifted by B/2 from the
 * previous stage's (the alternating point sets of Section 3), started from
 * the V of leading edges that the two neighbouring triangles wrote to the
 * plan's edge buffer.  nsteps = q*h + rem (h = B/(2 radius)) takes q + 1
 * stages when rem == 0, q + 2 otherwise (the last stage ends with a
 * trapezoid of height rem and its fill).  Full diamond stages run on the
 * kernel chosen by SWEPT_OPT_DIAMOND; with SWEPT_OPT_STREAM they run as one
 * launch, so an advance is as few as 4 kernel launches.
 *   u       device, state layout of the plan's dtype, overwritten in place.
 *   nsteps  >= 0; 0 is a no-op.
 * Errors: SWEPT_EINVAL (null plan/u, nsteps < 0), SWEPT_ECUDA.
 */
int swept_advance(swept_plan_t plan, void *u, int64_t nsteps, void *stream);

/*
 * swept_naive_advance -- the same result by per-step stepping: one kernel
 * launch and one full read and write of u per sub-timestep (the "straight"
 * decomposition that Section 6 compares against).  Uses the plan's scratch
 * as the second buffer.  Euler plans take two launches per time step (each
 * fuses a slope sub-timestep with the flux sub-timestep that follows it).
 * Same arguments and errors as swept_advance.
 */
int swept_naive_advance(swept_plan_t plan, void *u, int64_t nsteps, void *stream);

/*
 * swept_plan_status -- synchronise `stream` and return the device status of
 * the plan's last persistent or streamed advance (SWEPT_OPT_PERSISTENT,
 * SWEPT_OPT_STREAM): SWEPT_OK or SWEPT_ETIMEOUT (a device wait ran out; the
 * state is then undefined).  Other advances leave it as it was.
 */
int swept_plan_status(swept_plan_t plan, void *stream);

/*
 * swept_plan_last_advance -- what the plan's last swept_advance enqueued:
 * the kernel launches (stages; a streamed ring launch and a cluster-resident
 * advance, SWEPT_OPT_RESIDENT, count once) in
 * *launches, the ring launches among them in *ring_launches, and, when
 * SWEPT_OPT_TIME_RING is on and the advance was not captured, the device time
 * from the first ring launch's start to the last one's end in *ring_ms
 * (waits for it); else *ring_ms = -1.  With SWEPT_OPT_GRAPH the counts are
 * those of the captured advance.  Errors: SWEPT_EINVAL for a null argument.
 */
int swept_plan_last_advance(swept_plan_t plan, int64_t *launches, int64_t *ring_launches, double *ring_ms);

/* ---- one stage at a time (a slice of a problem sharded over nodes) ------ */

/*
 * swept_stage -- stage k of swept_advance's schedule on every window of the
 * plan: a V-fill of height hv from the leading edges of stage k-1, then a
 * trapezoid of height ht whose leading edges it writes (Section 3, one
 * stage of every node; swept_advance is the sequence stage(0, 0, h),
 * stage(k, h, h) for k = 1..q-1, stage(q, h, rem), stage(q+1, rem, 0) for
 * nsteps = q*h + rem > h, and stage(0, 0, rem), stage(1, rem, 0) below h).
 * Windows are shifted by B/2 when k is odd; the windows wrap around the
 * plan's N points, so a plan over one node's slice of a larger periodic
 * problem computes every window inside the slice exactly, and the one window
 * that straddles the slice's end reads the edge half that swept_edge_copy
 * put into its neighbour slot (the exchange of Section 3).  hv = 0 loads the
 * flat state from u; ht = 0 stores the filled level to u, as do the top of a
 * partial trapezoid (ht < h) and the gap of a partial fill.
 *   u   device state of the plan's layout.
 *   k   >= 0; hv, ht in [0, h], not both 0.
 * Errors: SWEPT_EINVAL, SWEPT_ENOTSUP (uneven tiles), SWEPT_ECUDA.
 */
int swept_stage(swept_plan_t plan, void *u, int64_t k, int hv, int ht, void *stream);

/*
 * swept_edge_copy -- copy one window's leading-edge half of stage k's edge
 * buffer (the message a node sends after a stage, Section 3): side 0 is the
 * left edges L[h][2r], side 1 the right edges R[h][2r], B edge elements of the
 * plan's edge element size (8 bytes for FP64 and F32C (hi, lo) pairs, 4 for
 * F32, 16 for the Runge-Kutta pairs, 72 / 48 for Euler point states), level
 * by level.  dir 0: from the plan into buf; dir 1: from buf into the plan.
 *   buf  device memory of B edge elements.
 * Errors: SWEPT_EINVAL (window, side, dir, pointers; uneven tiles), SWEPT_ECUDA.
 */
int swept_edge_copy(swept_plan_t plan, int64_t k, int window, int side, void *buf, int dir, void *stream);

/* ---- adjoint ----------------------------------------------------------- */

/*
 * swept_adjoint -- vector-Jacobian product of the nsteps-step map:
 * grad_u0 = (d u(nsteps) / d u0)^T lambda_T.  With lambda_T = u(nsteps) this
 * is the gradient of J = 1/2 sum u(nsteps)^2 with respect to u0.  The paper
 * has no adjoint; the transposed step is derived from the update's Jacobian:
 *   heat: lambda' = lambda + r L2 lambda (the forward update itself);
 *   KS:   lambda'_j = lambda_j + 2a u_j (lambda_{j-1} - lambda_{j+1})
 *                     + b (L2 lambda)_j + e (L2 L2 lambda)_j,
 * u_j the forward state at that level.  The cotangent is advanced backwards
 * in time by the swept rule (same stages, transposed stencil), one stage per
 * launch.  KS needs the forward state at every level (checkpoints plus
 * recomputation): the forward pass is one swept advance whose kernels also
 * store the flat level that ends every m-th stage (a checkpoint every m*h
 * levels, nothing extra to compute); the reverse pass recomputes the forward
 * levels from those checkpoints, m*h at a time and each once, by per-step
 * stepping into a ring of m + 1 chunks of h levels, from which each
 * transposed stage reads its 2h levels.  m is at most 2*K_cycles stages
 * (K_cycles swept cycles of two stages; <= 0 means 64) and is the value that
 * minimises the scratch.  FP64 plans, even or uneven tiles.
 *   u0, lambda_T, grad_u0  device double[N]; grad_u0 may not alias u0.
 * Scratch (plan-owned, grown on demand, kept until swept_destroy), for KS
 * with nsteps = q*h + rem:
 *   8N * ([rem > 0] + ceil(q/m) + (m + 1)*h) bytes
 * (swept_adjoint_scratch returns it; N = 2^20, 20000 steps, h = 64: m = 2,
 * 349 states, 2.9 GB); none for heat.
 * Errors: SWEPT_EINVAL (null or misaligned pointers, grad_u0 == u0, memory of
 * another device, KS with nsteps >= 2^31), SWEPT_ENOTSUP (F32C, F32,
 * Runge-Kutta or Euler plan),
 * SWEPT_ENOMEM (the scratch does not fit), SWEPT_ECUDA.
 */
int swept_adjoint(swept_plan_t plan, const void *u0, const void *lambda_T, void *grad_u0,
                  int64_t nsteps, int K_cycles, void *stream);

/* Device scratch, in bytes, that swept_adjoint(plan, ..., nsteps, K_cycles)
 * allocates (the bound above); *bytes = 0 for heat.  Errors: SWEPT_EINVAL,
 * SWEPT_ENOTSUP (a plan swept_adjoint does not take). */
int swept_adjoint_scratch(swept_plan_t plan, int64_t nsteps, int K_cycles, int64_t *bytes);

/* ---- FP32-compensated state conversion -------------------------------- */

/*
 * swept_f32c_split -- hi = fl32(u), lo = fl32(u - hi) for N points.
 *   u64  device double[N];  u32c device float[2N] (hi then lo).
 * swept_f32c_merge -- u = (double)hi + (double)lo.
 * Errors: SWEPT_EINVAL, SWEPT_ECUDA.
 */
int swept_f32c_split(int64_t N, const double *u64, void *u32c, void *stream);
int swept_f32c_merge(int64_t N, const void *u32c, double *u64, void *stream);

/* ---- reductions -------------------------------------------------------- */

/*
 * swept_reduce -- FP64 reduction of the state (conserved sum, objective J,
 * or the directional derivative <u, v>).  Compensated (TwoSum/TwoProd)
 * accumulation in a fixed order, so repeated calls give identical bits.
 *   u    device state in the plan's layout (F32C values enter as
 *        fl64(hi + lo)); for an Euler plan, any one N-value block (pass
 *        u + N for the momentum, u + 2N for the energy).
 *   what SWEPT_SUM, SWEPT_HALF_SUMSQ or SWEPT_DOT.
 *   v    device double[N] for SWEPT_DOT, else ignored.
 *   out  device double[1]: the result is written there (no host sync).
 * Errors: SWEPT_EINVAL, SWEPT_ECUDA.
 */
int swept_reduce(swept_plan_t plan, const void *u, int what, const void *v,
                 double *out, void *stream);

/* ---- batched persistent launch ----------------------------------------- */

/* One problem of a batch.  Its state (layout of the batch's dtype, 8N bytes)
 * lives at byte `offset` of the caller's pool; offset must be 16-byte
 * aligned.  params: heat {r, unused}; KS {dt, dx}. */
typedef struct {
  int64_t N;
  int64_t nsteps;
  int64_t offset;
  int stencil;
  int reserved;
  double params[2];
} swept_problem_t;

typedef struct swept_batch_s *swept_batch_t;

/*
 * swept_batch_plan -- plan one persistent launch that advances `nprob`
 * independent periodic problems of uneven N and nsteps (each as
 * swept_advance would; Section 3's stages, per problem).
 *   probs   host array, copied.  Each N must be a multiple of the tile width
 *           of its stencil.
 *   dtype   SWEPT_F64 or SWEPT_F32C for the whole batch.
 *   B_heat, B_ks  tile widths for heat and KS problems, each 256 or 512
 *           (0 = 512); picked by the autotuner in the Python layer.
 * The work is one queue of (problem, run of up to 8 windows, stage) items
 * in stage-major order; a warp takes an item and, window by window, waits
 * (bounded) until the two windows of the previous stage it reads from have
 * published their edges, runs the stage and publishes.  Full diamond stages
 * stream the run through the ring-pipelined kernel code.  Allocates per-problem edge buffers (32N
 * bytes each), per-window stage counters and the item tables.
 * Errors: SWEPT_EINVAL, SWEPT_ENOTSUP, SWEPT_ENOMEM, SWEPT_ECUDA.
 */
int swept_batch_plan(swept_batch_t *out, int nprob, const swept_problem_t *probs, int dtype,
                     int B_heat, int B_ks);

/*
 * swept_batch_set -- options.
 *   SWEPT_BOPT_TIMEOUT_S  budget of every device-side wait, seconds (default
 *                         2): a wait that runs out records SWEPT_ETIMEOUT
 *                         and the launch winds down instead of hanging.
 *   SWEPT_BOPT_DROP_ITEM  test hook (a message lost on the host side): the
 *                         first window of the item with this queue index
 *                         never publishes its counter, so the items waiting
 *                         on it time out.
 *                         -1 = none (default).
 *   SWEPT_BOPT_GRID       number of thread blocks (default: all resident).
 *   SWEPT_BOPT_GRAPH      1 (default): replay the advance as a CUDA graph;
 *                         0: enqueue the resets and the launch directly.
 *   SWEPT_BOPT_RUN_LEN    windows per work item, 1..1024 (default: the longest
 *                         of 32, 16, 8 that leaves at least 8 items per
 *                         resident warp); rebuilds the item tables after
 *                         waiting for the device.  Results do not depend on it.
 */
#define SWEPT_BOPT_TIMEOUT_S  0
#define SWEPT_BOPT_DROP_ITEM  1
#define SWEPT_BOPT_GRID       2
#define SWEPT_BOPT_GRAPH      3
#define SWEPT_BOPT_RUN_LEN    4
int swept_batch_set(swept_batch_t batch, int option, double value);

/* Query: items, stages, windows, grid, problems, windows per item (the plan
 * takes the longest of 32, 16, 8 that leaves at least 8 items per resident
 * warp) in info[0..6). */
int swept_batch_info(swept_batch_t batch, int64_t *info, int ninfo);

/*
 * swept_advance_batch -- advance every problem of the batch in `pool`
 * (device) in place, as one CUDA graph (counter/status/flag resets + one
 * persistent kernel) captured on first use for this pool pointer and
 * replayed afterwards.  Asynchronous; errors found on the device are read
 * with swept_batch_status.
 * Errors: SWEPT_EINVAL, SWEPT_ECUDA.
 */
int swept_advance_batch(swept_batch_t batch, void *pool, void *stream);

/*
 * swept_batch_naive_advance -- the same result by per-step stepping over the
 * whole batch: one launch per time step covering every problem that still
 * has steps left (Section 6's straight decomposition, batched: one read and
 * one write of every active state per step).  The baseline the persistent
 * swept launch is measured against.  Allocates a scratch pool (the extent of
 * the problems' states) on first use; the result is back in `pool` when the
 * stream reaches the end.
 * Errors: SWEPT_EINVAL, SWEPT_ENOMEM, SWEPT_ECUDA.
 */
int swept_batch_naive_advance(swept_batch_t batch, void *pool, void *stream);

/* Synchronise `stream` and return the device status of the last advance:
 * SWEPT_OK or SWEPT_ETIMEOUT. */
int swept_batch_status(swept_batch_t batch, void *stream);

void swept_batch_destroy(swept_batch_t batch);

/* ---- advance without any device allocation ---------------------------- */

/*
 * swept_advance_noalloc -- swept_advance for callers that cannot allocate
 * device memory (no plan, no cudaMalloc, no allocating library call).
 *
 * The paper has no counterpart: this is a deployment variant.  Some callers
 * cannot call cudaMalloc -- a host that gives a plugin a fixed device-memory
 * budget and forbids allocations after start-up, or code that must not take
 * the implicit device synchronisation an allocation can cause.  This entry
 * point keeps the leading-edge scratch in a fixed array in device global
 * memory declared inside the library (32 * SWEPT_NOALLOC_MAX_N bytes =
 * 32 MiB); every GPU that loads the library holds that array until the
 * process exits.
 *   stencil_id  SWEPT_HEAT (params {r}) or SWEPT_KS (params {dt, dx});
 *               any other stencil: SWEPT_EINVAL.  The radius is implied.
 *   dtype       SWEPT_F64 or SWEPT_F32C; SWEPT_F32 or another value:
 *               SWEPT_EINVAL.
 *   B           must be given: 32*K with K in {1,2,4,8,16,32} (other
 *               multiples of 32: SWEPT_ENOTSUP; not a positive multiple of
 *               32, or K not a multiple of the radius: SWEPT_EINVAL).
 *   N           a positive multiple of B (the plan's uneven tiles are not
 *               taken here: N % B != 0 gives SWEPT_EINVAL), at most
 *               SWEPT_NOALLOC_MAX_N, else SWEPT_ETOOBIG.
 *   u       device state of the current device, 16-byte aligned, overwritten
 *           with u(nsteps), as swept_advance; u or the stream on another
 *           device: SWEPT_EINVAL.
 *   nsteps  >= 0 sub-timesteps; 0 is a no-op.
 * Results are identical to swept_advance with the same arguments.
 * All calls share the one array: calls that overlap on the GPU (different
 * streams or host threads without ordering) race and corrupt each other.
 * Nothing in the array needs to start at zero (each stage writes the edges
 * the next stage reads).  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress, with that device current) and caches
 * it; make that first call before any stream capture.  The cached address
 * lasts as long as the process: after cudaDeviceReset (or anything else that
 * destroys the device's primary context) unload and reload the library
 * before calling it again on that device.
 * Errors: SWEPT_EINVAL, SWEPT_ENOTSUP, SWEPT_ETOOBIG, SWEPT_ECUDA.
 */
#define SWEPT_NOALLOC_MAX_N (1 << 20)
int swept_advance_noalloc(int64_t N, int stencil_id, const double *params, int nparams,
                          int dtype, int B, void *u, int64_t nsteps, void *stream);

/* ---- measured peaks ---------------------------------------------------- */

/*
 * swept_probe_alu -- measure this GPU's peak arithmetic rate, the roofline
 * denominator of the swept kernels (they are bound by the FP32 pipe for the
 * compensated state and by the FP64 pipe for FP64, not by memory).  Section 4
 * models a node by its speed as a given constant; this measures it.  Enqueues
 * one kernel on `stream` whose blocks fill every SM at full residency; each
 * thread runs independent dependency chains of the chosen operation, so the
 * launch time is set by the pipe's throughput.  Time the launch with events
 * on the same stream: rate = *ops / seconds.  Nothing is allocated or written
 * (the chains' sum goes to an internal array only if it reaches a value it
 * never reaches).
 *   kind   SWEPT_PROBE_F32_ADD, SWEPT_PROBE_F32_FMA, SWEPT_PROBE_F64_ADD or
 *          SWEPT_PROBE_F64_FMA.
 *   iters  loop trips per thread, 1 .. 2^40 (each trip is 64 operations per
 *          thread; about 2e5 trips make an FP32 launch of a few milliseconds).
 *   ops    host double: the operations the launch performs (an add or an fma
 *          counts as one).
 * Errors: SWEPT_EINVAL (kind, iters, null ops, a stream of another device),
 * SWEPT_ECUDA.
 */
#define SWEPT_PROBE_F32_ADD 0
#define SWEPT_PROBE_F32_FMA 1
#define SWEPT_PROBE_F64_ADD 2
#define SWEPT_PROBE_F64_FMA 3
int swept_probe_alu(int kind, int64_t iters, double *ops, void *stream);

/*
 * swept_check_div_sqrt -- the Euler flux's binary32 division and square root
 * beside CUDA's correctly rounded ones (the paper has no counterpart: this
 * checks an implementation detail of the Euler kernels of Section 7).  The
 * compensated Euler kernels divide and take square roots with straight-line
 * code (an approximate reciprocal or reciprocal square root, one Newton step,
 * Markstein's fma correction) and accept a result only where an exact test
 * on its remainder proves it is the correctly rounded one; elsewhere they
 * recompute with the correctly rounded library operation.  This entry runs
 * both forms on n pairs (a[i], b[i]) in one kernel on `stream`:
 *   out[i]       straight-line a[i] / b[i]     out[n + i]    __fdiv_rn(a[i], b[i])
 *   out[2n + i]  straight-line sqrt(a[i])      out[3n + i]   __fsqrt_rn(a[i])
 *   ok[i]        1 where the division was proven, 0 where a kernel recomputes it
 *   ok[n + i]    the same for the square root
 * a, b (n floats each), out (4n floats) and ok (2n ints) are device memory of
 * the current device, owned by the caller.  Wherever ok is 1 the two results
 * must agree bit for bit.
 * Errors: SWEPT_EINVAL (n < 0, a null pointer, memory or a stream of another
 * device), SWEPT_ECUDA.
 */
int swept_check_div_sqrt(const float *a, const float *b, int64_t n, float *out, int *ok, void *stream);

/* ---- diagnostics ------------------------------------------------------ */

/* Name of a status code (static string). */
const char *swept_strerror(int code);

/* Library build identification: "<version> sm_103a". */
const char *swept_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SWEPT_H */
