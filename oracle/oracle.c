/*
 * Swept-rule oracle: plain, slow, per-step CPU stepping of a 1D periodic
 * explicit scheme.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header, table
 * or constant generator with the CUDA path.
 *
 * What it computes.  The swept rule (Sections 2-3) is an exact reordering of
 * per-step time stepping: every sub-timestep output is computed once, from
 * the same inputs, with no redundant or approximate work (Abstract;
 * Section 1, comparison with communication-avoiding methods).  So the oracle
 * is the definition itself: apply the sub-timestep to every point of the
 * periodic grid, one time level after another (Section 2; Section 3 fixes the
 * periodic 1D domain).
 *
 * Sub-timestep expressions.  The paper gives the schemes in words (Section 2:
 * a finite-difference sub-timestep that reads a point and its two
 * neighbours; Section 6: finite differences for Kuramoto-Sivashinsky) but no
 * evaluation order.  This file fixes one; it is the canonical order for the
 * whole project (the GPU kernels restate it independently):
 *
 *   heat  u_t = u_xx,  r = dt/dx^2 (Table 2 counts 3 FLOP per point):
 *       s  = u[i-1] + u[i+1]
 *       w  = s - 2*u[i]                      (2*u exact, one rounding)
 *       u' = fma(r, w, u[i])
 *
 *   Kuramoto-Sivashinsky  u_t = -u u_x - u_xx - u_xxxx  (Section 6), central
 *   differences, flux u^2/2, the 3-point second difference applied twice:
 *       G[j] = u[j]*u[j]
 *       w[j] = (u[j-1] + u[j+1]) - 2*u[j]
 *       D    = (w[i-1] + w[i+1]) - 2*w[i]
 *       t    = G[i+1] - G[i-1]
 *       u'   = fma(e, D, fma(b, w[i], fma(a, t, u[i])))
 *     with a = -(dt/(4 dx)), b = -(dt/(dx dx)), e = -(dt/((dx dx)(dx dx))),
 *     computed here in FP64 in exactly that order.
 *
 *   FP32-compensated state (hi, lo), value = hi + lo.  The increment is
 *   evaluated in FP32 on hi only, with differences taken first: h[j-1] - h[j]
 *   is exact when neighbours are within a factor 2 (Sterbenz), so on smooth
 *   data the second difference carries a relative, not an absolute, rounding
 *   error (the sum form s - 2h loses |h|*2^-24 per step to cancellation):
 *       heat: w = (h[i-1] - h[i]) + (h[i+1] - h[i]);  y = fmaf(r, w, lo)
 *       KS:   W[j] = (h[j-1] - h[j]) + (h[j+1] - h[j]);
 *             D = (W[i-1] - W[i]) + (W[i+1] - W[i]);
 *             t = (h[i+1] - h[i-1]) * (h[i+1] + h[i-1])      (= G[i+1] - G[i-1])
 *             y = fmaf(e, D, fmaf(b, W[i], fmaf(a, t, lo)))
 *       (hi', lo') = TwoSum(hi, y)           (Knuth, 6 operations)
 *     FP32 constants are the FP64 constants rounded to nearest.
 *     Split: hi = (float)u, lo = (float)(u - (double)hi);
 *     merge: u = (double)hi + (double)lo.
 *
 *   Two-stage Runge-Kutta (midpoint) as two sub-timesteps (Section 2: the
 *   first sub-timestep forwards u and outputs the midpoint state, the second
 *   outputs the next step from the forwarded u and the midpoint's
 *   neighbours).  One time step = two sub-timesteps, each of radius r:
 *       A: m = u + (dt/2) f(u)      B: u' = u + dt f(m)
 *   with the FP64 increments written exactly as the forward-Euler ones
 *   above, the constants halved for A (r/2; a/2, b/2, e/2, exact halvings):
 *       heat A: w = (u[i-1] + u[i+1]) - 2u[i];  m = fma(r/2, w, u[i])
 *       heat B: w = (m[i-1] + m[i+1]) - 2m[i];  u' = fma(r, w, u[i])
 *       KS   A: m = fma(e/2, D(u), fma(b/2, W(u)[i], fma(a/2, t(u), u[i])))
 *       KS   B: u' = fma(e, D(m), fma(b, W(m)[i], fma(a, t(m), u[i])))
 *   with W, D, t the KS terms above evaluated on the argument.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off (no fast-math).  fma()/fmaf()
 * are the C library's correctly rounded fused multiply-adds.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_HEAT = 0, OR_KS = 1, OR_HEAT_RK2 = 2, OR_KS_RK2 = 3 };
enum { OR_OK = 0, OR_EINVAL = -1, OR_ENOMEM = -2 };

typedef struct {
    int stencil;
    int radius;
    double r;            /* heat */
    double a, b, e;      /* KS */
    float r32, a32, b32, e32;
} or_consts;

static int make_consts(int stencil, const double *prm, or_consts *c)
{
    memset(c, 0, sizeof *c);
    if (stencil == OR_HEAT_RK2 || stencil == OR_KS_RK2) {
        /* same constants as the forward-Euler stencil; the RK2 drivers use them */
        int rc = make_consts(stencil - 2, prm, c);
        c->stencil = stencil;
        return rc;
    }
    c->stencil = stencil;
    if (stencil == OR_HEAT) {
        c->radius = 1;
        c->r = prm[0];
        c->r32 = (float)c->r;
        return OR_OK;
    }
    if (stencil == OR_KS) {
        double dt = prm[0], dx = prm[1];
        if (!(dx > 0.0)) return OR_EINVAL;
        double dx2 = dx * dx;
        c->radius = 2;
        c->a = -(dt / (4.0 * dx));
        c->b = -(dt / dx2);
        c->e = -(dt / (dx2 * dx2));
        c->a32 = (float)c->a;
        c->b32 = (float)c->b;
        c->e32 = (float)c->e;
        return OR_OK;
    }
    return OR_EINVAL;
}

static inline int64_t wrap(int64_t i, int64_t n)
{
    if (i >= 0 && i < n) return i;
    i %= n;
    return i < 0 ? i + n : i;
}

/* ---------------------------------------------------------------- FP64 -- */

/* One sub-timestep at point i, reading u[i-2..i+2] (periodic). */
static inline double point_f64(const or_consts *c, const double *u, int64_t i, int64_t n)
{
    if (c->stencil == OR_HEAT) {
        double um = u[wrap(i - 1, n)], u0 = u[i], up = u[wrap(i + 1, n)];
        double s = um + up;
        double w = s - 2.0 * u0;
        return fma(c->r, w, u0);
    } else {
        double v[5];
        for (int k = -2; k <= 2; ++k) v[k + 2] = u[wrap(i + k, n)];
        double Gm = v[1] * v[1];
        double Gp = v[3] * v[3];
        double wm = (v[0] + v[2]) - 2.0 * v[1];
        double w0 = (v[1] + v[3]) - 2.0 * v[2];
        double wp = (v[2] + v[4]) - 2.0 * v[3];
        double D = (wm + wp) - 2.0 * w0;
        double t = Gp - Gm;
        return fma(c->e, D, fma(c->b, w0, fma(c->a, t, v[2])));
    }
}

int oracle_step_f64(int stencil, const double *prm, const double *u, double *out, int64_t n)
{
    or_consts c;
    if (n <= 0 || make_consts(stencil, prm, &c) != OR_OK) return OR_EINVAL;
    for (int64_t i = 0; i < n; ++i) out[i] = point_f64(&c, u, i, n);
    return OR_OK;
}

/* u <- u after nsteps sub-timesteps (in place).  nthreads <= 0: default. */
int oracle_advance_f64(int stencil, const double *prm, double *u, int64_t n,
                       int64_t nsteps, int nthreads)
{
    or_consts c;
    if (n <= 0 || nsteps < 0 || make_consts(stencil, prm, &c) != OR_OK) return OR_EINVAL;
    if (nsteps == 0) return OR_OK;
    double *tmp = (double *)malloc((size_t)n * sizeof(double));
    if (!tmp) return OR_ENOMEM;
    double *src = u, *dst = tmp;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    for (int64_t s = 0; s < nsteps; ++s) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) dst[i] = point_f64(&c, src, i, n);
        double *t = src; src = dst; dst = t;
    }
    if (src != u) memcpy(u, src, (size_t)n * sizeof(double));
    free(tmp);
    return OR_OK;
}

/* ---------------------------------------------------------- plain FP32 -- */
/*
 * The FP64 expressions above evaluated in binary32, with the FP32 constants
 * (a diagnostic precision: what the compensated state below buys):
 *   heat: s = u[i-1] + u[i+1]; w = s - 2u[i]; u' = fmaf(r32, w, u[i])
 *   KS:   G, W, D, t as in FP64; u' = fmaf(e32, D, fmaf(b32, W[i], fmaf(a32, t, u[i])))
 */
static inline float point_f32(const or_consts *c, const float *u, int64_t i, int64_t n)
{
    if (c->stencil == OR_HEAT) {
        float um = u[wrap(i - 1, n)], u0 = u[i], up = u[wrap(i + 1, n)];
        float s = um + up;
        float w = s - 2.0f * u0;
        return fmaf(c->r32, w, u0);
    } else {
        float v[5];
        for (int k = -2; k <= 2; ++k) v[k + 2] = u[wrap(i + k, n)];
        float Gm = v[1] * v[1];
        float Gp = v[3] * v[3];
        float wm = (v[0] + v[2]) - 2.0f * v[1];
        float w0 = (v[1] + v[3]) - 2.0f * v[2];
        float wp = (v[2] + v[4]) - 2.0f * v[3];
        float D = (wm + wp) - 2.0f * w0;
        float t = Gp - Gm;
        return fmaf(c->e32, D, fmaf(c->b32, w0, fmaf(c->a32, t, v[2])));
    }
}

int oracle_step_f32(int stencil, const double *prm, const float *u, float *out, int64_t n)
{
    or_consts c;
    if (n <= 0 || make_consts(stencil, prm, &c) != OR_OK) return OR_EINVAL;
    for (int64_t i = 0; i < n; ++i) out[i] = point_f32(&c, u, i, n);
    return OR_OK;
}

int oracle_advance_f32(int stencil, const double *prm, float *u, int64_t n, int64_t nsteps, int nthreads)
{
    or_consts c;
    if (n <= 0 || nsteps < 0 || make_consts(stencil, prm, &c) != OR_OK) return OR_EINVAL;
    if (nsteps == 0) return OR_OK;
    float *tmp = (float *)malloc((size_t)n * sizeof(float));
    if (!tmp) return OR_ENOMEM;
    float *src = u, *dst = tmp;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    for (int64_t s = 0; s < nsteps; ++s) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) dst[i] = point_f32(&c, src, i, n);
        float *t = src; src = dst; dst = t;
    }
    if (src != u) memcpy(u, src, (size_t)n * sizeof(float));
    free(tmp);
    return OR_OK;
}

/* ------------------------------------------------- FP32 compensated ---- */

static inline void two_sum(float a, float b, float *s, float *err)
{
    float x = a + b;
    float bb = x - a;
    float ea = a - (x - bb);
    float eb = b - bb;
    *s = x;
    *err = ea + eb;
}

static inline void point_f32c(const or_consts *c, const float *hi, const float *lo,
                              int64_t i, int64_t n, float *ho, float *lout)
{
    float y;
    float h0 = hi[i];
    if (c->stencil == OR_HEAT) {
        float hm = hi[wrap(i - 1, n)], hp = hi[wrap(i + 1, n)];
        float w = (hm - h0) + (hp - h0);
        y = fmaf(c->r32, w, lo[i]);
    } else {
        float v[5];
        for (int k = -2; k <= 2; ++k) v[k + 2] = hi[wrap(i + k, n)];
        float wm = (v[0] - v[1]) + (v[2] - v[1]);
        float w0 = (v[1] - v[2]) + (v[3] - v[2]);
        float wp = (v[2] - v[3]) + (v[4] - v[3]);
        float D = (wm - w0) + (wp - w0);
        float t = (v[3] - v[1]) * (v[3] + v[1]);
        y = fmaf(c->e32, D, fmaf(c->b32, w0, fmaf(c->a32, t, lo[i])));
    }
    two_sum(h0, y, ho, lout);
}

int oracle_split_f32c(const double *u, float *hi, float *lo, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) {
        float h = (float)u[i];
        hi[i] = h;
        lo[i] = (float)(u[i] - (double)h);
    }
    return OR_OK;
}

int oracle_merge_f32c(const float *hi, const float *lo, double *u, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) u[i] = (double)hi[i] + (double)lo[i];
    return OR_OK;
}

int oracle_step_f32c(int stencil, const double *prm, const float *hi, const float *lo,
                     float *hi_out, float *lo_out, int64_t n)
{
    or_consts c;
    if (n <= 0 || make_consts(stencil, prm, &c) != OR_OK) return OR_EINVAL;
    for (int64_t i = 0; i < n; ++i) point_f32c(&c, hi, lo, i, n, &hi_out[i], &lo_out[i]);
    return OR_OK;
}

int oracle_advance_f32c(int stencil, const double *prm, float *hi, float *lo, int64_t n,
                        int64_t nsteps, int nthreads)
{
    or_consts c;
    if (n <= 0 || nsteps < 0 || make_consts(stencil, prm, &c) != OR_OK) return OR_EINVAL;
    if (nsteps == 0) return OR_OK;
    float *th = (float *)malloc((size_t)n * sizeof(float));
    float *tl = (float *)malloc((size_t)n * sizeof(float));
    if (!th || !tl) { free(th); free(tl); return OR_ENOMEM; }
    float *sh = hi, *sl = lo, *dh = th, *dl = tl;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    for (int64_t s = 0; s < nsteps; ++s) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) point_f32c(&c, sh, sl, i, n, &dh[i], &dl[i]);
        float *t;
        t = sh; sh = dh; dh = t;
        t = sl; sl = dl; dl = t;
    }
    if (sh != hi) {
        memcpy(hi, sh, (size_t)n * sizeof(float));
        memcpy(lo, sl, (size_t)n * sizeof(float));
    }
    free(th);
    free(tl);
    return OR_OK;
}

/* ----------------------------------------------------- RK2 (FP64) ----- */

/* Increment of one Euler sub-timestep of size scale*dt applied to argument
 * v at point i, added to base: the same expression as point_f64 with the
 * constants multiplied by `scale` (1 or 1/2, exact) and the stencil read from
 * v while the result is based on `base`. */
static inline double rk2_sub(const or_consts *c, const double *v, double base, int64_t i, int64_t n,
                             double scale)
{
    if (c->stencil == OR_HEAT_RK2) {
        double s = v[wrap(i - 1, n)] + v[wrap(i + 1, n)];
        double w = s - 2.0 * v[i];
        return fma(scale * c->r, w, base);
    } else {
        double x[5];
        for (int k = -2; k <= 2; ++k) x[k + 2] = v[wrap(i + k, n)];
        double Gm = x[1] * x[1];
        double Gp = x[3] * x[3];
        double wm = (x[0] + x[2]) - 2.0 * x[1];
        double w0 = (x[1] + x[3]) - 2.0 * x[2];
        double wp = (x[2] + x[4]) - 2.0 * x[3];
        double D = (wm + wp) - 2.0 * w0;
        double t = Gp - Gm;
        return fma(scale * c->e, D, fma(scale * c->b, w0, fma(scale * c->a, t, base)));
    }
}

/* u <- u after nsteps RK2 time steps (2*nsteps sub-timesteps). */
int oracle_advance_rk2_f64(int stencil, const double *prm, double *u, int64_t n, int64_t nsteps,
                           int nthreads)
{
    or_consts c;
    if (n <= 0 || nsteps < 0 || (stencil != OR_HEAT_RK2 && stencil != OR_KS_RK2) ||
        make_consts(stencil, prm, &c) != OR_OK)
        return OR_EINVAL;
    if (nsteps == 0) return OR_OK;
    double *m = (double *)malloc((size_t)n * sizeof(double));
    double *tmp = (double *)malloc((size_t)n * sizeof(double));
    if (!m || !tmp) { free(m); free(tmp); return OR_ENOMEM; }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    for (int64_t s = 0; s < nsteps; ++s) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) m[i] = rk2_sub(&c, u, u[i], i, n, 0.5);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) tmp[i] = rk2_sub(&c, m, u[i], i, n, 1.0);
        memcpy(u, tmp, (size_t)n * sizeof(double));
    }
    free(m);
    free(tmp);
    return OR_OK;
}

/* One sub-timestep for tests: sub = 0 gives m from u; sub = 1 gives u' from (u, m). */
int oracle_rk2_substep_f64(int stencil, const double *prm, int sub, const double *u, const double *m,
                           double *out, int64_t n)
{
    or_consts c;
    if (n <= 0 || (stencil != OR_HEAT_RK2 && stencil != OR_KS_RK2) || make_consts(stencil, prm, &c) != OR_OK)
        return OR_EINVAL;
    for (int64_t i = 0; i < n; ++i)
        out[i] = sub == 0 ? rk2_sub(&c, u, u[i], i, n, 0.5) : rk2_sub(&c, m, u[i], i, n, 1.0);
    return OR_OK;
}

/* ------------------------------------------------ Euler (FP64) -------- */
/*
 * 1D Euler equations of gas dynamics (Section 7), q = (rho, m = rho u, E),
 * p = (gamma - 1)(E - m^2/(2 rho)).  Second-order finite volumes (Section 2:
 * a gradient sub-timestep, then a flux-and-update sub-timestep), minmod
 * limiter, interface flux with scalar dissipation equal to the spectral
 * radius of the Roe matrix, midpoint Runge-Kutta: four sub-timesteps of
 * radius 1 per time step (Section 2's count):
 *   G  : s_i = minmod(q_i - q_{i-1}, q_{i+1} - q_i) per component
 *   F_a: q'_i = q_i - a (dt/dx) (F_{i+1/2} - F_{i-1/2}),  a = 1/2, then 1
 *   step: (G on q, F_{1/2} -> q_mid, G on q_mid, F_1 from q_mid's fluxes on q)
 * Canonical evaluation (every operation IEEE round-to-nearest; / and sqrt
 * correctly rounded):
 *   minmod(a, b) = (a > 0 && b > 0) ? fmin(a, b) : (a < 0 && b < 0) ? fmax(a, b) : 0
 *   face i+1/2: qL = fma(0.5, s_i, q_i), qR = fma(-0.5, s_{i+1}, q_{i+1})
 *   state (rho, m, E): u = m / rho; p = g1 * (E - 0.5 * (m * u)); H = (E + p) / rho
 *   f(q) = (m, fma(m, u, p), (E + p) * u)
 *   Roe: sl = sqrt(rho_L), sr = sqrt(rho_R), d = sl + sr,
 *        ut = (sl*u_L + sr*u_R) / d, Ht = (sl*H_L + sr*H_R) / d,
 *        c2 = g1 * (Ht - 0.5 * (ut * ut)), lam = |ut| + sqrt(fmax(c2, 0))
 *   F_k = 0.5 * ((fL_k + fR_k) - lam * (qR_k - qL_k))
 *   q'_k = fma(-ca, F_{i+1/2,k} - F_{i-1/2,k}, q_k),  ca = a * (dt / dx)
 * with g1 = gamma - 1; params = {dt, dx, gamma}.
 */
static inline double minmod(double a, double b)
{
    if (a > 0.0 && b > 0.0) return fmin(a, b);
    if (a < 0.0 && b < 0.0) return fmax(a, b);
    return 0.0;
}

static void euler_face_flux(const double *qL, const double *qR, double g1, double *F)
{
    double uL = qL[1] / qL[0], uR = qR[1] / qR[0];
    double pL = g1 * (qL[2] - 0.5 * (qL[1] * uL));
    double pR = g1 * (qR[2] - 0.5 * (qR[1] * uR));
    double HL = (qL[2] + pL) / qL[0], HR = (qR[2] + pR) / qR[0];
    double fL[3] = {qL[1], fma(qL[1], uL, pL), (qL[2] + pL) * uL};
    double fR[3] = {qR[1], fma(qR[1], uR, pR), (qR[2] + pR) * uR};
    double sl = sqrt(qL[0]), sr = sqrt(qR[0]);
    double d = sl + sr;
    double ut = (sl * uL + sr * uR) / d;
    double Ht = (sl * HL + sr * HR) / d;
    double c2 = g1 * (Ht - 0.5 * (ut * ut));
    double lam = fabs(ut) + sqrt(fmax(c2, 0.0));
    for (int k = 0; k < 3; ++k) F[k] = 0.5 * ((fL[k] + fR[k]) - lam * (qR[k] - qL[k]));
}

/* q, s: arrays of 3n (component-major per point: q[3i+k]). */
static void euler_slopes(const double *q, double *s, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) {
        int64_t im = wrap(i - 1, n), ip = wrap(i + 1, n);
        for (int k = 0; k < 3; ++k)
            s[3 * i + k] = minmod(q[3 * i + k] - q[3 * im + k], q[3 * ip + k] - q[3 * i + k]);
    }
}

/* out = base - ca * (F_{i+1/2} - F_{i-1/2}), fluxes from (q, s). */
static void euler_update(const double *q, const double *s, const double *base, double ca, double g1,
                         double *out, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) {
        double Fl[3], Fr[3], qL[3], qR[3];
        int64_t im = wrap(i - 1, n), ip = wrap(i + 1, n);
        for (int k = 0; k < 3; ++k) {
            qL[k] = fma(0.5, s[3 * im + k], q[3 * im + k]);
            qR[k] = fma(-0.5, s[3 * i + k], q[3 * i + k]);
        }
        euler_face_flux(qL, qR, g1, Fl);
        for (int k = 0; k < 3; ++k) {
            qL[k] = fma(0.5, s[3 * i + k], q[3 * i + k]);
            qR[k] = fma(-0.5, s[3 * ip + k], q[3 * ip + k]);
        }
        euler_face_flux(qL, qR, g1, Fr);
        for (int k = 0; k < 3; ++k) out[3 * i + k] = fma(-ca, Fr[k] - Fl[k], base[3 * i + k]);
    }
}

/* q (3n values, point-major) <- q after nsteps RK2 time steps (4 sub-timesteps each). */
int oracle_euler_advance(const double *prm, double *q, int64_t n, int64_t nsteps)
{
    if (n <= 0 || nsteps < 0 || !(prm[1] > 0.0)) return OR_EINVAL;
    double dtdx = prm[0] / prm[1], g1 = prm[2] - 1.0;
    double *s = (double *)malloc((size_t)3 * n * sizeof(double));
    double *qm = (double *)malloc((size_t)3 * n * sizeof(double));
    double *qn = (double *)malloc((size_t)3 * n * sizeof(double));
    if (!s || !qm || !qn) { free(s); free(qm); free(qn); return OR_ENOMEM; }
    for (int64_t t = 0; t < nsteps; ++t) {
        euler_slopes(q, s, n);
        euler_update(q, s, q, 0.5 * dtdx, g1, qm, n);
        euler_slopes(qm, s, n);
        euler_update(qm, s, q, 1.0 * dtdx, g1, qn, n);
        memcpy(q, qn, (size_t)3 * n * sizeof(double));
    }
    free(s); free(qm); free(qn);
    return OR_OK;
}

/*
 * Euler equations with the FP32-compensated state (the precision of the
 * compensated heat and KS steppers above): q = hi + lo per component, fluxes
 * and slopes in FP32 from hi (or from the FP32 midpoint), the update added
 * to lo and renormalised by TwoSum.  Same expressions as the FP64 scheme
 * above with every operation in binary32 (/ and sqrtf correctly rounded):
 *   slopes of the argument a (hi, then q_mid): s = minmodf(a_i - a_{i-1}, a_{i+1} - a_i)
 *   midpoint:  y = fmaf(-ch, F_{i+1/2} - F_{i-1/2}, lo_i);  q_mid_i = hi_i + y
 *   full step: y = fmaf(-cf, F_{i+1/2} - F_{i-1/2}, lo_i);  (hi_i, lo_i) = TwoSum(hi_i, y)
 * with fluxes from (hi, s) for the midpoint and from (q_mid, s) for the full
 * step; cf = (float)(dt/dx), ch = 0.5f * cf, g1 = (float)(gamma - 1).
 */
static inline float minmodf_(float a, float b)
{
    if (a > 0.0f && b > 0.0f) return fminf(a, b);
    if (a < 0.0f && b < 0.0f) return fmaxf(a, b);
    return 0.0f;
}

static void euler_face_flux_f(const float *qL, const float *qR, float g1, float *F)
{
    float uL = qL[1] / qL[0], uR = qR[1] / qR[0];
    float pL = g1 * (qL[2] - 0.5f * (qL[1] * uL));
    float pR = g1 * (qR[2] - 0.5f * (qR[1] * uR));
    float eL = qL[2] + pL, eR = qR[2] + pR;
    float HL = eL / qL[0], HR = eR / qR[0];
    float fL[3] = {qL[1], fmaf(qL[1], uL, pL), eL * uL};
    float fR[3] = {qR[1], fmaf(qR[1], uR, pR), eR * uR};
    float sl = sqrtf(qL[0]), sr = sqrtf(qR[0]);
    float d = sl + sr;
    float ut = (sl * uL + sr * uR) / d;
    float Ht = (sl * HL + sr * HR) / d;
    float c2 = g1 * (Ht - 0.5f * (ut * ut));
    float lam = fabsf(ut) + sqrtf(fmaxf(c2, 0.0f));
    for (int k = 0; k < 3; ++k) F[k] = 0.5f * ((fL[k] + fR[k]) - lam * (qR[k] - qL[k]));
}

static void euler_slopes_f(const float *a, float *s, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) {
        int64_t im = wrap(i - 1, n), ip = wrap(i + 1, n);
        for (int k = 0; k < 3; ++k)
            s[3 * i + k] = minmodf_(a[3 * i + k] - a[3 * im + k], a[3 * ip + k] - a[3 * i + k]);
    }
}

/* dF[3i+k] = F_{i+1/2,k} - F_{i-1/2,k} with fluxes from (a, s). */
static void euler_flux_diff_f(const float *a, const float *s, float g1, float *dF, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) {
        float Fl[3], Fr[3], qL[3], qR[3];
        int64_t im = wrap(i - 1, n), ip = wrap(i + 1, n);
        for (int k = 0; k < 3; ++k) {
            qL[k] = fmaf(0.5f, s[3 * im + k], a[3 * im + k]);
            qR[k] = fmaf(-0.5f, s[3 * i + k], a[3 * i + k]);
        }
        euler_face_flux_f(qL, qR, g1, Fl);
        for (int k = 0; k < 3; ++k) {
            qL[k] = fmaf(0.5f, s[3 * i + k], a[3 * i + k]);
            qR[k] = fmaf(-0.5f, s[3 * ip + k], a[3 * ip + k]);
        }
        euler_face_flux_f(qL, qR, g1, Fr);
        for (int k = 0; k < 3; ++k) dF[3 * i + k] = Fr[k] - Fl[k];
    }
}

/* (hi, lo): 3n floats each, point-major; nsteps time steps of 4 sub-timesteps. */
int oracle_euler_advance_f32c(const double *prm, float *hi, float *lo, int64_t n, int64_t nsteps)
{
    if (n <= 0 || nsteps < 0 || !(prm[1] > 0.0)) return OR_EINVAL;
    const float cf = (float)(prm[0] / prm[1]);
    const float ch = 0.5f * cf;
    const float g1 = (float)(prm[2] - 1.0);
    float *s = (float *)malloc((size_t)3 * n * sizeof(float));
    float *qm = (float *)malloc((size_t)3 * n * sizeof(float));
    float *dF = (float *)malloc((size_t)3 * n * sizeof(float));
    if (!s || !qm || !dF) { free(s); free(qm); free(dF); return OR_ENOMEM; }
    for (int64_t t = 0; t < nsteps; ++t) {
        euler_slopes_f(hi, s, n);
        euler_flux_diff_f(hi, s, g1, dF, n);
        for (int64_t j = 0; j < 3 * n; ++j) qm[j] = hi[j] + fmaf(-ch, dF[j], lo[j]);
        euler_slopes_f(qm, s, n);
        euler_flux_diff_f(qm, s, g1, dF, n);
        for (int64_t j = 0; j < 3 * n; ++j) two_sum(hi[j], fmaf(-cf, dF[j], lo[j]), &hi[j], &lo[j]);
    }
    free(s); free(qm); free(dF);
    return OR_OK;
}

/* ------------------------------------------------------- adjoint ------ */

/*
 * Discrete adjoint of the FP64 stepper (reverse-mode derivative of the
 * composed map u0 -> u(nsteps)).  With Phi the one-step map, the cotangent
 * runs backwards as lambda^n = (dPhi/du (u^n))^T lambda^{n+1}; grad = lambda^0.
 *
 * The Jacobian of the canonical expressions in exact arithmetic:
 *   heat: dPhi = I + r*L2, L2 the periodic 3-point second difference, which
 *         is symmetric, so lambda' = lambda + r*L2 lambda.
 *   KS:   dPhi = I + a*dT + b*L2 + e*L2*L2 with (dT v)_i = 2 u_{i+1} v_{i+1}
 *         - 2 u_{i-1} v_{i-1}; its transpose is (dT^T l)_j = 2 u_j (l_{j-1}
 *         - l_{j+1}); L2 and L2*L2 are symmetric.
 *
 * Written as a plain dense-in-time computation: the whole trajectory is
 * stored (n * nsteps doubles), so it is for small cases only.
 *
 * Evaluation order (canonical for the adjoint):
 *   heat: w = (l[j-1] + l[j+1]) - 2 l[j];  l' = fma(r, w, l[j])
 *   KS:   W[j] = (l[j-1] + l[j+1]) - 2 l[j];  D = (W[j-1] + W[j+1]) - 2 W[j];
 *         q = l[j-1] - l[j+1];  c = (2a) * u[j];
 *         l' = fma(e, D, fma(b, W[j], fma(c, q, l[j])))
 */
static void adjoint_point_pass(const or_consts *c, const double *u, const double *l,
                               double *out, int64_t n)
{
    for (int64_t j = 0; j < n; ++j) {
        if (c->stencil == OR_HEAT) {
            double s = l[wrap(j - 1, n)] + l[wrap(j + 1, n)];
            double w = s - 2.0 * l[j];
            out[j] = fma(c->r, w, l[j]);
        } else {
            double v[5];
            for (int k = -2; k <= 2; ++k) v[k + 2] = l[wrap(j + k, n)];
            double Wm = (v[0] + v[2]) - 2.0 * v[1];
            double W0 = (v[1] + v[3]) - 2.0 * v[2];
            double Wp = (v[2] + v[4]) - 2.0 * v[3];
            double D = (Wm + Wp) - 2.0 * W0;
            double q = v[1] - v[3];
            double cj = (2.0 * c->a) * u[j];
            out[j] = fma(c->e, D, fma(c->b, W0, fma(cj, q, v[2])));
        }
    }
}

int oracle_adjoint_f64(int stencil, const double *prm, const double *u0, const double *lam_T,
                       double *grad, int64_t n, int64_t nsteps)
{
    or_consts c;
    if (n <= 0 || nsteps < 0 || make_consts(stencil, prm, &c) != OR_OK) return OR_EINVAL;
    double *traj = (double *)malloc((size_t)n * (size_t)(nsteps + 1) * sizeof(double));
    double *tmp = (double *)malloc((size_t)n * sizeof(double));
    if (!traj || !tmp) { free(traj); free(tmp); return OR_ENOMEM; }
    memcpy(traj, u0, (size_t)n * sizeof(double));
    for (int64_t s = 0; s < nsteps; ++s)
        for (int64_t i = 0; i < n; ++i)
            traj[(s + 1) * n + i] = point_f64(&c, traj + s * n, i, n);
    memcpy(grad, lam_T, (size_t)n * sizeof(double));
    for (int64_t s = nsteps - 1; s >= 0; --s) {
        adjoint_point_pass(&c, traj + s * n, grad, tmp, n);
        memcpy(grad, tmp, (size_t)n * sizeof(double));
    }
    free(traj);
    free(tmp);
    return OR_OK;
}

/* One adjoint step (transpose Jacobian at state u applied to l), for tests. */
int oracle_adjoint_step_f64(int stencil, const double *prm, const double *u, const double *l,
                            double *out, int64_t n)
{
    or_consts c;
    if (n <= 0 || make_consts(stencil, prm, &c) != OR_OK) return OR_EINVAL;
    adjoint_point_pass(&c, u, l, out, n);
    return OR_OK;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
