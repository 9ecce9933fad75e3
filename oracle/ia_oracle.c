/*
 * ia_oracle.c -- plain, slow, FP64 CPU oracle for the classical ion-atom trajectory method of
 * "Chaotic scattering and heating in cold ion-atom collisions: two sides of the same coin"
 * (Chowdhury & Perez-Rios, arXiv 2509.15117).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE. Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load this library. It shares no source, header, table or helper with the
 * CUDA library; the two meet only in the seeded initial conditions that the tests hand to both.
 *
 * What it computes, in the paper's order:
 *   - Eq. 1 (the Hamiltonian) gives Newton's equations for the twelve variables (ion and atom
 *     positions and velocities). The trap term sum_j (a_j + 2 q_j cos(Omega t)) m_i Omega^2/8 r_j^2
 *     is read with r_j the ion's Cartesian coordinate j (the paper reuses the index i for both the
 *     ion label and the axis). A phase phi0 and a sign s (+1 for Eq. 1 as printed) are added:
 *     cos(Omega t) -> s*cos(Omega t + phi0).
 *   - The text after Eq. 1 gives V(r) = C8/r^8 - C4/r^4 with C4 = alpha/2. C8 is fixed by the well
 *     depth D_e: V has its minimum -D_e at r_e^4 = 2 C8/C4, hence C8 = C4^2/(4 D_e).
 *   - The same passage names the integrator: the adaptive Dormand-Prince 5(4) pair of Dormand &
 *     Prince (1980) as used in the MATLAB ODE suite of Shampine & Reichelt (1997), i.e. ode45.
 *     This file uses the textbook form: seven stage derivatives k_1..k_7 of all twelve
 *     components, FSAL, fifth-order propagation, embedded fourth-order error estimate, the
 *     ode45 error weights, step-size rules and initial-step rule, and the ode45 continuous
 *     extension (Shampine 1986) for event location.
 *   - The head-on paragraph (ion at rest at the trap centre, atom on a sphere of radius r0 moving
 *     radially inward) and the termination reading: integration stops when the ion-atom separation
 *     |x_a - x_i| crosses r0 outward, or at t_max.
 *   - The Fig. 1 caption defines the observables: scattering angle between the atom's initial and
 *     final velocities, number of bounces (short-range collisions), momentum transfer
 *     |p_f - p_i| of the atom. The text adds the ion heating (ion energy change) and complex
 *     formation (more than one bounce; the regular region scatters after a single bounce).
 *
 * Compiled with -O2 -fno-fast-math -ffp-contract=off so every operation is one IEEE-754 double
 * operation in source order. OpenMP is used across trajectories only.
 */
#define __STDC_WANT_IEC_60559_TYPES_EXT__ 1 /* _Float128 and its f128 functions */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <float.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_N 12 /* y = [x_ion(3), v_ion(3), x_atom(3), v_atom(3)] */

/* Per-system physical and numerical parameters (atomic units throughout). */
typedef struct {
    double m_ion, m_atom;   /* masses, m_e */
    double alpha;           /* atom static dipole polarisability, a.u.; C4 = alpha/2 */
    double De;              /* well depth, E_h; C8 = C4^2/(4 De) (0 if alpha == 0) */
    double Omega;           /* rf angular frequency, rad per a.u. of time */
    double a[3], q[3];      /* Mathieu parameters per axis */
    double r0;              /* sphere radius of the start and of the outward-crossing event, a0 */
    double t_max;           /* a.u. of time */
    double rtol, atol_pos, atol_vel;
    double h_max;           /* largest step, a.u. of time */
    int32_t rf_sign;        /* s in s*cos(Omega t + phi0): +1 is Eq. 1 as printed */
    int32_t pad_;
    int64_t max_attempts;   /* cap on attempted steps (accepted + rejected) */
} orc_system;

/* Per-trajectory outcome. */
typedef struct {
    double theta_s;         /* scattering angle of the atom, rad */
    double dp;              /* |p_f - p_i| of the atom, a.u. */
    double dE_ion;          /* E_ion(t_f) - E_ion(0), E_h */
    double t_final;         /* a.u. */
    double t_first_bounce, t_last_bounce;
    double y_final[ORC_N];
    int64_t n_steps, n_rej; /* accepted, rejected */
    int32_t n_bounce;
    uint32_t status;
} orc_result;

enum {
    ORC_EXIT = 0,            /* crossed r0 outward */
    ORC_TMAX = 1u << 0,
    ORC_MAX_STEPS = 1u << 1,
    ORC_H_UNDERFLOW = 1u << 2,
    ORC_NONFINITE = 1u << 3,
    ORC_BAD_IC = 1u << 4,
    ORC_EXIT_OUTSIDE = 1u << 5, /* moving outward beyond r0 without a crossing inside the step */
    ORC_COMPLEX = 1u << 8     /* n_bounce >= 2 */
};

/* ------------------------------------------------------------------------------------------ */
/* Dormand & Prince (1980) coefficients, RK5(4)7M, as tabulated by Shampine & Reichelt (1997). */

static const double DP_C[7] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 4.0 / 5.0, 8.0 / 9.0, 1.0, 1.0};
static const double DP_A[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5.0, 0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0},
    {44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0, 0, 0},
    {19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0, 0},
    {9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0, 0},
    {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0}};
/* fifth-order weights b (= last row of A, FSAL) and fourth-order weights bhat */
static const double DP_B[7] = {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0,
                               -2187.0 / 6784.0, 11.0 / 84.0, 0.0};
static const double DP_BHAT[7] = {5179.0 / 57600.0, 0.0, 7571.0 / 16695.0, 393.0 / 640.0,
                                  -92097.0 / 339200.0, 187.0 / 2100.0, 1.0 / 40.0};
/* Continuous extension of ode45 (Shampine 1986): y(t + s h) = y + h sum_j k_j sum_p BI[j][p] s^(p+1) */
static const double DP_BI[7][4] = {
    {1.0, -183.0 / 64.0, 37.0 / 12.0, -145.0 / 128.0},
    {0.0, 0.0, 0.0, 0.0},
    {0.0, 1500.0 / 371.0, -1000.0 / 159.0, 1000.0 / 371.0},
    {0.0, -125.0 / 32.0, 125.0 / 12.0, -375.0 / 64.0},
    {0.0, 9477.0 / 3392.0, -729.0 / 106.0, 25515.0 / 6784.0},
    {0.0, -11.0 / 7.0, 11.0 / 3.0, -55.0 / 28.0},
    {0.0, 3.0 / 2.0, -4.0, 5.0 / 2.0}};

/* ------------------------------------------------------------------------------------------ */
/* Generic DP5(4) machinery over n <= ORC_N components with a callback right-hand side.        */

typedef void (*orc_rhs_fn)(const void* ctx, double t, const double* y, double* f);

/* One attempted step from (t, y) with k[0] = f(t, y) already filled. Fills k[1..6], ynew (the
 * fifth-order solution, whose derivative is k[6]) and err (h * sum_j (b_j - bhat_j) k_j). */
static void dp5_attempt(orc_rhs_fn rhs, const void* ctx, int n, double t, const double* y,
                        double h, double k[7][ORC_N], double* ynew, double* err)
{
    double ys[ORC_N];
    for (int s = 1; s < 7; ++s) {
        for (int i = 0; i < n; ++i) {
            double acc = 0.0;
            for (int j = 0; j < s; ++j) acc += DP_A[s][j] * k[j][i];
            ys[i] = y[i] + h * acc;
        }
        rhs(ctx, t + DP_C[s] * h, ys, k[s]);
        if (s == 6)
            for (int i = 0; i < n; ++i) ynew[i] = ys[i];
    }
    for (int i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int j = 0; j < 7; ++j) acc += (DP_B[j] - DP_BHAT[j]) * k[j][i];
        err[i] = h * acc;
    }
}

/* ode45 error measure: max_i |err_i| / max(rtol*max(|y_i|,|ynew_i|), atol_i). Accept if <= 1. */
static double dp5_error_norm(int n, const double* y, const double* ynew, const double* err,
                             double rtol, const double* atol)
{
    double e = 0.0;
    for (int i = 0; i < n; ++i) {
        double w = fmax(fabs(y[i]), fabs(ynew[i]));
        double sc = fmax(rtol * w, atol[i]);
        double r = fabs(err[i]) / sc;
        if (r > e) e = r;
    }
    return e;
}

/* Dense output at y(t + s h) from the stage derivatives of the accepted step. */
static void dp5_dense(int n, const double* y, double h, double k[7][ORC_N], double s, double* out)
{
    double w[7];
    for (int j = 0; j < 7; ++j)
        w[j] = s * (DP_BI[j][0] + s * (DP_BI[j][1] + s * (DP_BI[j][2] + s * DP_BI[j][3])));
    for (int i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int j = 0; j < 7; ++j) acc += w[j] * k[j][i];
        out[i] = y[i] + h * acc;
    }
}

/* ode45 initial step: h = 0.8 rtol^(1/5) / || f0 / max(|y0|, atol/rtol) ||_inf, capped by hmax. */
static double dp5_initial_step(int n, const double* y0, const double* f0, double rtol,
                               const double* atol, double hmax, double span)
{
    double h = fmin(hmax, span);
    double rh = 0.0;
    for (int i = 0; i < n; ++i) {
        double w = fmax(fabs(y0[i]), atol[i] / rtol);
        double r = fabs(f0[i]) / w;
        if (r > rh) rh = r;
    }
    rh = rh / (0.8 * pow(rtol, 0.2));
    if (h * rh > 1.0) h = 1.0 / rh;
    return h;
}

/* Spacing of doubles at |t| (MATLAB's eps(t)). */
static double spacing(double t)
{
    double a = fabs(t);
    if (a < DBL_MIN) return DBL_MIN;
    return nextafter(a, INFINITY) - a;
}

/* What the step loop should do after an accepted step. */
typedef int (*orc_accept_fn)(void* obs, double t_old, const double* y_old, double h,
                             const double* y_new, double k[7][ORC_N]);

/* Constants of ode45's step-size rules (Shampine & Reichelt 1997). Macros so that a test can build
 * the oracle with one of them changed and check that its pins catch the change. */
#ifndef ORC_CTRL_SAFETY
#define ORC_CTRL_SAFETY 1.25      /* growth: h / (ORC_CTRL_SAFETY err^ORC_CTRL_EXPONENT) */
#endif
#ifndef ORC_CTRL_EXPONENT
#define ORC_CTRL_EXPONENT 0.2     /* 1/5: the local error of the pair behaves as h^5 */
#endif
#ifndef ORC_CTRL_GROW_MAX
#define ORC_CTRL_GROW_MAX 5.0     /* largest growth of h after an accepted step */
#endif
#ifndef ORC_CTRL_SHRINK_SAFETY
#define ORC_CTRL_SHRINK_SAFETY 0.8  /* first failure: h * max(floor, 0.8 err^(-1/5)) */
#endif
#ifndef ORC_CTRL_SHRINK_MIN
#define ORC_CTRL_SHRINK_MIN 0.1   /* floor of that factor */
#endif
#ifndef ORC_CTRL_RETRY
#define ORC_CTRL_RETRY 0.5        /* second and later failures of one step: h * 0.5 */
#endif

/* Optional record of every attempted step (test hook): start time, step size, error measure and
 * whether it was accepted. */
typedef struct {
    int64_t cap, n;
    double *t, *h, *err;
    int32_t* acc;
} orc_trace;

/* Rounding-noise model (test hook): after every accepted step each component moves by m ulps
 * (nextafter, exact), m uniform on -ulps..ulps from a splitmix64 hash of (seed, trajectory, step,
 * component). It stands for the accumulated effect of another rounding order at every step, to measure
 * how far FP64 rounding alone moves a trajectory's observables. */
typedef struct {
    uint64_t seed, traj;
    int32_t ulps;
} orc_noise;

/* splitmix64 (Steele, Lea & Flood, OOPSLA 2014): one output of the generator whose state is x. */
static uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static void noise_apply(const orc_noise* nz, int64_t step, int n, double* y)
{
    if (!nz || nz->ulps <= 0) return;
    const uint64_t key = splitmix64(nz->seed ^ splitmix64(nz->traj));
    for (int i = 0; i < n; ++i) {
        const uint64_t r = splitmix64(key ^ ((uint64_t)step * 16u + (uint64_t)i));
        const int m = (int)(r % (uint64_t)(2 * nz->ulps + 1)) - nz->ulps;
        for (int u = 0; u < (m < 0 ? -m : m); ++u) y[i] = nextafter(y[i], m < 0 ? -INFINITY : INFINITY);
    }
}

static void trace_put(orc_trace* tr, double t, double h, double err, int acc)
{
    if (!tr || tr->n >= tr->cap) return;
    tr->t[tr->n] = t;
    tr->h[tr->n] = h;
    tr->err[tr->n] = err;
    tr->acc[tr->n] = acc;
    tr->n += 1;
}

typedef struct {
    int64_t n_steps, n_rej;
    uint32_t status;
    double t, h_next;
} orc_loop_state;

/*
 * Adaptive DP5(4) driver with the step-size rules of ode45 (Shampine & Reichelt 1997):
 *   accept if err <= 1; after an accepted step with no failure in it, h <- h / (1.25 err^(1/5)),
 *   at most 5x; first failure h <- h * max(0.1, 0.8 err^(-1/5)); further failures h <- h/2;
 *   steps never below 16 eps(t) (failure H_UNDERFLOW); the last step lands on t_end.
 * on_accept returns nonzero to stop (the event handler of the caller).
 * y holds the current state on entry and the state at the end of the last accepted step on exit.
 */
static void dp5_drive(orc_rhs_fn rhs, const void* ctx, int n, double t0, double t_end, double* y,
                      double rtol, const double* atol, double hmax, double h0, int64_t max_attempts,
                      orc_accept_fn on_accept, void* obs, orc_loop_state* st, orc_trace* tr,
                      const orc_noise* nz)
{
    double k[7][ORC_N], ynew[ORC_N], err[ORC_N];
    double t = t0;
    rhs(ctx, t, y, k[0]);
    double h = h0 > 0.0 ? h0 : dp5_initial_step(n, y, k[0], rtol, atol, hmax, t_end - t0);
    st->n_steps = 0;
    st->n_rej = 0;
    st->status = 0;
    for (;;) {
        if (t >= t_end) {
            st->status |= ORC_TMAX;
            break;
        }
        if (st->n_steps + st->n_rej >= max_attempts) {
            st->status |= ORC_MAX_STEPS;
            break;
        }
        double hmin = 16.0 * spacing(t);
        h = fmin(h, hmax);
        h = fmax(h, hmin);
        if (t + h > t_end) h = t_end - t;
        int nofailed = 1;
        double errn;
        for (;;) {
            dp5_attempt(rhs, ctx, n, t, y, h, k, ynew, err);
            errn = dp5_error_norm(n, y, ynew, err, rtol, atol);
            int finite = isfinite(errn);
            for (int i = 0; i < n; ++i) finite = finite && isfinite(ynew[i]);
            if (!finite) {
                st->status |= ORC_NONFINITE;
                st->t = t;
                st->h_next = h;
                return;
            }
            trace_put(tr, t, h, errn, errn <= 1.0);
            if (errn <= 1.0) break;
            st->n_rej += 1;
            if (h <= hmin) {
                st->status |= ORC_H_UNDERFLOW;
                st->t = t;
                st->h_next = h;
                return;
            }
            if (nofailed) {
                nofailed = 0;
                h = fmax(hmin, h * fmax(ORC_CTRL_SHRINK_MIN, ORC_CTRL_SHRINK_SAFETY * pow(errn, -ORC_CTRL_EXPONENT)));
            } else {
                h = fmax(hmin, ORC_CTRL_RETRY * h);
            }
            if (st->n_steps + st->n_rej >= max_attempts) {
                st->status |= ORC_MAX_STEPS;
                st->t = t;
                st->h_next = h;
                return;
            }
        }
        st->n_steps += 1;
        int stop = on_accept ? on_accept(obs, t, y, h, ynew, k) : 0;
        double t_new = (t + h >= t_end) ? t_end : t + h;
        for (int i = 0; i < n; ++i) {
            y[i] = ynew[i];
            k[0][i] = k[6][i];
        }
        t = t_new;
        if (stop) break;
        noise_apply(nz, st->n_steps, n, y);
        if (nofailed) {
            double temp = ORC_CTRL_SAFETY * pow(errn, ORC_CTRL_EXPONENT);
            if (temp > 1.0 / ORC_CTRL_GROW_MAX)
                h = h / temp;
            else
                h = ORC_CTRL_GROW_MAX * h;
        }
    }
    st->t = t;
    st->h_next = h;
}

/* ------------------------------------------------------------------------------------------ */
/* Ion-atom system                                                                            */

static double sys_C4(const orc_system* s) { return 0.5 * s->alpha; }
static double sys_C8(const orc_system* s)
{
    double C4 = sys_C4(s);
    if (C4 == 0.0) return 0.0;
    return C4 * C4 / (4.0 * s->De);
}

/* V(r) = C8/r^8 - C4/r^4 and dV/dr. */
void orc_potential(const orc_system* s, double r, double* V, double* dVdr)
{
    double C4 = sys_C4(s), C8 = sys_C8(s);
    *V = C8 / pow(r, 8) - C4 / pow(r, 4);
    *dVdr = -8.0 * C8 / pow(r, 9) + 4.0 * C4 / pow(r, 5);
}

typedef struct {
    const orc_system* sys;
    double phi0;
} ionatom_ctx;

/* Newton's equations from Eq. 1: for the ion, -grad of the trap term and of V; for the atom,
 * -grad of V. f = [v_ion, a_ion, v_atom, a_atom]. */
static void ionatom_rhs(const void* vctx, double t, const double* y, double* f)
{
    const ionatom_ctx* c = (const ionatom_ctx*)vctx;
    const orc_system* s = c->sys;
    const double* xi = y + 0;
    const double* vi = y + 3;
    const double* xa = y + 6;
    const double* va = y + 9;
    double d[3], r = 0.0;
    for (int j = 0; j < 3; ++j) d[j] = xa[j] - xi[j];
    r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double V, dVdr;
    orc_potential(s, r, &V, &dVdr);
    double cosv = (double)s->rf_sign * cos(s->Omega * t + c->phi0);
    for (int j = 0; j < 3; ++j) {
        double F_atom = -dVdr * d[j] / r; /* force on the atom, -dV/dx_a */
        double F_trap = -(s->m_ion * s->Omega * s->Omega / 4.0) * (s->a[j] + 2.0 * s->q[j] * cosv) * xi[j];
        f[0 + j] = vi[j];
        f[3 + j] = (F_trap - F_atom) / s->m_ion;
        f[6 + j] = va[j];
        f[9 + j] = F_atom / s->m_atom;
    }
}

/* Ion energy without V: kinetic plus the trap term of Eq. 1 at time t. */
static double ion_energy(const orc_system* s, double phi0, double t, const double* y)
{
    double cosv = (double)s->rf_sign * cos(s->Omega * t + phi0);
    double E = 0.0;
    for (int j = 0; j < 3; ++j) {
        E += 0.5 * s->m_ion * y[3 + j] * y[3 + j];
        E += (s->a[j] + 2.0 * s->q[j] * cosv) * (s->m_ion * s->Omega * s->Omega / 8.0) * y[j] * y[j];
    }
    return E;
}

static void separation(const double* y, double d[3]) {
    for (int j = 0; j < 3; ++j) d[j] = y[6 + j] - y[j];
}
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* radial velocity sign carrier: d . (v_atom - v_ion) = |d| * dr/dt */
static double rdot_times_r(const double* y)
{
    double d[3], w[3];
    separation(y, d);
    for (int j = 0; j < 3; ++j) w[j] = y[9 + j] - y[3 + j];
    return dot3(d, w);
}

typedef struct {
    ionatom_ctx ctx;
    double r0sq;
    double rdot_prev;
    int32_t n_bounce;
    double t_first, t_last;
    int exited;
    uint32_t exit_flags;
    double t_exit;
    double y_exit[ORC_N];
} ionatom_obs;

/* Event and bounce bookkeeping after every accepted step.
 * Bounce: d.(v_a - v_i) changes from < 0 to >= 0 (pericentre passage), counted at the step end.
 * Exit: |d|^2 >= r0^2 with d.(v_a - v_i) > 0 at the step end. If |d| < r0 at the step start the
 * crossing |d| = r0 is located on the continuous extension by bisection and the state there is
 * final; otherwise the step end is final (flag EXIT_OUTSIDE). */
static int ionatom_on_accept(void* vobs, double t_old, const double* y_old, double h,
                             const double* y_new, double k[7][ORC_N])
{
    ionatom_obs* o = (ionatom_obs*)vobs;
    double rd = rdot_times_r(y_new);
    double t_new = t_old + h;
    if (o->rdot_prev < 0.0 && rd >= 0.0) {
        o->n_bounce += 1;
        if (o->n_bounce == 1) o->t_first = t_new;
        o->t_last = t_new;
    }
    o->rdot_prev = rd;
    double d[3];
    separation(y_new, d);
    double g_new = dot3(d, d) - o->r0sq;
    if (g_new >= 0.0 && rd > 0.0) {
        double dold[3];
        separation(y_old, dold);
        double g_old = dot3(dold, dold) - o->r0sq;
        o->exited = 1;
        if (g_old < 0.0) {
            double lo = 0.0, hi = 1.0, ys[ORC_N];
            for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
                double mid = 0.5 * (lo + hi);
                if (mid <= lo || mid >= hi) break;
                dp5_dense(ORC_N, y_old, h, k, mid, ys);
                double ds[3];
                separation(ys, ds);
                if (dot3(ds, ds) - o->r0sq < 0.0)
                    lo = mid;
                else
                    hi = mid;
            }
            dp5_dense(ORC_N, y_old, h, k, hi, o->y_exit);
            o->t_exit = t_old + hi * h;
            o->exit_flags = 0;
        } else {
            memcpy(o->y_exit, y_new, sizeof(double) * ORC_N);
            o->t_exit = t_new;
            o->exit_flags = ORC_EXIT_OUTSIDE;
        }
        return 1;
    }
    return 0;
}

/* Integrate one trajectory from y0 at t = 0 with rf phase phi0 (nz: rounding-noise model or NULL). */
static void trajectory(const orc_system* s, const double* y0, double phi0, orc_result* r, const orc_noise* nz)
{
    memset(r, 0, sizeof(*r));
    int ok = 1;
    for (int i = 0; i < ORC_N; ++i) ok = ok && isfinite(y0[i]);
    ok = ok && isfinite(phi0) && s->m_ion > 0.0 && s->m_atom > 0.0 && s->r0 > 0.0 && s->t_max > 0.0;
    double d0[3];
    separation(y0, d0);
    ok = ok && dot3(d0, d0) > 0.0;
    if (!ok) {
        r->status = ORC_BAD_IC;
        memcpy(r->y_final, y0, sizeof(double) * ORC_N);
        return;
    }
    double atol[ORC_N];
    for (int b = 0; b < 4; ++b)
        for (int j = 0; j < 3; ++j) atol[3 * b + j] = (b % 2 == 0) ? s->atol_pos : s->atol_vel;

    ionatom_obs o;
    memset(&o, 0, sizeof(o));
    o.ctx.sys = s;
    o.ctx.phi0 = phi0;
    o.r0sq = s->r0 * s->r0;
    o.rdot_prev = rdot_times_r(y0);
    double y[ORC_N];
    memcpy(y, y0, sizeof(y));
    orc_loop_state st;
    dp5_drive(ionatom_rhs, &o.ctx, ORC_N, 0.0, s->t_max, y, s->rtol, atol, s->h_max, 0.0,
              s->max_attempts, ionatom_on_accept, &o, &st, NULL, nz);

    double t_f;
    if (o.exited) {
        memcpy(r->y_final, o.y_exit, sizeof(double) * ORC_N);
        t_f = o.t_exit;
        r->status = o.exit_flags;
    } else {
        memcpy(r->y_final, y, sizeof(double) * ORC_N);
        t_f = st.t;
        r->status = st.status;
    }
    r->t_final = t_f;
    r->n_steps = st.n_steps;
    r->n_rej = st.n_rej;
    r->n_bounce = o.n_bounce;
    r->t_first_bounce = o.t_first;
    r->t_last_bounce = o.t_last;
    if (o.n_bounce >= 2) r->status |= ORC_COMPLEX;

    /* Fig. 1 caption: scattering angle between initial and final atom velocity (written as atan2 of
     * |v_i x v_f| and v_i . v_f, equal to the printed arccos and well conditioned near 0 and pi);
     * momentum transfer |p_f - p_i| of the atom. Ion energy change: Eq. 1's ion terms. */
    const double* v0 = y0 + 9;
    const double* vf = r->y_final + 9;
    double cr[3] = {v0[1] * vf[2] - v0[2] * vf[1], v0[2] * vf[0] - v0[0] * vf[2],
                    v0[0] * vf[1] - v0[1] * vf[0]};
    r->theta_s = atan2(sqrt(dot3(cr, cr)), dot3(v0, vf));
    double dv[3] = {vf[0] - v0[0], vf[1] - v0[1], vf[2] - v0[2]};
    r->dp = s->m_atom * sqrt(dot3(dv, dv));
    r->dE_ion = ion_energy(s, phi0, t_f, r->y_final) - ion_energy(s, phi0, 0.0, y0);
}

void orc_trajectory(const orc_system* s, const double* y0, double phi0, orc_result* r)
{
    trajectory(s, y0, phi0, r, NULL);
}

/* Batch over n trajectories: y0 is n x 12 row-major; sys_id may be NULL (all system 0). */
void orc_run_batch(const orc_system* systems, int32_t n_sys, const int32_t* sys_id,
                   const double* y0, const double* phi0, int64_t n, orc_result* out, int32_t nthreads)
{
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int64_t i = 0; i < n; ++i) {
        int32_t sid = sys_id ? sys_id[i] : 0;
        if (sid < 0 || sid >= n_sys) {
            memset(&out[i], 0, sizeof(orc_result));
            out[i].status = ORC_BAD_IC;
            continue;
        }
        orc_trajectory(&systems[sid], y0 + ORC_N * i, phi0[i], &out[i]);
    }
}

/* The same batch under the rounding-noise model (test hook): trajectory i draws its noise from
 * (seed, i), moving every component by up to `ulps` ulps after each accepted step. */
void orc_run_batch_noise(const orc_system* systems, int32_t n_sys, const int32_t* sys_id, const double* y0,
                         const double* phi0, int64_t n, orc_result* out, int32_t nthreads, uint64_t seed,
                         int32_t ulps)
{
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int64_t i = 0; i < n; ++i) {
        int32_t sid = sys_id ? sys_id[i] : 0;
        if (sid < 0 || sid >= n_sys) {
            memset(&out[i], 0, sizeof(orc_result));
            out[i].status = ORC_BAD_IC;
            continue;
        }
        orc_noise nz = {seed, (uint64_t)i, ulps};
        trajectory(&systems[sid], y0 + ORC_N * i, phi0[i], &out[i], &nz);
    }
}

int32_t orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Right-hand side of the ion-atom system, exposed for tests. */
void orc_ionatom_rhs(const orc_system* s, double phi0, double t, const double* y, double* f)
{
    ionatom_ctx c = {s, phi0};
    ionatom_rhs(&c, t, y, f);
}

double orc_ion_energy(const orc_system* s, double phi0, double t, const double* y)
{
    return ion_energy(s, phi0, t, y);
}

/* ------------------------------------------------------------------------------------------ */
/* Test problems for the integrator alone (pin the tableau, controller and continuous extension) */

typedef struct {
    int kind;     /* 0: y' = lam*y (n=1); 1: harmonic oscillator x'' = -w^2 x (n=2); 2: x'' = -w^2 x
                     for three independent oscillators with w, 2w, 3w (n=6) */
    double p;
} test_ctx;

static void test_rhs(const void* vctx, double t, const double* y, double* f)
{
    (void)t;
    const test_ctx* c = (const test_ctx*)vctx;
    if (c->kind == 0) {
        f[0] = c->p * y[0];
    } else if (c->kind == 1) {
        f[0] = y[1];
        f[1] = -c->p * c->p * y[0];
    } else {
        for (int m = 0; m < 3; ++m) {
            double w = c->p * (m + 1);
            f[2 * m] = y[2 * m + 1];
            f[2 * m + 1] = -w * w * y[2 * m];
        }
    }
}

static int test_n(int kind) { return kind == 0 ? 1 : (kind == 1 ? 2 : 6); }

/* Adaptive solve of a test problem from t = 0 to t_end; y in/out. */
void orc_test_solve(int32_t kind, double p, double t_end, double rtol, double atol, double hmax,
                    double* y, int64_t* n_steps, int64_t* n_rej)
{
    test_ctx c = {kind, p};
    int n = test_n(kind);
    double at[ORC_N];
    for (int i = 0; i < n; ++i) at[i] = atol;
    orc_loop_state st;
    dp5_drive(test_rhs, &c, n, 0.0, t_end, y, rtol, at, hmax, 0.0, INT64_MAX, NULL, NULL, &st, NULL, NULL);
    *n_steps = st.n_steps;
    *n_rej = st.n_rej;
}

/* Adaptive solve of a test problem from t = 0 to t_end starting with step h0 (> 0; 0 = ode45's
 * initial-step rule), recording every attempted step: start time, step size, error measure, accepted
 * (at most cap records). Returns the number of records. y in/out. */
int64_t orc_test_trace(int32_t kind, double p, double t_end, double rtol, double atol, double hmax, double h0,
                       double* y, int64_t cap, double* t_out, double* h_out, double* err_out, int32_t* acc_out)
{
    test_ctx c = {kind, p};
    int n = test_n(kind);
    double at[ORC_N];
    for (int i = 0; i < n; ++i) at[i] = atol;
    orc_trace tr = {cap, 0, t_out, h_out, err_out, acc_out};
    orc_loop_state st;
    dp5_drive(test_rhs, &c, n, 0.0, t_end, y, rtol, at, hmax, h0, cap, NULL, NULL, &st, &tr, NULL);
    return tr.n;
}

/* nsteps fixed steps of size h of a test problem; y in/out, err_out = last step's error estimate. */
void orc_test_fixed(int32_t kind, double p, double h, int64_t nsteps, double* y, double* err_out)
{
    test_ctx c = {kind, p};
    int n = test_n(kind);
    double k[7][ORC_N], ynew[ORC_N], err[ORC_N];
    double t = 0.0;
    for (int64_t s = 0; s < nsteps; ++s) {
        test_rhs(&c, t, y, k[0]);
        dp5_attempt(test_rhs, &c, n, t, y, h, k, ynew, err);
        for (int i = 0; i < n; ++i) {
            y[i] = ynew[i];
            err_out[i] = err[i];
        }
        t += h;
    }
}

/* One step of size h from y, then the continuous extension at fraction s; out = y(s h). */
void orc_test_dense(int32_t kind, double p, double h, double s, const double* y, double* out)
{
    test_ctx c = {kind, p};
    int n = test_n(kind);
    double k[7][ORC_N], ynew[ORC_N], err[ORC_N];
    test_rhs(&c, 0.0, y, k[0]);
    dp5_attempt(test_rhs, &c, n, 0.0, y, h, k, ynew, err);
    dp5_dense(n, y, h, k, s, out);
}

/* Fixed-step DP5 on the ion-atom system (no events): the same stages as the adaptive path, used by
 * tests that compare against an independent fixed-step integrator. y in/out. */
void orc_ionatom_fixed(const orc_system* s, double phi0, double t0, double h, int64_t nsteps, double* y)
{
    ionatom_ctx c = {s, phi0};
    double k[7][ORC_N], ynew[ORC_N], err[ORC_N];
    double t = t0;
    for (int64_t m = 0; m < nsteps; ++m) {
        ionatom_rhs(&c, t, y, k[0]);
        dp5_attempt(ionatom_rhs, &c, ORC_N, t, y, h, k, ynew, err);
        for (int i = 0; i < ORC_N; ++i) y[i] = ynew[i];
        t = t0 + (double)(m + 1) * h;
    }
}

/* Adaptive DP5 on the ion-atom system from t0 to t1 without events; y in/out. */
void orc_ionatom_segment(const orc_system* s, double phi0, double t0, double t1, double* y,
                         int64_t* n_steps, int64_t* n_rej)
{
    ionatom_ctx c = {s, phi0};
    double atol[ORC_N];
    for (int b = 0; b < 4; ++b)
        for (int j = 0; j < 3; ++j) atol[3 * b + j] = (b % 2 == 0) ? s->atol_pos : s->atol_vel;
    orc_loop_state st;
    dp5_drive(ionatom_rhs, &c, ORC_N, t0, t1, y, s->rtol, atol, s->h_max, 0.0, s->max_attempts,
              NULL, NULL, &st, NULL, NULL);
    *n_steps = st.n_steps;
    *n_rej = st.n_rej;
}

/* ------------------------------------------------------------------------------------------ */
/* Differentiation along a frozen step sequence (the derivative of the computed map with the     */
/* accepted step sizes held fixed), used to check the tangent and adjoint kernels.               */

typedef struct {
    ionatom_obs o;
    double* hs;
    int64_t cap, n;
} steps_obs;

static int record_on_accept(void* vobs, double t_old, const double* y_old, double h, const double* y_new,
                            double k[7][ORC_N])
{
    steps_obs* so = (steps_obs*)vobs;
    if (so->n < so->cap) so->hs[so->n] = h;
    so->n += 1;
    return ionatom_on_accept(&so->o, t_old, y_old, h, y_new, k);
}

/* orc_trajectory that also records the accepted step sizes (hs, up to cap) and how the trajectory
 * ended: *mode = 0 crossing inside the last step, 1 otherwise (the end of the last step is final). */
int64_t orc_trajectory_steps(const orc_system* s, const double* y0, double phi0, orc_result* r, double* hs,
                             int64_t cap, int32_t* mode)
{
    orc_trajectory(s, y0, phi0, r);
    /* repeat the integration with the recording callback (same arithmetic, same decisions) */
    double atol[ORC_N];
    for (int b = 0; b < 4; ++b)
        for (int j = 0; j < 3; ++j) atol[3 * b + j] = (b % 2 == 0) ? s->atol_pos : s->atol_vel;
    steps_obs so;
    memset(&so, 0, sizeof(so));
    so.o.ctx.sys = s;
    so.o.ctx.phi0 = phi0;
    so.o.r0sq = s->r0 * s->r0;
    so.o.rdot_prev = rdot_times_r(y0);
    so.hs = hs;
    so.cap = cap;
    double y[ORC_N];
    memcpy(y, y0, sizeof(y));
    orc_loop_state st;
    dp5_drive(ionatom_rhs, &so.o.ctx, ORC_N, 0.0, s->t_max, y, s->rtol, atol, s->h_max, 0.0,
              s->max_attempts, record_on_accept, &so, &st, NULL, NULL);
    *mode = (so.o.exited && so.o.exit_flags == 0) ? 0 : 1;
    return so.n;
}

/* Jacobian of the right-hand side with respect to y (12 x 12, row-major), from V'(r) and V''(r):
 * the force on the atom F(d) = -V'(r) d/r has dF/dd = -V'' dd^T/r^2 - (V'/r)(I - dd^T/r^2). */
static void ionatom_jac(const orc_system* s, double phi0, double t, const double* y, double J[ORC_N][ORC_N])
{
    double C4 = sys_C4(s), C8 = sys_C8(s);
    double d[3];
    separation(y, d);
    double r = sqrt(dot3(d, d));
    double V1 = -8.0 * C8 / pow(r, 9) + 4.0 * C4 / pow(r, 5);
    double V2 = 72.0 * C8 / pow(r, 10) - 20.0 * C4 / pow(r, 6);
    double dF[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double nn = d[a] * d[b] / (r * r);
            dF[a][b] = -V2 * nn - (V1 / r) * ((a == b ? 1.0 : 0.0) - nn);
        }
    double cosv = (double)s->rf_sign * cos(s->Omega * t + phi0);
    memset(J, 0, sizeof(double) * ORC_N * ORC_N);
    for (int j = 0; j < 3; ++j) {
        J[0 + j][3 + j] = 1.0;
        J[6 + j][9 + j] = 1.0;
        J[3 + j][0 + j] = -(s->Omega * s->Omega / 4.0) * (s->a[j] + 2.0 * s->q[j] * cosv);
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            J[3 + a][0 + b] += dF[a][b] / s->m_ion;   /* d a_ion / d x_ion */
            J[3 + a][6 + b] += -dF[a][b] / s->m_ion;  /* d a_ion / d x_atom */
            J[9 + a][6 + b] += dF[a][b] / s->m_atom;  /* d a_atom / d x_atom */
            J[9 + a][0 + b] += -dF[a][b] / s->m_atom; /* d a_atom / d x_ion */
        }
}

/* d f / d q_j (q-vector direction dq): only the ion acceleration depends on q. */
static void ionatom_dfdq(const orc_system* s, double phi0, double t, const double* y, const double* dq, double* out)
{
    double cosv = (double)s->rf_sign * cos(s->Omega * t + phi0);
    memset(out, 0, sizeof(double) * ORC_N);
    for (int j = 0; j < 3; ++j) out[3 + j] = -(s->Omega * s->Omega / 4.0) * 2.0 * dq[j] * cosv * y[j];
}

/* The continuous extension's weights b_j(s) and their s-derivatives. */
static void dense_weights(double sv, double w[7], double dw[7])
{
    for (int j = 0; j < 7; ++j) {
        w[j] = sv * (DP_BI[j][0] + sv * (DP_BI[j][1] + sv * (DP_BI[j][2] + sv * DP_BI[j][3])));
        dw[j] = DP_BI[j][0] + sv * (2.0 * DP_BI[j][1] + sv * (3.0 * DP_BI[j][2] + sv * 4.0 * DP_BI[j][3]));
    }
}

/* Observables from initial and final states (same definitions as orc_trajectory). */
static void observables(const orc_system* s, double phi0, const double* y0, const double* yf, double tf, double* obs)
{
    const double* v0 = y0 + 9;
    const double* vf = yf + 9;
    double cr[3] = {v0[1] * vf[2] - v0[2] * vf[1], v0[2] * vf[0] - v0[0] * vf[2], v0[0] * vf[1] - v0[1] * vf[0]};
    obs[0] = atan2(sqrt(dot3(cr, cr)), dot3(v0, vf));
    double dv[3] = {vf[0] - v0[0], vf[1] - v0[1], vf[2] - v0[2]};
    obs[1] = s->m_atom * sqrt(dot3(dv, dv));
    obs[2] = ion_energy(s, phi0, tf, yf) - ion_energy(s, phi0, 0.0, y0);
    obs[3] = tf;
}

/* Replay of the step sequence hs[0..nh-1] from y0 (fixed steps, no error control). mode 0: the
 * end is the crossing |d| = r0 located by bisection on the last step's continuous extension,
 * searched on s in [-0.5, 1.5] (the same polynomial, so small perturbations keep it in that step);
 * mode 1: the end of the last step. Outputs the observables (theta_s, dp, dE_ion, t_final) and y_f. */
void orc_replay(const orc_system* s, const double* y0, double phi0, const double* hs, int64_t nh, int32_t mode,
                double* obs, double* yf)
{
    ionatom_ctx c = {s, phi0};
    double y[ORC_N], k[7][ORC_N], ynew[ORC_N], err[ORC_N];
    memcpy(y, y0, sizeof(y));
    double t = 0.0;
    for (int64_t m = 0; m < nh; ++m) {
        double h = hs[m];
        ionatom_rhs(&c, t, y, k[0]);
        dp5_attempt(ionatom_rhs, &c, ORC_N, t, y, h, k, ynew, err);
        if (m == nh - 1 && mode == 0) {
            double lo = -0.5, hi = 1.5, ys[ORC_N], dd[3];
            for (int it = 0; it < 200; ++it) {
                double mid = 0.5 * (lo + hi);
                if (mid <= lo || mid >= hi) break;
                dp5_dense(ORC_N, y, h, k, mid, ys);
                separation(ys, dd);
                if (dot3(dd, dd) - s->r0 * s->r0 < 0.0)
                    lo = mid;
                else
                    hi = mid;
            }
            dp5_dense(ORC_N, y, h, k, hi, yf);
            observables(s, phi0, y0, yf, t + hi * h, obs);
            return;
        }
        memcpy(y, ynew, sizeof(y));
        t = t + h;
    }
    memcpy(yf, y, sizeof(y));
    observables(s, phi0, y0, yf, t, obs);
}

/* Discrete tangent of the replayed map along ndir directions: Y (12 per direction) follows the
 * stages K_s = J(t_s, y_s) Y_s + (df/dq) dq, Y_s = Y + h sum_l a_sl K_l, Y_new = Y + h sum_l b_l K_l;
 * at a crossing (mode 0) d s_star / d p = -(d . dY_d) / (d . dd/ds) on the continuous extension and
 * dy_f = Y(s_star) + (dy/ds) d s_star. The observables are differentiated by hand below.
 * dy0: ndir x 12; dq: ndir x 3; out: ndir x 4 (theta_s, dp, dE_ion, t_final); dyf: ndir x 12. */
void orc_tangent(const orc_system* s, const double* y0, double phi0, const double* hs, int64_t nh, int32_t mode,
                 const double* dy0, const double* dq, int32_t ndir, double* out, double* dyf)
{
    ionatom_ctx c = {s, phi0};
    enum { MAXD = 4 };
    double y[ORC_N], k[7][ORC_N], ys[ORC_N];
    double Y[MAXD][ORC_N], K[MAXD][7][ORC_N], Ys[MAXD][ORC_N];
    double J[ORC_N][ORC_N], fq[ORC_N];
    memcpy(y, y0, sizeof(y));
    for (int d = 0; d < ndir; ++d) memcpy(Y[d], dy0 + ORC_N * d, sizeof(double) * ORC_N);
    double t = 0.0, sstar = 1.0, h = 0.0, tf = 0.0;
    double yfin[ORC_N], dyfin[MAXD][ORC_N], dtf[MAXD];
    for (int d = 0; d < ndir; ++d) dtf[d] = 0.0;
    for (int64_t m = 0; m < nh; ++m) {
        h = hs[m];
        /* stages of the primal and of each direction */
        for (int st = 0; st < 7; ++st) {
            double tsv = t + DP_C[st] * h;
            for (int i = 0; i < ORC_N; ++i) {
                double acc = 0.0;
                for (int l = 0; l < st; ++l) acc += DP_A[st][l] * k[l][i];
                ys[i] = y[i] + h * acc;
            }
            ionatom_rhs(&c, tsv, ys, k[st]);
            ionatom_jac(s, phi0, tsv, ys, J);
            for (int d = 0; d < ndir; ++d) {
                for (int i = 0; i < ORC_N; ++i) {
                    double acc = 0.0;
                    for (int l = 0; l < st; ++l) acc += DP_A[st][l] * K[d][l][i];
                    Ys[d][i] = Y[d][i] + h * acc;
                }
                ionatom_dfdq(s, phi0, tsv, ys, dq + 3 * d, fq);
                for (int i = 0; i < ORC_N; ++i) {
                    double acc = fq[i];
                    for (int jj = 0; jj < ORC_N; ++jj) acc += J[i][jj] * Ys[d][jj];
                    K[d][st][i] = acc;
                }
            }
        }
        if (m == nh - 1 && mode == 0) {
            /* locate the crossing as orc_replay does, then the event sensitivity */
            double lo = -0.5, hi = 1.5, yt[ORC_N], dd[3];
            for (int it = 0; it < 200; ++it) {
                double mid = 0.5 * (lo + hi);
                if (mid <= lo || mid >= hi) break;
                dp5_dense(ORC_N, y, h, k, mid, yt);
                separation(yt, dd);
                if (dot3(dd, dd) - s->r0 * s->r0 < 0.0)
                    lo = mid;
                else
                    hi = mid;
            }
            sstar = hi;
            double w[7], dw[7];
            dense_weights(sstar, w, dw);
            double ydot[ORC_N];
            for (int i = 0; i < ORC_N; ++i) {
                double a1 = 0.0, a2 = 0.0;
                for (int j = 0; j < 7; ++j) {
                    a1 += w[j] * k[j][i];
                    a2 += dw[j] * k[j][i];
                }
                yfin[i] = y[i] + h * a1;
                ydot[i] = h * a2; /* dy/ds */
            }
            double df[3], dfs[3];
            separation(yfin, df);
            separation(ydot, dfs);
            for (int d = 0; d < ndir; ++d) {
                double Yi[ORC_N];
                for (int i = 0; i < ORC_N; ++i) {
                    double a1 = 0.0;
                    for (int j = 0; j < 7; ++j) a1 += w[j] * K[d][j][i];
                    Yi[i] = Y[d][i] + h * a1;
                }
                double dY[3];
                separation(Yi, dY);
                double ds = -dot3(df, dY) / dot3(df, dfs);
                for (int i = 0; i < ORC_N; ++i) dyfin[d][i] = Yi[i] + ydot[i] * ds;
                dtf[d] = h * ds;
            }
            tf = t + sstar * h;
            goto done;
        }
        for (int i = 0; i < ORC_N; ++i) {
            double acc = 0.0;
            for (int l = 0; l < 7; ++l) acc += DP_B[l] * k[l][i];
            y[i] = y[i] + h * acc;
        }
        for (int d = 0; d < ndir; ++d)
            for (int i = 0; i < ORC_N; ++i) {
                double acc = 0.0;
                for (int l = 0; l < 7; ++l) acc += DP_B[l] * K[d][l][i];
                Y[d][i] = Y[d][i] + h * acc;
            }
        t = t + h;
    }
    memcpy(yfin, y, sizeof(y));
    for (int d = 0; d < ndir; ++d) memcpy(dyfin[d], Y[d], sizeof(double) * ORC_N);
    tf = t;
done:
    for (int d = 0; d < ndir; ++d) {
        /* chain rule for the observables (Fig. 1 caption definitions and the ion energy of Eq. 1) */
        const double* dy0d = dy0 + ORC_N * d;
        const double* v0 = y0 + 9;
        const double* vf = yfin + 9;
        const double* dv0 = dy0d + 9;
        const double* dvf = dyfin[d] + 9;
        double cr[3] = {v0[1] * vf[2] - v0[2] * vf[1], v0[2] * vf[0] - v0[0] * vf[2], v0[0] * vf[1] - v0[1] * vf[0]};
        double dcr[3] = {dv0[1] * vf[2] + v0[1] * dvf[2] - dv0[2] * vf[1] - v0[2] * dvf[1],
                         dv0[2] * vf[0] + v0[2] * dvf[0] - dv0[0] * vf[2] - v0[0] * dvf[2],
                         dv0[0] * vf[1] + v0[0] * dvf[1] - dv0[1] * vf[0] - v0[1] * dvf[0]};
        double C = sqrt(dot3(cr, cr)), D = dot3(v0, vf);
        double dC = C > 0.0 ? dot3(cr, dcr) / C : 0.0;
        double dD = dot3(dv0, vf) + dot3(v0, dvf);
        out[4 * d + 0] = (D * dC - C * dD) / (C * C + D * D);
        double u[3] = {vf[0] - v0[0], vf[1] - v0[1], vf[2] - v0[2]};
        double du[3] = {dvf[0] - dv0[0], dvf[1] - dv0[1], dvf[2] - dv0[2]};
        double un = sqrt(dot3(u, u));
        out[4 * d + 1] = un > 0.0 ? s->m_atom * dot3(u, du) / un : 0.0;
        /* E_ion(t, y; q) = m/2 |v_i|^2 + sum_j (m Omega^2/8)(a_j + 2 s q_j cos(Omega t + phi0)) x_j^2 */
        double W = s->m_ion * s->Omega * s->Omega / 8.0;
        double sg = (double)s->rf_sign;
        double cf = cos(s->Omega * tf + phi0), sf = sin(s->Omega * tf + phi0), c0 = cos(phi0);
        const double* dqd = dq + 3 * d;
        double e = 0.0;
        for (int j = 0; j < 3; ++j) {
            double xf = yfin[j], x0 = y0[j];
            e += s->m_ion * (yfin[3 + j] * dyfin[d][3 + j] - y0[3 + j] * dy0d[3 + j]);
            e += 2.0 * W * (s->a[j] + 2.0 * sg * s->q[j] * cf) * xf * dyfin[d][j];
            e -= 2.0 * W * (s->a[j] + 2.0 * sg * s->q[j] * c0) * x0 * dy0d[j];
            e += W * 2.0 * sg * s->q[j] * (-s->Omega * sf) * xf * xf * dtf[d];
            e += W * 2.0 * sg * dqd[j] * (cf * xf * xf - c0 * x0 * x0);
        }
        out[4 * d + 2] = e;
        out[4 * d + 3] = dtf[d];
        if (dyf) memcpy(dyf + ORC_N * d, dyfin[d], sizeof(double) * ORC_N);
    }
}

/* ------------------------------------------------------------------------------------------ */
/* The same frozen-step replay in IEEE quad precision (_Float128, 113-bit mantissa, with glibc's    */
/* f128 functions; the same format on x86-64 and aarch64). FP64 rounding is amplified ~10^7-10^8   */
/* by a bounce, which floors finite differences of the FP64 replay near 1e-5 (and of an 80-bit      */
/* replay near 1e-6 at 1.5 uK); in quad precision the rounding of the replay is ~1e-34 and the      */
/* differences resolve the discrete derivative far below the FP64 tangent's own rounding.           */

typedef _Float128 qreal;


static void rhs_q(const orc_system* s, const qreal* qv, qreal phi0, qreal t, const qreal* y, qreal* f)
{
    qreal C4 = (qreal)0.5 * (qreal)s->alpha;
    qreal C8 = C4 == (qreal)0.0 ? (qreal)0.0 : C4 * C4 / ((qreal)4.0 * (qreal)s->De);
    qreal d[3];
    for (int j = 0; j < 3; ++j) d[j] = y[6 + j] - y[j];
    qreal r = sqrtf128(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    qreal dVdr = (qreal)-8.0 * C8 / powf128(r, 9) + (qreal)4.0 * C4 / powf128(r, 5);
    qreal Om = (qreal)s->Omega;
    qreal cosv = (qreal)s->rf_sign * cosf128(Om * t + phi0);
    for (int j = 0; j < 3; ++j) {
        qreal Fa = -dVdr * d[j] / r;
        qreal Ft = -((qreal)s->m_ion * Om * Om / (qreal)4.0) * ((qreal)s->a[j] + (qreal)2.0 * qv[j] * cosv) * y[j];
        f[0 + j] = y[3 + j];
        f[3 + j] = (Ft - Fa) / (qreal)s->m_ion;
        f[6 + j] = y[9 + j];
        f[9 + j] = Fa / (qreal)s->m_atom;
    }
}

static qreal ion_energy_q(const orc_system* s, const qreal* qv, qreal phi0, qreal t, const qreal* y)
{
    qreal Om = (qreal)s->Omega;
    qreal cosv = (qreal)s->rf_sign * cosf128(Om * t + phi0);
    qreal E = (qreal)0.0;
    for (int j = 0; j < 3; ++j) {
        E += (qreal)0.5 * (qreal)s->m_ion * y[3 + j] * y[3 + j];
        E += ((qreal)s->a[j] + (qreal)2.0 * qv[j] * cosv) * ((qreal)s->m_ion * Om * Om / (qreal)8.0) * y[j] * y[j];
    }
    return E;
}

/* Replay from the initial state y0 + eps dy0 with q + eps dq, both formed in quad precision; the
 * observables (theta_s, dp, dE_ion, t_final) in quad precision. */
static void replay_q(const orc_system* s, const double* y0d, const double* dy0, const double* dq, qreal eps,
                     double phi0d, const double* hs, int64_t nh, int32_t mode, qreal* obs)
{
    qreal y[ORC_N], k[7][ORC_N], ys[ORC_N], y0[ORC_N], qv[3];
    qreal phi0 = (qreal)phi0d;
    for (int i = 0; i < ORC_N; ++i) y0[i] = y[i] = (qreal)y0d[i] + eps * (qreal)dy0[i];
    for (int j = 0; j < 3; ++j) qv[j] = (qreal)s->q[j] + eps * (qreal)dq[j];
    qreal t = (qreal)0.0;
    qreal yf[ORC_N];
    qreal tf = (qreal)0.0;
    for (int64_t m = 0; m < nh; ++m) {
        qreal h = (qreal)hs[m];
        rhs_q(s, qv, phi0, t, y, k[0]);
        for (int st = 1; st < 7; ++st) {
            for (int i = 0; i < ORC_N; ++i) {
                qreal acc = (qreal)0.0;
                for (int l = 0; l < st; ++l) acc += (qreal)DP_A[st][l] * k[l][i];
                ys[i] = y[i] + h * acc;
            }
            rhs_q(s, qv, phi0, t + (qreal)DP_C[st] * h, ys, k[st]);
        }
        if (m == nh - 1 && mode == 0) {
            qreal lo = (qreal)-0.5, hi = (qreal)1.5, r0sq = (qreal)s->r0 * (qreal)s->r0;
            for (int it = 0; it < 400; ++it) {
                qreal mid = (qreal)0.5 * (lo + hi);
                if (mid <= lo || mid >= hi) break;
                qreal d2 = (qreal)0.0;
                for (int j = 0; j < 3; ++j) {
                    qreal pa = (qreal)0.0, pi = (qreal)0.0;
                    for (int jj = 0; jj < 7; ++jj) {
                        qreal w = mid * ((qreal)DP_BI[jj][0] + mid * ((qreal)DP_BI[jj][1] + mid * ((qreal)DP_BI[jj][2] +
                                        mid * (qreal)DP_BI[jj][3])));
                        pa += w * k[jj][6 + j];
                        pi += w * k[jj][j];
                    }
                    qreal dj = (y[6 + j] + h * pa) - (y[j] + h * pi);
                    d2 += dj * dj;
                }
                if (d2 - r0sq < (qreal)0.0)
                    lo = mid;
                else
                    hi = mid;
            }
            for (int i = 0; i < ORC_N; ++i) {
                qreal acc = (qreal)0.0;
                for (int jj = 0; jj < 7; ++jj) {
                    qreal w = hi * ((qreal)DP_BI[jj][0] + hi * ((qreal)DP_BI[jj][1] + hi * ((qreal)DP_BI[jj][2] +
                                   hi * (qreal)DP_BI[jj][3])));
                    acc += w * k[jj][i];
                }
                yf[i] = y[i] + h * acc;
            }
            tf = t + hi * h;
            goto done;
        }
        for (int i = 0; i < ORC_N; ++i) {
            qreal acc = (qreal)0.0;
            for (int l = 0; l < 7; ++l) acc += (qreal)DP_B[l] * k[l][i];
            y[i] = y[i] + h * acc;
        }
        t = t + h;
    }
    for (int i = 0; i < ORC_N; ++i) yf[i] = y[i];
    tf = t;
done:
    {
        const qreal* v0 = y0 + 9;
        const qreal* vf = yf + 9;
        qreal cr[3] = {v0[1] * vf[2] - v0[2] * vf[1], v0[2] * vf[0] - v0[0] * vf[2], v0[0] * vf[1] - v0[1] * vf[0]};
        obs[0] = atan2f128(sqrtf128(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]),
                                v0[0] * vf[0] + v0[1] * vf[1] + v0[2] * vf[2]);
        qreal dv[3] = {vf[0] - v0[0], vf[1] - v0[1], vf[2] - v0[2]};
        obs[1] = (qreal)s->m_atom * sqrtf128(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
        obs[2] = ion_energy_q(s, qv, phi0, tf, yf) - ion_energy_q(s, qv, phi0, (qreal)0.0, y0);
        obs[3] = tf;
    }
}

/* Central differences of the quad-precision replay along direction (dy0, dq), with the perturbed
 * initial state and q formed in quad precision; Richardson-combined spacings delta and delta/2
 * (truncation O(delta^4)), all in quad precision. out: derivatives of (theta_s, dp, dE_ion, t_final). */
void orc_fd_ld(const orc_system* s, const double* y0, double phi0, const double* hs, int64_t nh, int32_t mode,
               const double* dy0, const double* dq, double delta, double* out)
{
    qreal D[2][4];
    for (int pass = 0; pass < 2; ++pass) {
        qreal dl = pass == 0 ? (qreal)delta : (qreal)0.5 * (qreal)delta;
        qreal op[4], om[4];
        replay_q(s, y0, dy0, dq, dl, phi0, hs, nh, mode, op);
        replay_q(s, y0, dy0, dq, -dl, phi0, hs, nh, mode, om);
        for (int o = 0; o < 4; ++o) D[pass][o] = (op[o] - om[o]) / ((qreal)2.0 * dl);
    }
    for (int o = 0; o < 4; ++o) out[o] = (double)(((qreal)4.0 * D[1][o] - D[0][o]) / (qreal)3.0);
}
