// ia_traj.cuh -- device code: classical ion-atom trajectories integrated with Dormand-Prince 5(4)
// in the form that suits x'' = a(t, x), reduced on the fly to the observables.
//
// Method (arXiv 2509.15117): Eq. 1 gives the forces (Paul trap on the ion, V = C8/r^8 - C4/r^4
// between ion and atom, text after Eq. 1); integrator DP5(4) with the step control of ode45
// (Dormand & Prince 1980, Shampine & Reichelt 1997); a trajectory ends at the outward crossing of
// |x_a - x_i| = r0 (head-on paragraph) or at t_max; observables of the Fig. 1 caption.
//
// Two execution layouts share every arithmetic expression, so they give the same bits:
//   lane mode   one trajectory per lane (bulk throughput);
//   group mode  one trajectory per group of G lanes, lane c holding component c of
//               [x_ion(3), x_atom(3)] with its velocity and stage accelerations (low latency for the
//               few trajectories that run 10^5-10^7 steps: long-lived complexes).
//
// GB300 notes. One FP64 warp instruction occupies an SM sub-partition's FP64 unit for ~68 cycles
// whatever the number of active lanes, and a dependent FP64 result is ready after the same ~68
// cycles; FP32 and integer instructions are ~60x cheaper. So this file spends FP64 instructions only
// on the method's arithmetic:
//   * stage velocities are never formed (Nystrom form, gen_dp5_nystrom.py);
//   * comparisons and max/min of non-negative doubles are integer operations on their bit patterns;
//   * 1/r^2 is a Newton-Raphson refinement of an FP32 seed (two iterations, ~1 ulp);
//   * the step-size factor (a smooth function of the error ratio, not a decision) is computed in
//     FP32; the accept/reject decision stays exact in FP64;
//   * float <-> double conversions are integer operations on the bit patterns;
//   * in group mode, per-step scalars are spread over the lanes of a group and exchanged by shuffles,
//     and two independent products share one FMA instruction on different lanes.
// The library is compiled with -fmad=false: only explicit fma() calls fuse, so the same expression
// gives the same bits in both layouts.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dp5_nystrom.h"

namespace ia {

constexpr unsigned FULL = 0xffffffffu;

// Per-system constants, precomputed on the host from ia_system_desc.
struct SysDev {
    double inv_mi, inv_ma;  // 1/m
    double neg_inv_mi;      // -1/m_i
    double c8x8, c4x4;      // 8 C8, 4 C4: -V'(r)/r = s^3 (8 C8 s^2 - 4 C4), s = 1/r^2
    double ci8, ci4;        // -8 C8 / m_i, -4 C4 / m_i: ion acceleration per unit separation = s^3 (ci8 s^2 - ci4)
    double ca8, ca4;        // 8 C8 / m_a, 4 C4 / m_a: the same for the atom
    double Omega;
    double ka[3];           // ion acceleration per unit displacement, static part: -(Omega^2/4) a_j
    double kq[3];           // rf part, times cos(Omega t + phi0): -(Omega^2/4) 2 s q_j
    double ua[3];           // ion trap energy per unit displacement^2, static: (m_i Omega^2 / 8) a_j
    double uq[3];           // rf part, times cos: (m_i Omega^2 / 8) 2 s q_j
    double m_i, m_a;
    double r0sq;
    double t_max, h_max;
    double rtol, atol_pos, atol_vel;
    double thr_pos, thr_vel;  // atol / rtol, used by the initial-step rule
    double hinit_den;         // 0.8 rtol^(1/5)
    long long max_attempts;
    // derivatives and scales used by the tangent kernel
    double kq_per_q;          // d kq_j / d q_j = -(Omega^2/4) 2 s
    double uq_per_q;          // d uq_j / d q_j = (m_i Omega^2 / 8) 2 s
    double inv_len, inv_vel;  // 1/r_e and 1/sqrt(2 D_e / mu): units of the FTLE norm
};

// Output pointers (device, SoA).
struct ObsPtrs {
    double* theta_s;
    double* dp;
    double* dE_ion;
    double* t_final;
    double* t_first;
    double* t_last;
    int32_t* n_bounce;
    uint32_t* status;
    int32_t* n_steps;
    int32_t* n_rej;
    double* y_final;
    long long ld_out;
};

struct IcPtrs {
    const double* y0;
    const double* phi0;
    const int32_t* sys_id;
    const long long* order;  // queue position -> trajectory index, or null (identity)
    long long ld;
};

enum : uint32_t {
    ST_EXIT = 0u,
    ST_TMAX = 1u << 0,
    ST_MAX_STEPS = 1u << 1,
    ST_H_UNDERFLOW = 1u << 2,
    ST_NONFINITE = 1u << 3,
    ST_BAD_IC = 1u << 4,
    ST_EXIT_OUTSIDE = 1u << 5,
    ST_COMPLEX = 1u << 8,
};

// Saved state of a trajectory moved from lane mode to group mode (256 bytes).
// Components are ordered [x_ion(3), x_atom(3)].
struct __align__(16) Susp {
    double x[6], v[6], a1[6];
    double t, h, phi0, rdot_prev, t_first, t_last;
    long long idx;
    int sid, n_acc, n_rej, n_bounce, flags, pad0;
    double pad1[4];
};
static_assert(sizeof(Susp) == 256, "Susp layout");

// ---------------------------------------------------------------------------------------------
// Bit-level helpers (integer pipe).

__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ double dabs(double x)
{
    return __longlong_as_double(__double_as_longlong(x) & 0x7fffffffffffffffLL);
}
// For non-negative doubles (including +0) the bit patterns order like the values.
__device__ __forceinline__ bool nn_le(double a, double b) { return dbits(a) <= dbits(b); }
__device__ __forceinline__ bool nn_lt(double a, double b) { return dbits(a) < dbits(b); }
__device__ __forceinline__ double nn_max(double a, double b) { return dbits(a) >= dbits(b) ? a : b; }
__device__ __forceinline__ double nn_min(double a, double b) { return dbits(a) <= dbits(b) ? a : b; }
// x < 0 (a negative zero counts as zero)
__device__ __forceinline__ bool is_neg(double x)
{
    long long b = dbits(x);
    return b < 0 && (b & 0x7fffffffffffffffLL) != 0;
}
__device__ __forceinline__ bool is_finite(double x)
{
    return (__double2hiint(x) & 0x7ff00000) != 0x7ff00000;
}
// Non-negative double to float by truncating the mantissa (relative error < 2^-20); values below
// 2^-126 become 0, values above 2^127 become +inf. Integer instructions only.
__device__ __forceinline__ float nn_to_float(double x)
{
    int hi = __double2hiint(x);
    int e = (hi >> 20) & 0x7ff;
    if (e < 1023 - 126) return 0.0f;
    if (e > 1023 + 127) return __int_as_float(0x7f800000);
    return __int_as_float(((hi - ((1023 - 127) << 20)) << 3));
}
// Positive normal float to double, exactly. Integer instructions only.
__device__ __forceinline__ double pos_float_to_double(float f)
{
    unsigned u = __float_as_uint(f);
    int hi = (int)((u >> 3) + ((1023u - 127u) << 20));
    int lo = (int)(u << 29);
    return __hiloint2double(hi, lo);
}
// 16 times the spacing of doubles at t >= 0 (ode45's minimum step 16 eps(t)).
__device__ __forceinline__ double hmin_at(double t)
{
    int hi = __double2hiint(t);
    int e = (hi >> 20) & 0x7ff;  // biased exponent of t
    if (e < 53 + 1) return 16.0 * 2.2250738585072014e-308;
    // spacing = 2^(e - 1023 - 52); times 16 = 2^(e - 1071)
    return __hiloint2double((e - 48) << 20, 0);
}

__device__ __forceinline__ float rcp_approx_f32(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1/x for x > 0 from the FP32 hardware reciprocal of x truncated to float (seed y0 with relative
// error < 2^-19), refined by one third-order step of the iteration for 1/x (Householder's method of
// order 3; equivalently the geometric series 1/x = y0 / (1 - e) = y0 (1 + e + e^2 + ...) truncated
// after e^2, with e = 1 - x y0): y = y0 + y0 (e + e^2). The truncation error e^3 < 2^-57 is far below
// the final rounding, so the result is within an ulp of 1/x; three dependent FMAs instead of the four
// of two Newton steps. Falls back to division outside the float range.
__device__ __forceinline__ double rcp_nr(double x)
{
    int e = (__double2hiint(x) >> 20) & 0x7ff;
    if (e < 1023 - 120 || e > 1023 + 120) return 1.0 / x;
    const double y = pos_float_to_double(rcp_approx_f32(nn_to_float(x)));
    const double r = fma(-x, y, 1.0);
    return fma(y, fma(r, r, r), y);
}

__device__ __forceinline__ double ion_energy(const SysDev& P, double cs, const double xi[3], const double vi[3])
{
    double k = 0.5 * P.m_i * fma(vi[0], vi[0], fma(vi[1], vi[1], vi[2] * vi[2]));
    double u = fma(P.uq[0], cs, P.ua[0]) * (xi[0] * xi[0]);
    u = fma(fma(P.uq[1], cs, P.ua[1]), xi[1] * xi[1], u);
    u = fma(fma(P.uq[2], cs, P.ua[2]), xi[2] * xi[2], u);
    return k + u;
}

// Lane-mode accelerations at positions (xi, xa) with cs = cos(Omega t + phi0) (Eq. 1 and V).
// Ion: (ka + kq cs) x_i - (g / m_i) d;  atom: (g / m_a) d;  d = x_a - x_i.
__device__ __forceinline__ void accel(const SysDev& P, const double xi[3], const double xa[3], double cs,
                                      double ai[3], double aa[3], double& r2out, double dout[3])
{
    double d0 = xa[0] - xi[0], d1 = xa[1] - xi[1], d2 = xa[2] - xi[2];
    double r2 = fma(d0, d0, fma(d1, d1, d2 * d2));
    // -V'(r)/(r m) = s^3 (8 C8 s^2 - 4 C4) / m with s = 1/r^2, the 1/m folded into the constants
    const double s = rcp_nr(r2);
    const double s2 = s * s;
    const double s3 = fma(s2, s, 0.0);
    const double gmi = s3 * fma(P.ci8, s2, -P.ci4);
    const double gma = s3 * fma(P.ca8, s2, -P.ca4);
    aa[0] = gma * d0;
    aa[1] = gma * d1;
    aa[2] = gma * d2;
    ai[0] = fma(fma(P.kq[0], cs, P.ka[0]), xi[0], gmi * d0);
    ai[1] = fma(fma(P.kq[1], cs, P.ka[1]), xi[1], gmi * d1);
    ai[2] = fma(fma(P.kq[2], cs, P.ka[2]), xi[2], gmi * d2);
    r2out = r2;
    dout[0] = d0;
    dout[1] = d1;
    dout[2] = d2;
}

// ---------------------------------------------------------------------------------------------
// Per-component stage expressions (shared by both layouts).
// Step coefficients, all products of a tableau constant with h or h^2.
struct Coef {
    double h2, c2, c3, c4, c5;
    double w31, w41, w42, w51, w52, w53, w61, w62, w63, w64, w71, w73, w74, w75;
    double b1, b3, b4, b5, b6;
    double e1, e3, e4, e5, e6, e7;
    double f1, f3, f4, f5, f6;
};
constexpr int N_COEF = 34;  // all but h2
// tableau constants in the order of Coef after h2; the second table flags the h^2 ones
__device__ __constant__ double COEF_K[N_COEF] = {
    DP_C2, DP_C3, DP_C4, DP_C5,
    DP_AA31, DP_AA41, DP_AA42, DP_AA51, DP_AA52, DP_AA53, DP_AA61, DP_AA62, DP_AA63, DP_AA64,
    DP_AA71, DP_AA73, DP_AA74, DP_AA75,
    DP_B1, DP_B3, DP_B4, DP_B5, DP_B6,
    DP_E1, DP_E3, DP_E4, DP_E5, DP_E6, DP_E7,
    DP_EA1, DP_EA3, DP_EA4, DP_EA5, DP_EA6};
__device__ __constant__ unsigned char COEF_H2[N_COEF] = {
    0, 0, 0, 0,
    1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1,
    0, 0, 0, 0, 0,
    0, 0, 0, 0, 0, 0,
    1, 1, 1, 1, 1};

__device__ __forceinline__ void coef_all(double h, Coef& K)
{
    K.h2 = h * h;
    double* out = &K.c2;
#pragma unroll
    for (int k = 0; k < N_COEF; ++k) out[k] = COEF_K[k] * (COEF_H2[k] ? K.h2 : h);
}

__device__ __forceinline__ double pos2(const Coef& K, double x, double v) { return fma(K.c2, v, x); }
__device__ __forceinline__ double pos3(const Coef& K, double x, double v, double a1)
{
    return fma(K.w31, a1, fma(K.c3, v, x));
}
__device__ __forceinline__ double pos4(const Coef& K, double x, double v, double a1, double a2)
{
    return fma(K.w42, a2, fma(K.w41, a1, fma(K.c4, v, x)));
}
__device__ __forceinline__ double pos5(const Coef& K, double x, double v, double a1, double a2, double a3)
{
    return fma(K.w53, a3, fma(K.w52, a2, fma(K.w51, a1, fma(K.c5, v, x))));
}
__device__ __forceinline__ double pos6(const Coef& K, double h, double x, double v, double a1, double a2,
                                       double a3, double a4)
{
    return fma(K.w64, a4, fma(K.w63, a3, fma(K.w62, a2, fma(K.w61, a1, fma(h, v, x)))));
}
__device__ __forceinline__ double pos7(const Coef& K, double h, double x, double v, double a1, double a3,
                                       double a4, double a5)
{
    return fma(K.w75, a5, fma(K.w74, a4, fma(K.w73, a3, fma(K.w71, a1, fma(h, v, x)))));
}
__device__ __forceinline__ double vel_new(const Coef& K, double v, double a1, double a3, double a4, double a5,
                                          double a6)
{
    return fma(K.b6, a6, fma(K.b5, a5, fma(K.b4, a4, fma(K.b3, a3, fma(K.b1, a1, v)))));
}
__device__ __forceinline__ double err_v(const Coef& K, double a1, double a3, double a4, double a5, double a6,
                                        double a7)
{
    return fma(K.e7, a7, fma(K.e6, a6, fma(K.e5, a5, fma(K.e4, a4, fma(K.e3, a3, K.e1 * a1)))));
}
__device__ __forceinline__ double err_x(const Coef& K, double a1, double a3, double a4, double a5, double a6)
{
    return fma(K.f6, a6, fma(K.f5, a5, fma(K.f4, a4, fma(K.f3, a3, K.f1 * a1))));
}

// ode45 error test of one component: ok iff |e| <= sc = max(rtol max(|y|, |ynew|), atol). The ratio
// |e| / sc is returned in FP32 (to find the component with the largest ratio cheaply), with |e| and sc.
__device__ __forceinline__ void err_check(double rtol, double atol, double y_old, double y_new, double e,
                                          bool& ok, bool& finite, float& ratio, double& ae, double& sc)
{
    double w = nn_max(dabs(y_old), dabs(y_new));
    sc = nn_max(rtol * w, atol);
    ae = dabs(e);
    ok = nn_le(ae, sc);
    finite = is_finite(y_new) && is_finite(e);
    ratio = nn_to_float(ae) * __frcp_rn(nn_to_float(sc));
}

// ode45's error measure err = max_k |e_k| / sc_k over the twelve components. The components' ratios
// are compared in FP32; the step-size rules then use the winner's |e| and sc in FP64 (ties go to the
// lowest index k in the order x_ion0, v_ion0, x_ion1, ..., x_atom2, v_atom2, the same in every layout),
// so that the step sizes follow the oracle's rules to far below the ~1e-8 by which the two sides' error
// estimates (differences of O(h) terms, summed in different orders) differ anyway.
struct ErrMax {
    unsigned long long key;  // bits of the FP32 ratio << 32 | (15 - k): larger key = larger ratio, lower k
    double ae, sc;
};
__device__ __forceinline__ unsigned long long err_key(float ratio, int k)
{
    return ((unsigned long long)__float_as_uint(ratio) << 32) | (unsigned long long)(15 - k);
}
__device__ __forceinline__ void err_take(ErrMax& m, float ratio, int k, double ae, double sc)
{
    const unsigned long long key = err_key(ratio, k);
    if (key > m.key) {
        m.key = key;
        m.ae = ae;
        m.sc = sc;
    }
}

// The error measure as the step-size rules use it: its FP32 value errf and, in FP64, the winning
// component's |e| and sc (err = ae / sc).
struct ErrMeas {
    float f;
    double ae, sc;
};

// err^(-1/5) for err = ae/sc in [0.16^5, 0.125^-5] (where the factor is not clamped): the FP32 value
// y = exp2(-0.2 log2 errf) (relative error ~2^-21) refined by one Newton step on err y^5 = 1,
// y <- y (1 - r/5), r = (ae y^5 - sc)/sc, which leaves 3 eps^2 ~ 2^-40; r is small, so forming it with
// the FP32 reciprocal of sc costs only ~2^-23 of it (~2^-46 in y).
__device__ __forceinline__ double err_pow_m02(const ErrMeas& e)
{
    const double y = pos_float_to_double(exp2f(-0.2f * __log2f(e.f)));
    const double y2 = y * y;
    const double y5 = (y2 * y2) * y;
    const double inv_sc = pos_float_to_double(rcp_approx_f32(nn_to_float(e.sc)));
    const double r = fma(e.ae, y5, -e.sc) * inv_sc;
    return fma(-0.2 * y, r, y);
}

// Step-size factors of ode45 (Shampine & Reichelt 1997). After an accepted step:
// h / (1.25 err^(1/5)) = h 0.8 err^(-1/5) when 1.25 err^(1/5) > 0.2, i.e. err > 0.16^5, else 5 h (the
// clamps decide on errf: the factor is continuous there).
__device__ __forceinline__ double grow_factor(const ErrMeas& e)
{
    return (e.f > 1.048576e-4f) ? 0.8 * err_pow_m02(e) : 5.0;
}
// After a first failure: max(0.1, 0.8 err^(-1/5)); the floor holds from err = 0.125^-5 = 32768 on.
__device__ __forceinline__ double shrink_factor(const ErrMeas& e)
{
    return (e.f < 32768.0f) ? nn_max(0.1, 0.8 * err_pow_m02(e)) : 0.1;
}

// ---------------------------------------------------------------------------------------------
// Scalars of a trajectory in flight (identical in both layouts).
struct Scal {
    double t, h, hmin, phi0;
    double rdot_prev;       // d . (v_a - v_i) at the current state
    double t_first, t_last;
    int n_acc, n_rej, n_bounce;
    bool nofailed;          // no rejection yet in the current step
    bool retry;             // the next attempt repeats the current step with a smaller h
};

// Lane-mode trajectory.
struct Lane {
    double xi[3], vi[3], xa[3], va[3];
    double a1i[3], a1a[3];  // accelerations at (t, x): first stage of the next step (FSAL)
    Scal s;
};

enum LaneResult : int { RUNNING = 0, FINISHED = 1 };

// Final state handed to the epilogue.
struct Final {
    double xi[3], vi[3], xa[3], va[3];
    double t;
    double s_exit;  // fraction of the last step at the r0 crossing (set by finish_exit; -1 otherwise)
    uint32_t status;
};

// Everything the exit epilogue needs from an accepted step, in lane-mode layout.
struct StepData {
    double xi[3], vi[3], xa[3], va[3];  // state at the step start
    double xni[3], xna[3], vni[3], vna[3];  // state at the step end
    double a1i[3], a1a[3], a3i[3], a3a[3], a4i[3], a4a[3], a5i[3], a5a[3], a6i[3], a6a[3], a7i[3], a7a[3];
    double h, t;
};

// Initial-step rule of ode45: h = min(h_max, t_max), shrunk to 1/rh with
// rh = ||f0 / max(|y0|, atol/rtol)||_inf / (0.8 rtol^(1/5)).
__device__ __forceinline__ double initial_step(const SysDev& P, const Lane& L)
{
    double h = nn_min(P.h_max, P.t_max);
    double rh = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        rh = nn_max(rh, dabs(L.vi[j]) / nn_max(dabs(L.xi[j]), P.thr_pos));
        rh = nn_max(rh, dabs(L.a1i[j]) / nn_max(dabs(L.vi[j]), P.thr_vel));
        rh = nn_max(rh, dabs(L.va[j]) / nn_max(dabs(L.xa[j]), P.thr_pos));
        rh = nn_max(rh, dabs(L.a1a[j]) / nn_max(dabs(L.va[j]), P.thr_vel));
    }
    rh = rh / P.hinit_den;
    if (h * rh > 1.0) h = 1.0 / rh;
    return h;
}

// Load trajectory i into the lane. Returns false (and fills fin as BAD_IC) if the input is unusable.
__device__ __forceinline__ bool lane_init(const SysDev& P, const IcPtrs& ic, long long i, Lane& L, Final& fin)
{
    const double* y = ic.y0 + i;
    const long long ld = ic.ld;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        L.xi[j] = __ldg(y + (0 + j) * ld);
        L.vi[j] = __ldg(y + (3 + j) * ld);
        L.xa[j] = __ldg(y + (6 + j) * ld);
        L.va[j] = __ldg(y + (9 + j) * ld);
    }
    L.s.phi0 = __ldg(ic.phi0 + i);
    bool ok = is_finite(L.s.phi0);
#pragma unroll
    for (int j = 0; j < 3; ++j)
        ok = ok && is_finite(L.xi[j]) && is_finite(L.vi[j]) && is_finite(L.xa[j]) && is_finite(L.va[j]);
    double d0 = L.xa[0] - L.xi[0], d1 = L.xa[1] - L.xi[1], d2 = L.xa[2] - L.xi[2];
    double r2 = fma(d0, d0, fma(d1, d1, d2 * d2));
    ok = ok && (dbits(r2) > 0);
    if (!ok) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            fin.xi[j] = L.xi[j]; fin.vi[j] = L.vi[j]; fin.xa[j] = L.xa[j]; fin.va[j] = L.va[j];
        }
        fin.t = 0.0;
        fin.status = ST_BAD_IC;
        return false;
    }
    double r2dummy, dd[3];
    accel(P, L.xi, L.xa, cos(L.s.phi0), L.a1i, L.a1a, r2dummy, dd);
    L.s.rdot_prev = fma(d0, L.va[0] - L.vi[0], fma(d1, L.va[1] - L.vi[1], d2 * (L.va[2] - L.vi[2])));
    L.s.t = 0.0;
    L.s.h = initial_step(P, L);
    L.s.hmin = 0.0;
    L.s.t_first = 0.0;
    L.s.t_last = 0.0;
    L.s.n_acc = 0;
    L.s.n_rej = 0;
    L.s.n_bounce = 0;
    L.s.nofailed = true;
    L.s.retry = false;
    return true;
}

// ---------------------------------------------------------------------------------------------
// Scalar control shared by both layouts.

// At the start of an attempt: the stop tests and the step clamps of ode45. Returns a stop status
// or 0xffffffff to go on.
__device__ __forceinline__ uint32_t attempt_begin(const SysDev& P, Scal& S)
{
    if (!S.retry) {
        if (nn_le(P.t_max, S.t)) return ST_TMAX;
        if ((long long)(S.n_acc + S.n_rej) >= P.max_attempts) return ST_MAX_STEPS;
        S.hmin = hmin_at(S.t);
        S.h = nn_min(S.h, P.h_max);
        S.h = nn_max(S.h, S.hmin);
        if (nn_lt(P.t_max, S.t + S.h)) S.h = P.t_max - S.t;
        S.nofailed = true;
    }
    return 0xffffffffu;
}

// After the error test of an attempt: bookkeeping of a rejection. Returns a stop status or
// 0xffffffff to go on (the attempt is repeated with the smaller h).
__device__ __forceinline__ uint32_t on_reject(const SysDev& P, Scal& S, const ErrMeas& em)
{
    const double h = S.h;
    S.n_rej += 1;
    if (nn_le(h, S.hmin)) return ST_H_UNDERFLOW;
    double fac;
    if (S.nofailed) {
        S.nofailed = false;
        fac = shrink_factor(em);  // max(0.1, 0.8 err^(-1/5))
    } else {
        fac = 0.5;
    }
    S.h = nn_max(S.hmin, h * fac);
    S.retry = true;
    if ((long long)(S.n_acc + S.n_rej) >= P.max_attempts) return ST_MAX_STEPS;
    return 0xffffffffu;
}

// After an accepted attempt: bounce bookkeeping. Returns true when the step ends beyond r0 moving
// outward (the trajectory ends in this step).
__device__ __forceinline__ bool on_accept(const SysDev& P, Scal& S, double rd, double r2new)
{
    const double t = S.t, h = S.h;
    S.n_acc += 1;
    S.retry = false;
    if (is_neg(S.rdot_prev) && !is_neg(rd)) {
        S.n_bounce += 1;
        if (S.n_bounce == 1) S.t_first = t + h;
        S.t_last = t + h;
    }
    S.rdot_prev = rd;
    return nn_le(P.r0sq, r2new) && dbits(rd) > 0;  // rd > 0
}

__device__ __forceinline__ void on_commit(const SysDev& P, Scal& S, const ErrMeas& em)
{
    const double t = S.t, h = S.h;
    S.t = nn_le(P.t_max, t + h) ? P.t_max : t + h;
    if (S.nofailed) S.h = h * grow_factor(em);
}

// ---------------------------------------------------------------------------------------------
// Exit epilogue: root of |d(s)|^2 = r0^2 on the continuous extension of the accepted step.
// d(s) = d + s h w + h^2 sum_m P_m(s) (a_a,m - a_i,m) with w = v_a - v_i; P_m(s) = sum_p PX_mp s^(p+1).
// Illinois variant of regula falsi on a bracket [lo, hi] with g(lo) < 0 <= g(hi); returns hi.
struct ExitData {
    double d[3], w[3], h;
    double da1[3], da3[3], da4[3], da5[3], da6[3];
};

__device__ __forceinline__ double exit_g(const ExitData& E, double r0sq, double s)
{
    double s2 = s * s;
    double p1 = s2 * fma(s, fma(s, DP_PX14, DP_PX13), DP_PX12);
    double p3 = s2 * fma(s, fma(s, DP_PX34, DP_PX33), DP_PX32);
    double p4 = s2 * fma(s, fma(s, DP_PX44, DP_PX43), DP_PX42);
    double p5 = s2 * fma(s, fma(s, DP_PX54, DP_PX53), DP_PX52);
    double p6 = s2 * fma(s, fma(s, DP_PX64, DP_PX63), DP_PX62);
    double sh = s * E.h, h2 = E.h * E.h;
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        double q = p1 * E.da1[j];
        q = fma(p3, E.da3[j], q);
        q = fma(p4, E.da4[j], q);
        q = fma(p5, E.da5[j], q);
        q = fma(p6, E.da6[j], q);
        double dj = fma(h2, q, fma(sh, E.w[j], E.d[j]));
        acc = fma(dj, dj, acc);
    }
    return acc - r0sq;
}

__device__ __noinline__ double locate_exit(const ExitData& E, double r0sq, double g0, double g1)
{
    double lo = 0.0, hi = 1.0, glo = g0, ghi = g1;
    int side = 0;
    for (int it = 0; it < 100; ++it) {
        if (!(hi - lo > 1e-15)) break;
        double s = (lo * ghi - hi * glo) / (ghi - glo);
        if (!(s > lo && s < hi)) s = 0.5 * (lo + hi);
        double gs = exit_g(E, r0sq, s);
        if (gs < 0.0) {
            lo = s;
            glo = gs;
            if (side == -1) ghi *= 0.5;
            side = -1;
        } else {
            hi = s;
            ghi = gs;
            if (side == +1) glo *= 0.5;
            side = +1;
        }
        if (gs == 0.0) break;
    }
    return hi;
}

// Final state of a trajectory whose accepted step (data D, end state xn/vn) ends beyond r0 moving out.
__device__ __noinline__ void finish_exit(const SysDev& P, const StepData& D, double r2new, Final& fin)
{
    const double h = D.h, t = D.t, h2 = h * h;
    double do0 = D.xa[0] - D.xi[0], do1 = D.xa[1] - D.xi[1], do2 = D.xa[2] - D.xi[2];
    double r2old = fma(do0, do0, fma(do1, do1, do2 * do2));
    if (nn_lt(r2old, P.r0sq)) {
        ExitData E;
        E.h = h;
        E.d[0] = do0; E.d[1] = do1; E.d[2] = do2;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            E.w[j] = D.va[j] - D.vi[j];
            E.da1[j] = D.a1a[j] - D.a1i[j];
            E.da3[j] = D.a3a[j] - D.a3i[j];
            E.da4[j] = D.a4a[j] - D.a4i[j];
            E.da5[j] = D.a5a[j] - D.a5i[j];
            E.da6[j] = D.a6a[j] - D.a6i[j];
        }
        const double s = locate_exit(E, P.r0sq, r2old - P.r0sq, r2new - P.r0sq);
        const double s2 = s * s;
        const double px1 = s2 * fma(s, fma(s, DP_PX14, DP_PX13), DP_PX12);
        const double px3 = s2 * fma(s, fma(s, DP_PX34, DP_PX33), DP_PX32);
        const double px4 = s2 * fma(s, fma(s, DP_PX44, DP_PX43), DP_PX42);
        const double px5 = s2 * fma(s, fma(s, DP_PX54, DP_PX53), DP_PX52);
        const double px6 = s2 * fma(s, fma(s, DP_PX64, DP_PX63), DP_PX62);
        const double b1 = s * fma(s, fma(s, fma(s, DP_BI14, DP_BI13), DP_BI12), DP_BI11);
        const double b3 = s2 * fma(s, fma(s, DP_BI34, DP_BI33), DP_BI32);
        const double b4 = s2 * fma(s, fma(s, DP_BI44, DP_BI43), DP_BI42);
        const double b5 = s2 * fma(s, fma(s, DP_BI54, DP_BI53), DP_BI52);
        const double b6 = s2 * fma(s, fma(s, DP_BI64, DP_BI63), DP_BI62);
        const double b7 = s2 * fma(s, fma(s, DP_BI74, DP_BI73), DP_BI72);
        const double sh = s * h;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double qi = fma(px6, D.a6i[j], fma(px5, D.a5i[j], fma(px4, D.a4i[j], fma(px3, D.a3i[j], px1 * D.a1i[j]))));
            double qa = fma(px6, D.a6a[j], fma(px5, D.a5a[j], fma(px4, D.a4a[j], fma(px3, D.a3a[j], px1 * D.a1a[j]))));
            fin.xi[j] = fma(h2, qi, fma(sh, D.vi[j], D.xi[j]));
            fin.xa[j] = fma(h2, qa, fma(sh, D.va[j], D.xa[j]));
            double ui = fma(b7, D.a7i[j], fma(b6, D.a6i[j], fma(b5, D.a5i[j], fma(b4, D.a4i[j], fma(b3, D.a3i[j], b1 * D.a1i[j])))));
            double ua = fma(b7, D.a7a[j], fma(b6, D.a6a[j], fma(b5, D.a5a[j], fma(b4, D.a4a[j], fma(b3, D.a3a[j], b1 * D.a1a[j])))));
            fin.vi[j] = fma(h, ui, D.vi[j]);
            fin.va[j] = fma(h, ua, D.va[j]);
        }
        fin.t = t + s * h;
        fin.s_exit = s;
        fin.status = ST_EXIT;
    } else {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            fin.xi[j] = D.xni[j]; fin.vi[j] = D.vni[j]; fin.xa[j] = D.xna[j]; fin.va[j] = D.vna[j];
        }
        fin.t = t + h;
        fin.s_exit = -1.0;
        fin.status = ST_EXIT_OUTSIDE;
    }
}

// ---------------------------------------------------------------------------------------------
// Lane mode: one attempted step. Returns FINISHED when the trajectory is over (fin filled).

__device__ __forceinline__ int lane_attempt(const SysDev& P, Lane& L, Final& fin)
{
    uint32_t st = attempt_begin(P, L.s);
    if (st != 0xffffffffu) {
        fin.status = st;
        goto stop_here;
    }
    {
        const double h = L.s.h, t = L.s.t;
        Coef K;
        coef_all(h, K);
        double a2i[3], a2a[3], a3i[3], a3a[3], a4i[3], a4a[3], a5i[3], a5a[3], a6i[3], a6a[3], a7i[3], a7a[3];
        double pi_[3], pa_[3], dd[3];
        double r2;
        {
            const double cs = cos(fma(P.Omega, t + K.c2, L.s.phi0));
#pragma unroll
            for (int j = 0; j < 3; ++j) { pi_[j] = pos2(K, L.xi[j], L.vi[j]); pa_[j] = pos2(K, L.xa[j], L.va[j]); }
            accel(P, pi_, pa_, cs, a2i, a2a, r2, dd);
        }
        {
            const double cs = cos(fma(P.Omega, t + K.c3, L.s.phi0));
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                pi_[j] = pos3(K, L.xi[j], L.vi[j], L.a1i[j]);
                pa_[j] = pos3(K, L.xa[j], L.va[j], L.a1a[j]);
            }
            accel(P, pi_, pa_, cs, a3i, a3a, r2, dd);
        }
        {
            const double cs = cos(fma(P.Omega, t + K.c4, L.s.phi0));
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                pi_[j] = pos4(K, L.xi[j], L.vi[j], L.a1i[j], a2i[j]);
                pa_[j] = pos4(K, L.xa[j], L.va[j], L.a1a[j], a2a[j]);
            }
            accel(P, pi_, pa_, cs, a4i, a4a, r2, dd);
        }
        {
            const double cs = cos(fma(P.Omega, t + K.c5, L.s.phi0));
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                pi_[j] = pos5(K, L.xi[j], L.vi[j], L.a1i[j], a2i[j], a3i[j]);
                pa_[j] = pos5(K, L.xa[j], L.va[j], L.a1a[j], a2a[j], a3a[j]);
            }
            accel(P, pi_, pa_, cs, a5i, a5a, r2, dd);
        }
        const double cs_end = cos(fma(P.Omega, t + h, L.s.phi0));  // stages 6 and 7 share t + h
        {
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                pi_[j] = pos6(K, h, L.xi[j], L.vi[j], L.a1i[j], a2i[j], a3i[j], a4i[j]);
                pa_[j] = pos6(K, h, L.xa[j], L.va[j], L.a1a[j], a2a[j], a3a[j], a4a[j]);
            }
            accel(P, pi_, pa_, cs_end, a6i, a6a, r2, dd);
        }
        double xni[3], xna[3], vni[3], vna[3];
        double r2new;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            xni[j] = pos7(K, h, L.xi[j], L.vi[j], L.a1i[j], a3i[j], a4i[j], a5i[j]);
            xna[j] = pos7(K, h, L.xa[j], L.va[j], L.a1a[j], a3a[j], a4a[j], a5a[j]);
        }
        accel(P, xni, xna, cs_end, a7i, a7a, r2new, dd);  // dd = x_a,new - x_i,new
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            vni[j] = vel_new(K, L.vi[j], L.a1i[j], a3i[j], a4i[j], a5i[j], a6i[j]);
            vna[j] = vel_new(K, L.va[j], L.a1a[j], a3a[j], a4a[j], a5a[j], a6a[j]);
        }
        // embedded error estimate and ode45's error test
        bool accept = true, finite = true;
        ErrMax em;
        em.key = 0ull;
        em.ae = 0.0;
        em.sc = 1.0;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            bool ok, fi;
            float r;
            double ae, sc;
            err_check(P.rtol, P.atol_pos, L.xi[j], xni[j], err_x(K, L.a1i[j], a3i[j], a4i[j], a5i[j], a6i[j]), ok, fi, r, ae, sc);
            accept = accept && ok; finite = finite && fi; err_take(em, r, 2 * j, ae, sc);
            err_check(P.rtol, P.atol_vel, L.vi[j], vni[j], err_v(K, L.a1i[j], a3i[j], a4i[j], a5i[j], a6i[j], a7i[j]), ok, fi, r, ae, sc);
            accept = accept && ok; finite = finite && fi; err_take(em, r, 2 * j + 1, ae, sc);
            err_check(P.rtol, P.atol_pos, L.xa[j], xna[j], err_x(K, L.a1a[j], a3a[j], a4a[j], a5a[j], a6a[j]), ok, fi, r, ae, sc);
            accept = accept && ok; finite = finite && fi; err_take(em, r, 2 * (3 + j), ae, sc);
            err_check(P.rtol, P.atol_vel, L.va[j], vna[j], err_v(K, L.a1a[j], a3a[j], a4a[j], a5a[j], a6a[j], a7a[j]), ok, fi, r, ae, sc);
            accept = accept && ok; finite = finite && fi; err_take(em, r, 2 * (3 + j) + 1, ae, sc);
        }
        if (!finite) {
            fin.status = ST_NONFINITE;
            goto stop_here;
        }
        const ErrMeas emeas{__uint_as_float((unsigned)(em.key >> 32)), em.ae, em.sc};
        if (!accept) {
            st = on_reject(P, L.s, emeas);
            if (st != 0xffffffffu) {
                fin.status = st;
                goto stop_here;
            }
            return RUNNING;
        }
        double w0 = vna[0] - vni[0], w1 = vna[1] - vni[1], w2 = vna[2] - vni[2];
        double rd = fma(dd[0], w0, fma(dd[1], w1, dd[2] * w2));
        if (on_accept(P, L.s, rd, r2new)) {
            StepData D;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                D.xi[j] = L.xi[j]; D.vi[j] = L.vi[j]; D.xa[j] = L.xa[j]; D.va[j] = L.va[j];
                D.a1i[j] = L.a1i[j]; D.a1a[j] = L.a1a[j]; D.a3i[j] = a3i[j]; D.a3a[j] = a3a[j];
                D.a4i[j] = a4i[j]; D.a4a[j] = a4a[j]; D.a5i[j] = a5i[j]; D.a5a[j] = a5a[j];
                D.a6i[j] = a6i[j]; D.a6a[j] = a6a[j]; D.a7i[j] = a7i[j]; D.a7a[j] = a7a[j];
                D.xni[j] = xni[j]; D.xna[j] = xna[j]; D.vni[j] = vni[j]; D.vna[j] = vna[j];
            }
            D.h = h;
            D.t = t;
            finish_exit(P, D, r2new, fin);
            return FINISHED;
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            L.xi[j] = xni[j]; L.xa[j] = xna[j]; L.vi[j] = vni[j]; L.va[j] = vna[j];
            L.a1i[j] = a7i[j]; L.a1a[j] = a7a[j];
        }
        on_commit(P, L.s, emeas);
        return RUNNING;
    }
stop_here:
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        fin.xi[j] = L.xi[j]; fin.vi[j] = L.vi[j]; fin.xa[j] = L.xa[j]; fin.va[j] = L.va[j];
    }
    fin.t = L.s.t;
    return FINISHED;
}

// Observables of the Fig. 1 caption from the final state; stores one trajectory.
// Scalars of a finished trajectory needed by the epilogue (passed by value: a reference to the live
// state would force it into local memory for the whole integration).
struct Tally {
    double phi0, t_first, t_last;
    int n_acc, n_rej, n_bounce;
};
__device__ __forceinline__ Tally tally(const Scal& S)
{
    Tally T;
    T.phi0 = S.phi0;
    T.t_first = S.t_first;
    T.t_last = S.t_last;
    T.n_acc = S.n_acc;
    T.n_rej = S.n_rej;
    T.n_bounce = S.n_bounce;
    return T;
}

__device__ __noinline__ void store_result(const SysDev& P, const IcPtrs& ic, const ObsPtrs& out, long long i,
                                          const Tally S, const Final fin, bool started)
{
    uint32_t st = fin.status;
    double theta = 0.0, dp = 0.0, dE = 0.0;
    if (started) {
        const double* y = ic.y0 + i;
        const long long ld = ic.ld;
        double v0[3], xi0[3], vi0[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            xi0[j] = __ldg(y + (0 + j) * ld);
            vi0[j] = __ldg(y + (3 + j) * ld);
            v0[j] = __ldg(y + (9 + j) * ld);
        }
        const double* vf = fin.va;
        double c0 = v0[1] * vf[2] - v0[2] * vf[1];
        double c1 = v0[2] * vf[0] - v0[0] * vf[2];
        double c2 = v0[0] * vf[1] - v0[1] * vf[0];
        double cr = sqrt(fma(c0, c0, fma(c1, c1, c2 * c2)));
        double dt = fma(v0[0], vf[0], fma(v0[1], vf[1], v0[2] * vf[2]));
        theta = atan2(cr, dt);
        double u0 = vf[0] - v0[0], u1 = vf[1] - v0[1], u2 = vf[2] - v0[2];
        dp = P.m_a * sqrt(fma(u0, u0, fma(u1, u1, u2 * u2)));
        dE = ion_energy(P, cos(fma(P.Omega, fin.t, S.phi0)), fin.xi, fin.vi) - ion_energy(P, cos(S.phi0), xi0, vi0);
        if (S.n_bounce >= 2) st |= ST_COMPLEX;
    }
    out.theta_s[i] = theta;
    out.dp[i] = dp;
    out.dE_ion[i] = dE;
    out.t_final[i] = started ? fin.t : 0.0;
    out.t_first[i] = started ? S.t_first : 0.0;
    out.t_last[i] = started ? S.t_last : 0.0;
    out.n_bounce[i] = started ? S.n_bounce : 0;
    out.status[i] = st;
    out.n_steps[i] = started ? S.n_acc : 0;
    out.n_rej[i] = started ? S.n_rej : 0;
    if (out.y_final) {
        double* yf = out.y_final + i;
        const long long ld = out.ld_out;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            yf[(0 + j) * ld] = fin.xi[j];
            yf[(3 + j) * ld] = fin.vi[j];
            yf[(6 + j) * ld] = fin.xa[j];
            yf[(9 + j) * ld] = fin.va[j];
        }
    }
}

// Write a lane's trajectory into a suspend record.
__device__ __forceinline__ void lane_suspend(const Lane& L, long long idx, int sid, Susp* rec)
{
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        rec->x[j] = L.xi[j]; rec->x[3 + j] = L.xa[j];
        rec->v[j] = L.vi[j]; rec->v[3 + j] = L.va[j];
        rec->a1[j] = L.a1i[j]; rec->a1[3 + j] = L.a1a[j];
    }
    rec->t = L.s.t;
    rec->h = L.s.h;
    rec->phi0 = L.s.phi0;
    rec->rdot_prev = L.s.rdot_prev;
    rec->t_first = L.s.t_first;
    rec->t_last = L.s.t_last;
    rec->idx = idx;
    rec->sid = sid;
    rec->n_acc = L.s.n_acc;
    rec->n_rej = L.s.n_rej;
    rec->n_bounce = L.s.n_bounce;
    rec->flags = (L.s.nofailed ? 1 : 0) | (L.s.retry ? 2 : 0);
}

// Load a saved trajectory back into a lane (the inverse of lane_suspend): the lane continues with the
// same state and controller scalars, so it produces the bits it would have produced without the stop.
// The record was written by an earlier kernel launch, so plain loads see it.
__device__ __forceinline__ void lane_resume(const Susp* __restrict__ rec, Lane& L, long long& idx, int& sid)
{
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        L.xi[j] = rec->x[j]; L.xa[j] = rec->x[3 + j];
        L.vi[j] = rec->v[j]; L.va[j] = rec->v[3 + j];
        L.a1i[j] = rec->a1[j]; L.a1a[j] = rec->a1[3 + j];
    }
    L.s.t = rec->t;
    L.s.h = rec->h;
    L.s.hmin = hmin_at(L.s.t);  // the value attempt_begin set for the step in progress
    L.s.phi0 = rec->phi0;
    L.s.rdot_prev = rec->rdot_prev;
    L.s.t_first = rec->t_first;
    L.s.t_last = rec->t_last;
    L.s.n_acc = rec->n_acc;
    L.s.n_rej = rec->n_rej;
    L.s.n_bounce = rec->n_bounce;
    const int flags = rec->flags;
    L.s.nofailed = (flags & 1) != 0;
    L.s.retry = (flags & 2) != 0;
    idx = rec->idx;
    sid = rec->sid;
}

// ---------------------------------------------------------------------------------------------
// Group mode: lanes base .. base + G - 1 of a warp hold one trajectory; lane comp c < 6 holds
// component c of [x_ion, x_atom] (lanes with c >= 6 compute on a copy of component 5 and are never
// read). Scalars are replicated across the group.

template <int G>
struct GroupLane {
    int base;   // first lane of the group
    int c;      // 0 .. 7 (>= 6: spare)
    int comp;   // min(c, 5)
};

template <int G>
__device__ __forceinline__ GroupLane<G> group_lane()
{
    constexpr int NG = 32 / G;
    const int lane = threadIdx.x & 31;
    int grp = lane / G;
    if (grp > NG - 1) grp = NG - 1;
    GroupLane<G> gl;
    gl.base = grp * G;
    gl.c = lane - gl.base;
    gl.comp = gl.c < 6 ? gl.c : 5;
    return gl;
}

__device__ __forceinline__ double shfl(double v, int src) { return __shfl_sync(FULL, v, src); }

// Group-mode accelerations: this lane's component of the acceleration at stage positions p (each
// lane holds its component), cs = cos(Omega t_s + phi0). Same expressions as accel().
// kq3, ka3: the ion trap coefficients of axis comp - 3 on lanes 3-5 (unused elsewhere).
template <int G>
__device__ __forceinline__ double accel_group(const SysDev& P, const GroupLane<G>& gl, double p, double cs,
                                              double kq3, double ka3, double& r2out, double d3[3])
{
    const int j = gl.comp < 3 ? gl.comp : gl.comp - 3;
    const double pi = shfl(p, gl.base + j);
    const double pa = shfl(p, gl.base + 3 + j);
    const double dj = pa - pi;
    const double d0 = shfl(dj, gl.base + 0), d1 = shfl(dj, gl.base + 1), d2 = shfl(dj, gl.base + 2);
    const double r2 = fma(d0, d0, fma(d1, d1, d2 * d2));
    const double s = rcp_nr(r2);
    const double s2 = s * s;
    // one FMA instruction: lane 0 forms s2 s, lane 1 the ion's ci8 s2 - ci4, lane 2 the atom's
    // ca8 s2 - ca4, lanes 3-5 the ion trap coefficients ka_j + kq_j cs (j = lane - 3)
    const int c = gl.c;
    const double ua = c == 0 ? s2 : (c == 1 ? P.ci8 : (c == 2 ? P.ca8 : kq3));
    const double ub = c == 0 ? s : (c < 3 ? s2 : cs);
    const double uc = c == 0 ? 0.0 : (c == 1 ? -P.ci4 : (c == 2 ? -P.ca4 : ka3));
    const double u = fma(ua, ub, uc);
    const double gm = shfl(u, gl.base + 0) * shfl(u, gl.base + (gl.comp < 3 ? 1 : 2));
    const double kcs = shfl(u, gl.base + 3 + (gl.comp < 3 ? gl.comp : 0));
    const double kc = gl.comp < 3 ? kcs : 0.0;
    const double q = gm * dj;
    r2out = r2;
    d3[0] = d0;
    d3[1] = d1;
    d3[2] = d2;
    return fma(kc, p, q);
}

// Error measure of a trajectory held by lanes base .. base + 5 (lane base + c holds component c of
// [x_ion, x_atom], whose position and velocity are components k = 2c and 2c + 1 of the measure): the
// largest FP32 ratio of the group, ties to the lowest k (as in lane mode), with that component's |e|
// and sc, identical on every lane. real = false on lanes outside the six.
__device__ __forceinline__ ErrMeas group_err(int base, int c, bool real, float rx, double aex, double scx, float rv,
                                             double aev, double scv)
{
    const unsigned long long kx = real ? err_key(rx, 2 * c) : 0ull;
    const unsigned long long kv = real ? err_key(rv, 2 * c + 1) : 0ull;
    const bool vb = kv > kx;
    const unsigned long long key = vb ? kv : kx;
    const double ae = vb ? aev : aex, sc = vb ? scv : scx;
    unsigned long long best = 0ull;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        const unsigned long long o = __shfl_sync(FULL, key, base + j);
        best = o > best ? o : best;
    }
    const int src = base + ((15 - (int)(best & 15ull)) >> 1);
    ErrMeas e;
    e.f = __uint_as_float((unsigned)(best >> 32));
    e.ae = shfl(ae, src);
    e.sc = shfl(sc, src);
    return e;
}

// Result of a trajectory whose sys_id is outside the table: its initial state, BAD_IC.
__device__ __forceinline__ void store_bad_sid(const IcPtrs& ic, const ObsPtrs& out, const SysDev* tab, long long i)
{
    Final fin;
    Tally S;
    S.phi0 = 0.0;
    S.t_first = S.t_last = 0.0;
    S.n_acc = S.n_rej = S.n_bounce = 0;
    const double* y = ic.y0 + i;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        fin.xi[j] = y[(0 + j) * ic.ld]; fin.vi[j] = y[(3 + j) * ic.ld];
        fin.xa[j] = y[(6 + j) * ic.ld]; fin.va[j] = y[(9 + j) * ic.ld];
    }
    fin.t = 0.0;
    fin.status = ST_BAD_IC;
    store_result(tab[0], ic, out, i, S, fin, false);
}

}  // namespace ia
