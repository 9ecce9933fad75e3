// ia_adjoint.cuh -- reverse-mode (adjoint) differentiation of the trajectory map, with checkpointing.
//
// The map differentiated is the one the tangent kernel differentiates: the computed map from
// (initial state, trap q vector) to the observables with the primal's step sizes and accept/reject
// decisions held fixed, plus the sensitivity of the exit time located on the continuous extension.
// One reverse sweep per objective gives its gradient with respect to all twelve initial-state
// components and the three q components at once; the derivatives along any seed directions are then
// inner products.
//
// Layout: one trajectory per warp, lane = obj * 6 + comp (lanes 30, 31 spare). Every group of six
// lanes carries its own copy of the primal (identical arithmetic, so identical bits) and, for
// obj = 1..4, the adjoint of J = theta_s, |p_f - p_i| (atom), dE_ion, t_final; comp indexes
// [x_ion(3), x_atom(3)] with the matching velocity.
//
// Passes:
//   1. forward: the primal (results bit-identical to ia_launch) with a checkpoint of the complete
//      controller state every `stride` committed steps. The checkpoint array has a fixed length;
//      when it is full every other checkpoint is dropped and the stride doubles, so memory stays
//      bounded for any trajectory length and only the recomputation grows.
//   2. the terminal step: lambda_f = dJ/dy_f with the exit-time correction
//        lambda_eff = lambda_f - c grad_y (d . d),  c = (lambda_f . y_s + (dJ/dt_f) h) / (d . d_s),
//      (d: separation at s*, y_s = dy/ds and d_s = dd/ds on the continuous extension) pulled back
//      through the continuous extension's weights at s*.
//   3. reverse, in blocks of at most `seg` steps from the end: restore the checkpoint below the
//      block, replay the primal up to the block (same decisions: the controller state is restored
//      whole), record the block's step starts, and pull the adjoint back through each step.
//
// One step of the Nystrom form (accelerations depend on positions only):
//   X_l = x + c_l h v + h^2 sum_m AA_lm a_m,  a_l = F(X_l, t + c_l h),
//   x' = x + h v + h^2 sum_m bA_m a_m,  v' = v + h sum_m b_m a_m.
// Its transpose, with abar_l the adjoint of a_l and Xbar_l = J_l^T abar_l:
//   abar_m = h^2 bA_m lx + h b_m lv;  xbar = lx;  vbar = h lx + lv;
//   for l = 6..1: Xbar_l = J_l^T abar_l;  xbar += Xbar_l;  vbar += c_l h Xbar_l;
//                 abar_m += h^2 AA_lm Xbar_l (m < l).
// For F_ion = k(t) x_ion + (-1/m_i) g d, F_atom = (1/m_a) g d, d = x_atom - x_ion, g = -V'(r)/r:
//   with u = abar_ion / m_i - abar_atom / m_a and H u = g u + 2 g_u (d . u) d (g_u = dg / d(r^2)),
//   J^T abar = (k abar_ion + H u, -H u), and the q gradient gains abar_ion,j (dk_j/dq_j) X_ion,j.
// Power-of-two rescaling keeps the adjoint of a long chaotic trajectory in range (exact scaling,
// as in the tangent kernel).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ia_traj.cuh"
#include "ia_tangent.cuh"

namespace ia {

constexpr int CK_DOUBLES = 32;  // checkpoint record (256 B)
constexpr int SR_DOUBLES = 16;  // step record (128 B)
constexpr int ADJ_WARPS = 4;    // warps per 128-thread block
constexpr int AUX_FIELDS = 6;   // per stage: X, d0, d1, d2, g, g_u
constexpr int AUX_STAGE = AUX_FIELDS * 32;

enum : int { PA_REJ = 0, PA_COMMIT = 1, PA_EXIT = 2, PA_STOP = 3 };

struct AdjIn {
    const double* dy0;  // [ndir][12][ld] seeds, or null when ndir = 0
    double dq[4][3];
    int ndir;
    long long ld;
};

struct AdjOut {
    double* grad_y0;  // [4][12][ld] or null
    double* grad_q;   // [4][3][ld] or null
    double* d_theta;  // [ndir][ld] (used when ndir > 0)
    double* d_dp;
    double* d_dE;
    double* d_tf;
    long long ld;
};

struct AdjBuf {
    double* ckpt;   // [warps][max_ckpt][CK_DOUBLES]
    double* steps;  // [warps][seg][SR_DOUBLES]
    unsigned long long* work;
    unsigned long long* errors;  // trajectories whose replay did not reproduce the forward pass
    long long warps;
    int max_ckpt;  // even
    int seg;
};

// What one attempted step leaves behind for the exit epilogue.
struct PrimStep {
    double h, t, a3, a4, a5, a6, a7, xn, vn, r2new, cs67;
};

// Coefficients and cosines of a step (lane-distributed products, then broadcast; the values are
// those of the tangent kernel bit for bit).
__device__ __forceinline__ void step_coefs(const SysDev& P, int lane, double h, double t, double phi0, Coef& K,
                                           double& cs2, double& cs3, double& cs4, double& cs5, double& cs67)
{
    K.h2 = h * h;
    const int k0 = lane < N_COEF ? lane : N_COEF - 1;
    const double cv0 = COEF_K[k0] * (COEF_H2[k0] ? K.h2 : h);
    const int k1 = lane + 32 < N_COEF ? lane + 32 : N_COEF - 1;
    const double cv1 = COEF_K[k1] * (COEF_H2[k1] ? K.h2 : h);
    double* kp = &K.c2;
#pragma unroll
    for (int k = 0; k < N_COEF; ++k) kp[k] = k < 32 ? shfl(cv0, k) : shfl(cv1, k - 32);
    const double chsel = lane < 4 ? cv0 : h;
    const double cl = cos(fma(P.Omega, t + chsel, phi0));
    cs2 = shfl(cl, 0);
    cs3 = shfl(cl, 1);
    cs4 = shfl(cl, 2);
    cs5 = shfl(cl, 3);
    cs67 = shfl(cl, 4);
}

// Acceleration component of this lane at positions X of its group (the primal arithmetic of the
// other layouts). When aux is not null, stores the stage quantities the reverse sweep needs.
__device__ __forceinline__ double adj_accel(const SysDev& P, const TLane& tl, double X, double cs, double kq, double ka,
                                            double coef, double* aux, double& r2, double d[3])
{
    const int j = tl.comp < 3 ? tl.comp : tl.comp - 3;
    const double dd = shfl(X, tl.base + 3 + j) - shfl(X, tl.base + j);
    const double d0 = shfl(dd, tl.base + 0), d1 = shfl(dd, tl.base + 1), d2 = shfl(dd, tl.base + 2);
    r2 = fma(d0, d0, fma(d1, d1, d2 * d2));
    const double s = rcp_nr(r2);
    const double s2 = s * s;
    const double s3 = fma(s2, s, 0.0);
    const bool ion = tl.comp < 3;
    const double gm = s3 * fma(ion ? P.ci8 : P.ca8, s2, -(ion ? P.ci4 : P.ca4));
    d[0] = d0;
    d[1] = d1;
    d[2] = d2;
    if (aux) {
        aux[0] = X;
        aux[32] = d0;
        aux[64] = d1;
        aux[96] = d2;
        aux[128] = s3 * fma(P.c8x8, s2, -P.c4x4);  // g = -V'(r)/r
        aux[160] = (s2 * s2) * fma(-5.0 * P.c8x8, s2, 3.0 * P.c4x4);
    }
    return fma(fma(kq, cs, ka), X, gm * dd);
}

// Xbar = J^T abar for this lane's component at the stage stored in aux; adds the stage's part of
// the q gradient (ion lanes).
__device__ __forceinline__ double adj_apply(const SysDev& P, const TLane& tl, const double* aux, double ab, double cs,
                                            double kq, double ka, double& gq)
{
    const int j = tl.comp < 3 ? tl.comp : tl.comp - 3;
    const double X = aux[0], d0 = aux[32], d1 = aux[64], d2 = aux[96], g = aux[128], gu = aux[160];
    const double ui = shfl(ab, tl.base + j), ua = shfl(ab, tl.base + 3 + j);
    const double uj = ui * P.inv_mi - ua * P.inv_ma;
    const double u0 = shfl(uj, tl.base + 0), u1 = shfl(uj, tl.base + 1), u2 = shfl(uj, tl.base + 2);
    const double du = fma(d0, u0, fma(d1, u1, d2 * u2));
    const double dj = j == 0 ? d0 : (j == 1 ? d1 : d2);
    const double Hu = fma((2.0 * gu) * du, dj, g * uj);
    if (tl.comp < 3) {
        gq = fma((ab * P.kq_per_q) * cs, X, gq);
        return fma(fma(kq, cs, ka), ab, Hu);
    }
    return -Hu;
}

// One attempted step of the primal: the control flow of the tangent kernel (decisions from group 0,
// which every group reproduces). On a commit x, v, a1, c1 advance.
__device__ __forceinline__ int prim_attempt(const SysDev& P, const TLane& tl, int lane, Scal& S, double& x, double& v,
                                            double& a1, double& c1, double kq, double ka, double coef, PrimStep& E,
                                            uint32_t& st)
{
    st = attempt_begin(P, S);
    if (st != 0xffffffffu) return PA_STOP;
    const double h = S.h, t = S.t;
    E.h = h;
    E.t = t;
    Coef K;
    double cs2, cs3, cs4, cs5, cs67;
    step_coefs(P, lane, h, t, S.phi0, K, cs2, cs3, cs4, cs5, cs67);
    double r2, d3[3];
    const double a2 = adj_accel(P, tl, pos2(K, x, v), cs2, kq, ka, coef, nullptr, r2, d3);
    const double a3 = adj_accel(P, tl, pos3(K, x, v, a1), cs3, kq, ka, coef, nullptr, r2, d3);
    const double a4 = adj_accel(P, tl, pos4(K, x, v, a1, a2), cs4, kq, ka, coef, nullptr, r2, d3);
    const double a5 = adj_accel(P, tl, pos5(K, x, v, a1, a2, a3), cs5, kq, ka, coef, nullptr, r2, d3);
    const double a6 = adj_accel(P, tl, pos6(K, h, x, v, a1, a2, a3, a4), cs67, kq, ka, coef, nullptr, r2, d3);
    const double xn = pos7(K, h, x, v, a1, a3, a4, a5);
    double r2new, dn[3];
    const double a7 = adj_accel(P, tl, xn, cs67, kq, ka, coef, nullptr, r2new, dn);
    const double vn = vel_new(K, v, a1, a3, a4, a5, a6);
    bool okx, fx, okv, fv;
    float rx, rv;
    double aex, scx, aev, scv;
    err_check(P.rtol, P.atol_pos, x, xn, err_x(K, a1, a3, a4, a5, a6), okx, fx, rx, aex, scx);
    err_check(P.rtol, P.atol_vel, v, vn, err_v(K, a1, a3, a4, a5, a6, a7), okv, fv, rv, aev, scv);
    const bool prim = tl.dir == 0;
    const bool accept = (__ballot_sync(FULL, prim && !(okx && okv)) & 0x3fu) == 0;
    const bool finite = (__ballot_sync(FULL, prim && !(fx && fv)) & 0x3fu) == 0;
    const ErrMeas em = group_err(0, tl.comp, prim, rx, aex, scx, rv, aev, scv);
    const int jj = tl.comp < 3 ? tl.comp : tl.comp - 3;
    const double wj = shfl(vn, 3 + jj) - shfl(vn, jj);
    const double w0 = shfl(wj, 0), w1 = shfl(wj, 1), w2 = shfl(wj, 2);
    const double e0 = shfl(dn[0], 0), e1 = shfl(dn[1], 0), e2 = shfl(dn[2], 0);
    const double rd = fma(e0, w0, fma(e1, w1, e2 * w2));
    const double r2n0 = shfl(r2new, 0);
    if (!finite) {
        st = ST_NONFINITE;
        return PA_STOP;
    }
    if (!accept) {
        st = on_reject(P, S, em);
        return st != 0xffffffffu ? PA_STOP : PA_REJ;
    }
    if (on_accept(P, S, rd, r2n0)) {
        E.a3 = a3; E.a4 = a4; E.a5 = a5; E.a6 = a6; E.a7 = a7;
        E.xn = xn; E.vn = vn; E.r2new = r2n0; E.cs67 = cs67;
        return PA_EXIT;
    }
    x = xn;
    v = vn;
    a1 = a7;
    c1 = cs67;
    on_commit(P, S, em);
    return PA_COMMIT;
}

// Pull (lx, lv) -- the adjoint of this lane's component at the end of a step, or at fraction s of
// the step on its continuous extension when ext -- back to the step start; adds the step's part of
// the q gradient to gq. (x, v): primal state at the step start; c1: the cosine of a1's evaluation.
__device__ __noinline__ void adj_step(const SysDev& P, const TLane& tl, int lane, double x, double v, double t,
                                      double h, double c1, double phi0, bool ext, double s, double kq, double ka,
                                      double coef, double& lx, double& lv, double& gq, double* sw)
{
    Coef K;
    double cs2, cs3, cs4, cs5, cs67;
    step_coefs(P, lane, h, t, phi0, K, cs2, cs3, cs4, cs5, cs67);
    double r2, d3[3];
    const double a1 = adj_accel(P, tl, x, c1, kq, ka, coef, sw + 0 * AUX_STAGE, r2, d3);
    const double a2 = adj_accel(P, tl, pos2(K, x, v), cs2, kq, ka, coef, sw + 1 * AUX_STAGE, r2, d3);
    const double a3 = adj_accel(P, tl, pos3(K, x, v, a1), cs3, kq, ka, coef, sw + 2 * AUX_STAGE, r2, d3);
    const double a4 = adj_accel(P, tl, pos4(K, x, v, a1, a2), cs4, kq, ka, coef, sw + 3 * AUX_STAGE, r2, d3);
    const double a5 = adj_accel(P, tl, pos5(K, x, v, a1, a2, a3), cs5, kq, ka, coef, sw + 4 * AUX_STAGE, r2, d3);
    adj_accel(P, tl, pos6(K, h, x, v, a1, a2, a3, a4), cs67, kq, ka, coef, sw + 5 * AUX_STAGE, r2, d3);
    if (ext) adj_accel(P, tl, pos7(K, h, x, v, a1, a3, a4, a5), cs67, kq, ka, coef, sw + 6 * AUX_STAGE, r2, d3);
    double ab1, ab2 = 0.0, ab3, ab4, ab5, ab6, xb, vb;
    if (!ext) {
        ab1 = fma(K.w71, lx, K.b1 * lv);
        ab3 = fma(K.w73, lx, K.b3 * lv);
        ab4 = fma(K.w74, lx, K.b4 * lv);
        ab5 = fma(K.w75, lx, K.b5 * lv);
        ab6 = K.b6 * lv;
        xb = lx;
        vb = fma(h, lx, lv);
    } else {
        // weights of the continuous extension at s: x(s) = x + s h v + h^2 sum P_m(s) a_m,
        // v(s) = v + h sum B_m(s) a_m
        const double s2 = s * s, h2 = K.h2;
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
        const double hx = h2 * lx, hv = h * lv;
        ab1 = fma(px1, hx, b1 * hv);
        ab3 = fma(px3, hx, b3 * hv);
        ab4 = fma(px4, hx, b4 * hv);
        ab5 = fma(px5, hx, b5 * hv);
        ab6 = fma(px6, hx, b6 * hv);
        const double ab7 = b7 * hv;
        xb = lx;
        vb = fma(s * h, lx, lv);
        // a7 = F(x'), x' = x + h v + sum w7m a_m
        const double X7 = adj_apply(P, tl, sw + 6 * AUX_STAGE, ab7, cs67, kq, ka, gq);
        xb += X7;
        vb = fma(h, X7, vb);
        ab1 = fma(K.w71, X7, ab1);
        ab3 = fma(K.w73, X7, ab3);
        ab4 = fma(K.w74, X7, ab4);
        ab5 = fma(K.w75, X7, ab5);
    }
    const double X6 = adj_apply(P, tl, sw + 5 * AUX_STAGE, ab6, cs67, kq, ka, gq);
    xb += X6;
    vb = fma(h, X6, vb);
    ab1 = fma(K.w61, X6, ab1);
    ab2 = fma(K.w62, X6, ab2);
    ab3 = fma(K.w63, X6, ab3);
    ab4 = fma(K.w64, X6, ab4);
    const double X5 = adj_apply(P, tl, sw + 4 * AUX_STAGE, ab5, cs5, kq, ka, gq);
    xb += X5;
    vb = fma(K.c5, X5, vb);
    ab1 = fma(K.w51, X5, ab1);
    ab2 = fma(K.w52, X5, ab2);
    ab3 = fma(K.w53, X5, ab3);
    const double X4 = adj_apply(P, tl, sw + 3 * AUX_STAGE, ab4, cs4, kq, ka, gq);
    xb += X4;
    vb = fma(K.c4, X4, vb);
    ab1 = fma(K.w41, X4, ab1);
    ab2 = fma(K.w42, X4, ab2);
    const double X3 = adj_apply(P, tl, sw + 2 * AUX_STAGE, ab3, cs3, kq, ka, gq);
    xb += X3;
    vb = fma(K.c3, X3, vb);
    ab1 = fma(K.w31, X3, ab1);
    const double X2 = adj_apply(P, tl, sw + 1 * AUX_STAGE, ab2, cs2, kq, ka, gq);
    xb += X2;
    vb = fma(K.c2, X2, vb);
    const double X1 = adj_apply(P, tl, sw + 0 * AUX_STAGE, ab1, c1, kq, ka, gq);
    lx = xb + X1;
    lv = vb;
}

// Explicit partial derivatives of objective obj (1 theta_s, 2 |p_f - p_i|, 3 dE_ion, 4 t_final) with
// respect to the initial state (gy0), the final state (gyf), the final time (jt) and q (gq), holding
// the others fixed. obj 0 gives zeros.
__device__ __noinline__ void objective_partials(const SysDev& P, int obj, double phi0, const double* y0,
                                                const double* yf, double tf, double* gy0, double* gyf, double& jt,
                                                double* gq)
{
    for (int c = 0; c < 12; ++c) {
        gy0[c] = 0.0;
        gyf[c] = 0.0;
    }
    gq[0] = gq[1] = gq[2] = 0.0;
    jt = 0.0;
    const double* v0 = y0 + 9;
    const double* vf = yf + 9;
    if (obj == 1) {
        // theta = atan2(C, D), C = |v0 x vf|, D = v0 . vf
        const double c[3] = {v0[1] * vf[2] - v0[2] * vf[1], v0[2] * vf[0] - v0[0] * vf[2],
                             v0[0] * vf[1] - v0[1] * vf[0]};
        const double C = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        const double D = v0[0] * vf[0] + v0[1] * vf[1] + v0[2] * vf[2];
        const double den = C * C + D * D;
        // dC/dvf = (v0 x vf)^ x ... : dC = c_hat . (dv0 x vf + v0 x dvf), so
        // dC/dvf = c_hat x v0, dC/dv0 = vf x c_hat (zero when C = 0, as in the tangent)
        double dCf[3] = {0.0, 0.0, 0.0}, dC0[3] = {0.0, 0.0, 0.0};
        if (C > 0.0) {
            const double ch[3] = {c[0] / C, c[1] / C, c[2] / C};
            dCf[0] = ch[1] * v0[2] - ch[2] * v0[1];
            dCf[1] = ch[2] * v0[0] - ch[0] * v0[2];
            dCf[2] = ch[0] * v0[1] - ch[1] * v0[0];
            dC0[0] = vf[1] * ch[2] - vf[2] * ch[1];
            dC0[1] = vf[2] * ch[0] - vf[0] * ch[2];
            dC0[2] = vf[0] * ch[1] - vf[1] * ch[0];
        }
        for (int k = 0; k < 3; ++k) {
            gyf[9 + k] = (D * dCf[k] - C * v0[k]) / den;
            gy0[9 + k] = (D * dC0[k] - C * vf[k]) / den;
        }
    } else if (obj == 2) {
        const double u[3] = {vf[0] - v0[0], vf[1] - v0[1], vf[2] - v0[2]};
        const double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        if (un > 0.0)
            for (int k = 0; k < 3; ++k) {
                gyf[9 + k] = P.m_a * u[k] / un;
                gy0[9 + k] = -P.m_a * u[k] / un;
            }
    } else if (obj == 3) {
        // E_ion = m_i |v_i|^2 / 2 + sum_j (ua_j + uq_j cos(Omega t + phi0)) x_j^2
        const double cf = cos(P.Omega * tf + phi0), sf = sin(P.Omega * tf + phi0), c0 = cos(phi0);
        for (int j = 0; j < 3; ++j) {
            gyf[3 + j] = P.m_i * yf[3 + j];
            gy0[3 + j] = -P.m_i * y0[3 + j];
            gyf[j] = 2.0 * (P.ua[j] + P.uq[j] * cf) * yf[j];
            gy0[j] = -2.0 * (P.ua[j] + P.uq[j] * c0) * y0[j];
            jt += -P.uq[j] * P.Omega * sf * yf[j] * yf[j];
            gq[j] = P.uq_per_q * (cf * yf[j] * yf[j] - c0 * y0[j] * y0[j]);
        }
    } else if (obj == 4) {
        jt = 1.0;
    }
}

__device__ __forceinline__ void ckpt_write(double* ck, int lane, double x, double v, double a1, double c1,
                                           const Scal& S)
{
    if (lane < 6) {
        ck[lane] = x;
        ck[6 + lane] = v;
        ck[12 + lane] = a1;
    }
    if (lane == 0) {
        ck[18] = S.t;
        ck[19] = S.h;
        ck[20] = S.rdot_prev;
        ck[21] = S.t_first;
        ck[22] = S.t_last;
        ck[23] = c1;
        ck[24] = (double)S.n_acc;
        ck[25] = (double)S.n_rej;
        ck[26] = (double)S.n_bounce;
    }
}

__device__ __forceinline__ void ckpt_read(const double* ck, int comp, double& x, double& v, double& a1, double& c1,
                                          Scal& S)
{
    x = ck[comp];
    v = ck[6 + comp];
    a1 = ck[12 + comp];
    S.t = ck[18];
    S.h = ck[19];
    S.rdot_prev = ck[20];
    S.t_first = ck[21];
    S.t_last = ck[22];
    c1 = ck[23];
    S.n_acc = (int)ck[24];
    S.n_rej = (int)ck[25];
    S.n_bounce = (int)ck[26];
    S.hmin = 0.0;
    S.nofailed = true;
    S.retry = false;
}

// Exact power-of-two rescaling of a group's adjoint (lx, lv, gq) when its largest entry leaves
// [2^-256, 2^256]; the exponent is collected in scale_e.
__device__ __forceinline__ void adj_rescale(const TLane& tl, double& lx, double& lv, double& gq, int& scale_e)
{
    int me = max_exp3(lx, lv, gq);
#pragma unroll
    for (int k = 1; k < 6; ++k) me = max(me, __shfl_sync(FULL, me, tl.base + ((tl.comp + k) % 6)));
    if (me < 2047 && (me > 1023 + 256 || (me > 0 && me < 1023 - 256))) {
        const int sh = me > 1023 + 256 ? -256 : 256;
        const double f = sh < 0 ? 0x1p-256 : 0x1p+256;
        lx *= f;
        lv *= f;
        gq *= f;
        scale_e -= sh;
    }
}

__device__ __forceinline__ void adj_zero_outputs(const AdjIn& ain, const AdjOut& aout, const TLane& tl, int lane,
                                                 long long i, double val)
{
    if (lane >= 30 || tl.dir == 0) return;
    const int obj = tl.dir - 1;
    const int yi = tl.comp < 3 ? tl.comp : tl.comp + 3;
    if (aout.grad_y0) {
        aout.grad_y0[((long long)obj * 12 + yi) * aout.ld + i] = val;
        aout.grad_y0[((long long)obj * 12 + yi + 3) * aout.ld + i] = val;
    }
    if (aout.grad_q && tl.comp < 3) aout.grad_q[((long long)obj * 3 + tl.comp) * aout.ld + i] = val;
    if (tl.comp == 0)
        for (int k = 0; k < ain.ndir; ++k) {
            double* dst = obj == 0 ? aout.d_theta : obj == 1 ? aout.d_dp : obj == 2 ? aout.d_dE : aout.d_tf;
            dst[(long long)k * aout.ld + i] = val;
        }
}

// Adjoint kernel: one trajectory per warp (see the file comment). buf.warps warps take trajectories
// from the work counter; each owns a checkpoint array and a step buffer.
__global__ void __launch_bounds__(128) k_adjoint(const SysDev* __restrict__ tab, int n_sys, IcPtrs ic, ObsPtrs out,
                                                 long long n, AdjIn ain, AdjOut aout, AdjBuf buf)
{
    __shared__ double s_aux[ADJ_WARPS][7 * AUX_STAGE];
    const TLane tl = tlane();
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const long long wg = (long long)blockIdx.x * ADJ_WARPS + wib;
    if (wg >= buf.warps) return;
    double* sw = &s_aux[wib][lane];
    double* ckw = buf.ckpt + wg * (long long)buf.max_ckpt * CK_DOUBLES;
    double* srw = buf.steps + wg * (long long)buf.seg * SR_DOUBLES;
    const int yi = tl.comp < 3 ? tl.comp : tl.comp + 3;
    const int yv = yi + 3;
    for (;;) {
        unsigned long long claim = 0;
        if (lane == 0) claim = atomicAdd(buf.work, 1ull);
        claim = __shfl_sync(FULL, claim, 0);
        if (claim >= (unsigned long long)n) break;
        const long long i = (long long)claim;
        const int sid = ic.sys_id ? __ldg(ic.sys_id + i) : 0;
        if (sid < 0 || sid >= n_sys) {
            if (lane == 0) store_bad_sid(ic, out, tab, i);
            adj_zero_outputs(ain, aout, tl, lane, i, 0.0);
            continue;
        }
        const SysDev& P = tab[sid];
        double x = __ldg(ic.y0 + yi * ic.ld + i);
        double v = __ldg(ic.y0 + yv * ic.ld + i);
        Scal S;
        S.phi0 = __ldg(ic.phi0 + i);
        const bool ok_state = __all_sync(FULL, is_finite(x) && is_finite(v)) && is_finite(S.phi0);
        double xs[6], vs[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            xs[k] = shfl(x, k);
            vs[k] = shfl(v, k);
        }
        const double dd0 = xs[3] - xs[0], dd1 = xs[4] - xs[1], dd2 = xs[5] - xs[2];
        const double r2init = fma(dd0, dd0, fma(dd1, dd1, dd2 * dd2));
        if (!ok_state || !(dbits(r2init) > 0)) {
            if (lane == 0) {
                Final fin;
                for (int k = 0; k < 3; ++k) {
                    fin.xi[k] = xs[k]; fin.xa[k] = xs[3 + k]; fin.vi[k] = vs[k]; fin.va[k] = vs[3 + k];
                }
                fin.t = 0.0;
                fin.s_exit = -1.0;
                fin.status = ST_BAD_IC;
                store_result(P, ic, out, i, tally(S), fin, false);
            }
            adj_zero_outputs(ain, aout, tl, lane, i, 0.0);
            continue;
        }
        const double kq = tl.comp < 3 ? P.kq[tl.comp] : 0.0;
        const double ka = tl.comp < 3 ? P.ka[tl.comp] : 0.0;
        const double coef = tl.comp < 3 ? P.neg_inv_mi : P.inv_ma;
        double c1 = cos(S.phi0);
        double a1;
        {
            double r2, d3[3];
            a1 = adj_accel(P, tl, x, c1, kq, ka, coef, nullptr, r2, d3);
        }
        {
            Lane L0;
            for (int k = 0; k < 3; ++k) {
                L0.xi[k] = xs[k]; L0.xa[k] = xs[3 + k]; L0.vi[k] = vs[k]; L0.va[k] = vs[3 + k];
                L0.a1i[k] = shfl(a1, k);
                L0.a1a[k] = shfl(a1, 3 + k);
            }
            S.h = initial_step(P, L0);
        }
        S.rdot_prev = fma(dd0, vs[3] - vs[0], fma(dd1, vs[4] - vs[1], dd2 * (vs[5] - vs[2])));
        S.t = 0.0; S.hmin = 0.0; S.t_first = 0.0; S.t_last = 0.0;
        S.n_acc = 0; S.n_rej = 0; S.n_bounce = 0; S.nofailed = true; S.retry = false;

        // ---- pass 1: forward with checkpoints
        int nck = 0;
        long long stride = buf.seg;
        ckpt_write(ckw, lane, x, v, a1, c1, S);
        nck = 1;
        PrimStep E;
        uint32_t st = 0xffffffffu;
        int res;
        for (;;) {
            const int r = prim_attempt(P, tl, lane, S, x, v, a1, c1, kq, ka, coef, E, st);
            if (r == PA_REJ) continue;
            if (r == PA_STOP) { res = 1; break; }
            if (r == PA_EXIT) { res = 2; break; }
            if ((long long)S.n_acc % stride == 0) {
                if (nck == buf.max_ckpt) {
                    // keep the even checkpoints (multiples of the doubled stride)
                    for (int k = 1; k < nck / 2; ++k) {
                        const double* src = ckw + (long long)(2 * k) * CK_DOUBLES;
                        double* dst = ckw + (long long)k * CK_DOUBLES;
                        if (lane < 6) {
                            dst[lane] = src[lane];
                            dst[6 + lane] = src[6 + lane];
                            dst[12 + lane] = src[12 + lane];
                        }
                        if (lane == 0)
                            for (int f = 18; f < 27; ++f) dst[f] = src[f];
                    }
                    nck /= 2;
                    stride *= 2;
                }
                if ((long long)S.n_acc % stride == 0) {
                    ckpt_write(ckw + (long long)nck * CK_DOUBLES, lane, x, v, a1, c1, S);
                    ++nck;
                }
            }
        }
        const long long n_com = res == 2 ? (long long)S.n_acc - 1 : (long long)S.n_acc;

        // ---- primal epilogue (as the tangent kernel) and the final state of every group
        Final fin;
        fin.s_exit = -1.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            fin.xi[k] = shfl(x, k); fin.xa[k] = shfl(x, 3 + k);
            fin.vi[k] = shfl(v, k); fin.va[k] = shfl(v, 3 + k);
        }
        fin.t = S.t;
        fin.status = st;
        double yfx = x, yfv = v;
        double ysx = 0.0, ysv = 0.0;
        if (res == 2) {
            StepData D;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                D.xi[k] = fin.xi[k]; D.xa[k] = fin.xa[k]; D.vi[k] = fin.vi[k]; D.va[k] = fin.va[k];
                D.a1i[k] = shfl(a1, k); D.a1a[k] = shfl(a1, 3 + k);
                D.a3i[k] = shfl(E.a3, k); D.a3a[k] = shfl(E.a3, 3 + k);
                D.a4i[k] = shfl(E.a4, k); D.a4a[k] = shfl(E.a4, 3 + k);
                D.a5i[k] = shfl(E.a5, k); D.a5a[k] = shfl(E.a5, 3 + k);
                D.a6i[k] = shfl(E.a6, k); D.a6a[k] = shfl(E.a6, 3 + k);
                D.a7i[k] = shfl(E.a7, k); D.a7a[k] = shfl(E.a7, 3 + k);
                D.xni[k] = shfl(E.xn, k); D.xna[k] = shfl(E.xn, 3 + k);
                D.vni[k] = shfl(E.vn, k); D.vna[k] = shfl(E.vn, 3 + k);
            }
            D.h = E.h;
            D.t = E.t;
            if (lane == 0) finish_exit(P, D, E.r2new, fin);
            fin.t = __shfl_sync(FULL, fin.t, 0);
            fin.s_exit = __shfl_sync(FULL, fin.s_exit, 0);
            fin.status = __shfl_sync(FULL, fin.status, 0);
            if (fin.s_exit >= 0.0) {
                const double s = fin.s_exit, s2 = s * s, h = E.h, h2 = h * h, sh = s * h;
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
                const double qx = fma(px6, E.a6, fma(px5, E.a5, fma(px4, E.a4, fma(px3, E.a3, px1 * a1))));
                const double ux = fma(b7, E.a7, fma(b6, E.a6, fma(b5, E.a5, fma(b4, E.a4, fma(b3, E.a3, b1 * a1)))));
                yfx = fma(h2, qx, fma(sh, v, x));
                yfv = fma(h, ux, v);
                const double dp1 = s * fma(s, 4.0 * DP_PX14, 3.0 * DP_PX13) + 2.0 * DP_PX12;
                const double dp3 = s * fma(s, 4.0 * DP_PX34, 3.0 * DP_PX33) + 2.0 * DP_PX32;
                const double dp4 = s * fma(s, 4.0 * DP_PX44, 3.0 * DP_PX43) + 2.0 * DP_PX42;
                const double dp5 = s * fma(s, 4.0 * DP_PX54, 3.0 * DP_PX53) + 2.0 * DP_PX52;
                const double dp6 = s * fma(s, 4.0 * DP_PX64, 3.0 * DP_PX63) + 2.0 * DP_PX62;
                const double db1 = fma(s, fma(s, 4.0 * DP_BI14, 3.0 * DP_BI13), 2.0 * DP_BI12) * s + DP_BI11;
                const double db3 = s * fma(s, 4.0 * DP_BI34, 3.0 * DP_BI33) + 2.0 * DP_BI32;
                const double db4 = s * fma(s, 4.0 * DP_BI44, 3.0 * DP_BI43) + 2.0 * DP_BI42;
                const double db5 = s * fma(s, 4.0 * DP_BI54, 3.0 * DP_BI53) + 2.0 * DP_BI52;
                const double db6 = s * fma(s, 4.0 * DP_BI64, 3.0 * DP_BI63) + 2.0 * DP_BI62;
                const double db7 = s * fma(s, 4.0 * DP_BI74, 3.0 * DP_BI73) + 2.0 * DP_BI72;
                const double dqx = s * (dp1 * a1 + dp3 * E.a3 + dp4 * E.a4 + dp5 * E.a5 + dp6 * E.a6);
                const double dux = db1 * a1 + s * (db3 * E.a3 + db4 * E.a4 + db5 * E.a5 + db6 * E.a6 + db7 * E.a7);
                ysx = fma(h, v, h2 * dqx);
                ysv = h * dux;
            } else {
                yfx = E.xn;
                yfv = E.vn;
            }
        }
        if (lane == 0) store_result(P, ic, out, i, tally(S), fin, true);

        // ---- pass 2: the terminal adjoint of each objective
        double y0v[12], yf[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) y0v[c] = __ldg(ic.y0 + c * ic.ld + i);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int pi = k < 3 ? k : k + 3;
            yf[pi] = shfl(yfx, tl.base + k);
            yf[pi + 3] = shfl(yfv, tl.base + k);
        }
        double gy0[12], gyf[12], gqe[3], jt;
        objective_partials(P, tl.dir, S.phi0, y0v, yf, fin.t, gy0, gyf, jt, gqe);
        double lx = gyf[yi], lv = gyf[yv];
        const double ex_x = gy0[yi], ex_v = gy0[yv];
        const double ex_q = tl.comp < 3 ? gqe[tl.comp] : 0.0;
        double gq = 0.0;
        int scale_e = 0;
        if (res == 2) {
            const bool ext = fin.s_exit >= 0.0;
            if (ext) {
                // exit-time correction: lambda -= c grad_y(d . d), c = (lambda . y_s + jt h) / (d . d_s)
                const int j = tl.comp < 3 ? tl.comp : tl.comp - 3;
                const double dprim = shfl(yfx, tl.base + 3 + j) - shfl(yfx, tl.base + j);
                const double dsep = shfl(ysx, tl.base + 3 + j) - shfl(ysx, tl.base + j);
                const double den = shfl(dprim, tl.base + 0) * shfl(dsep, tl.base + 0) +
                                   shfl(dprim, tl.base + 1) * shfl(dsep, tl.base + 1) +
                                   shfl(dprim, tl.base + 2) * shfl(dsep, tl.base + 2);
                const double part = fma(lx, ysx, lv * ysv);
                double ls = 0.0;
#pragma unroll
                for (int k = 0; k < 6; ++k) ls += shfl(part, tl.base + k);
                const double cc = (ls + jt * E.h) / den;
                lx -= cc * (tl.comp < 3 ? -dprim : dprim);
            }
            adj_step(P, tl, lane, x, v, E.t, E.h, c1, S.phi0, ext, fin.s_exit, kq, ka, coef, lx, lv, gq, sw);
            adj_rescale(tl, lx, lv, gq, scale_e);
        }

        // ---- pass 3: reverse sweep over the committed steps, in recomputed blocks
        __syncwarp();
        bool bad = false;
        long long hi = n_com;
        while (hi > 0 && !bad) {
            const long long c = (hi - 1) / stride;
            const long long base = c * stride;
            const long long lo = hi - buf.seg > base ? hi - buf.seg : base;
            Scal R;
            R.phi0 = S.phi0;
            double rx, rv, ra1, rc1;
            ckpt_read(ckw + c * CK_DOUBLES, tl.comp, rx, rv, ra1, rc1, R);
            long long k = base;
            while (k < hi) {
                const double x0 = rx, v0 = rv, c10 = rc1;
                uint32_t rst;
                PrimStep RE;
                const int r = prim_attempt(P, tl, lane, R, rx, rv, ra1, rc1, kq, ka, coef, RE, rst);
                if (r == PA_REJ) continue;
                if (r != PA_COMMIT) {
                    bad = true;
                    break;
                }
                if (k >= lo) {
                    double* rec = srw + (k - lo) * SR_DOUBLES;
                    if (lane < 6) {
                        rec[lane] = x0;
                        rec[6 + lane] = v0;
                    }
                    if (lane == 0) {
                        rec[12] = RE.t;
                        rec[13] = RE.h;
                        rec[14] = c10;
                    }
                }
                ++k;
            }
            __syncwarp();
            if (bad) break;
            for (long long kk = hi - 1; kk >= lo; --kk) {
                const double* rec = srw + (kk - lo) * SR_DOUBLES;
                const double sx = rec[tl.comp], sv = rec[6 + tl.comp];
                const double st0 = rec[12], sh0 = rec[13], sc1 = rec[14];
                adj_step(P, tl, lane, sx, sv, st0, sh0, sc1, S.phi0, false, 0.0, kq, ka, coef, lx, lv, gq, sw);
                adj_rescale(tl, lx, lv, gq, scale_e);
            }
            __syncwarp();
            hi = lo;
        }
        if (bad) {
            if (lane == 0) atomicAdd(buf.errors, 1ull);
            adj_zero_outputs(ain, aout, tl, lane, i, __longlong_as_double(0x7ff8000000000000ll));
            continue;
        }

        // ---- outputs: gradients (scaled back, plus the explicit terms) and seed projections
        const double gx = ldexp(lx, scale_e) + ex_x;
        const double gv = ldexp(lv, scale_e) + ex_v;
        const double gqt = tl.comp < 3 ? ldexp(gq, scale_e) + ex_q : 0.0;
        if (tl.dir > 0 && lane < 30) {
            const int obj = tl.dir - 1;
            if (aout.grad_y0) {
                aout.grad_y0[((long long)obj * 12 + yi) * aout.ld + i] = gx;
                aout.grad_y0[((long long)obj * 12 + yv) * aout.ld + i] = gv;
            }
            if (aout.grad_q && tl.comp < 3) aout.grad_q[((long long)obj * 3 + tl.comp) * aout.ld + i] = gqt;
        }
        for (int kd = 0; kd < ain.ndir; ++kd) {
            double part = gx * __ldg(ain.dy0 + ((long long)kd * 12 + yi) * ain.ld + i) +
                          gv * __ldg(ain.dy0 + ((long long)kd * 12 + yv) * ain.ld + i);
            if (tl.comp < 3) part = fma(gqt, ain.dq[kd][tl.comp], part);
            double sum = 0.0;
#pragma unroll
            for (int c = 0; c < 6; ++c) sum += shfl(part, tl.base + c);
            if (tl.dir > 0 && tl.comp == 0 && lane < 30) {
                const int obj = tl.dir - 1;
                double* dst = obj == 0 ? aout.d_theta : obj == 1 ? aout.d_dp : obj == 2 ? aout.d_dE : aout.d_tf;
                dst[(long long)kd * aout.ld + i] = sum;
            }
        }
    }
}

}  // namespace ia
