// ia_tangent.cuh -- forward (tangent) differentiation of the trajectory map, and finite-time
// Lyapunov exponents.
//
// What is differentiated: the computed map from (initial state, trap q vector) to the observables,
// with the step sizes and accept/reject decisions of the primal run held fixed (the discrete tangent
// of the DP5 recursion), plus the sensitivity of the exit time: the crossing |d| = r0 is found on the
// continuous extension at fraction s* of the last step, and
//     ds*/dp = -(d . dd/dp) / (d . dd/ds),   dy_f/dp = Y(s*) + (dy/ds)(s*) ds*/dp,   dt_f/dp = h ds*/dp,
// with Y(s*) the continuous extension applied to the tangent stages. The observables of the Fig. 1
// caption (scattering angle, momentum transfer of the atom) and the ion energy change are then
// differentiated by the chain rule, including their dependence on the initial state and on q.
//
// Layout: one trajectory per warp. Lane = dir * 6 + comp, dir 0 is the primal and dir 1..4 the
// tangent directions, comp indexes [x_ion(3), x_atom(3)] with its velocity and stage accelerations;
// lanes 30 and 31 are spare. The stage sums are linear, so one instruction stream advances the
// primal and every tangent; the force step is one expression that gives the primal exactly the
// lane-mode bits and the tangents the linearised force
//     dF = g dd + 2 g_u (d . dd) d,   g = -V'(r)/r,   g_u = dg / d(r^2),
// plus, for the ion, (dkq cos(Omega t + phi0)) x_ion from a change of q. So the primal results of
// ia_launch_tangent are those of ia_launch, bit for bit.
//
// FTLE: each tangent direction carries a power-of-two scale exponent; when its largest entry leaves
// [2^-256, 2^256] the direction is rescaled exactly (Benettin renormalisation without rounding). The
// FTLE of direction 1 is (ln|Y_f| + E ln 2 - ln|Y_0|) / t_f in the norm with positions in units of
// r_e and velocities in units of sqrt(2 D_e / mu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ia_traj.cuh"

namespace ia {

struct TanIn {
    const double* dy0;  // [ndir][12][ld]
    double dq[4][3];    // d q_vector / d p_k
    int ndir;
    long long ld;
};

struct TanOut {
    double* d_theta;   // [ndir][ld]
    double* d_dp;
    double* d_dE;
    double* d_tf;
    double* dy_final;  // [ndir][12][ld] or null
    double* ftle;      // [ld] or null
    long long ld;
};

struct TLane {
    int dir, comp, base;
};

__device__ __forceinline__ TLane tlane()
{
    const int lane = threadIdx.x & 31;
    TLane t;
    int d = lane / 6;
    if (d > 4) d = 4;
    t.dir = d;
    t.base = d * 6;
    t.comp = lane - t.base;
    if (t.comp > 5) t.comp = 5;
    return t;
}

// Stage acceleration component of this lane (primal or tangent); see the file comment.
__device__ __forceinline__ double tan_accel(const SysDev& P, const TLane& tl, double p, double cs, double kq, double ka,
                                            double dkq, double coef, double& r2out, double d3[3])
{
    const int j = tl.comp < 3 ? tl.comp : tl.comp - 3;
    const double dd = shfl(p, tl.base + 3 + j) - shfl(p, tl.base + j);
    const double d0 = shfl(dd, 0), d1 = shfl(dd, 1), d2 = shfl(dd, 2);
    const double r2 = fma(d0, d0, fma(d1, d1, d2 * d2));
    const double s = rcp_nr(r2);
    const double s2 = s * s;
    const double s3 = fma(s2, s, 0.0);
    // coef g with the 1/m folded into the constants (the primal expression of the other layouts)
    const bool ion = tl.comp < 3;
    const double gm = s3 * fma(ion ? P.ci8 : P.ca8, s2, -(ion ? P.ci4 : P.ca4));
    // dg/d(r^2) = s^4 (12 C4 - 40 C8 s^2)
    const double gu = (s2 * s2) * fma(-5.0 * P.c8x8, s2, 3.0 * P.c4x4);
    const double e0 = shfl(dd, tl.base + 0), e1 = shfl(dd, tl.base + 1), e2 = shfl(dd, tl.base + 2);
    const double dot = fma(d0, e0, fma(d1, e1, d2 * e2));
    const double S = tl.dir == 0 ? 0.0 : (2.0 * gu) * dot;
    const double q1 = gm * dd;
    const double dj = j == 0 ? d0 : (j == 1 ? d1 : d2);
    const double q2 = fma(coef * S, dj, q1);
    const double kc = fma(kq, cs, ka);
    const double xprim = shfl(p, tl.comp);
    const double q3 = q2 + (dkq * cs) * xprim;
    r2out = r2;
    d3[0] = d0;
    d3[1] = d1;
    d3[2] = d2;
    return fma(kc, p, q3);
}

// Derivatives of the observables along one direction (chain rule; see the file comment).
// y0, yf: primal initial and final states; dy0, dyf: their tangents; dtf: exit-time tangent;
// dq: q-vector tangent; tf: primal final time. Outputs dtheta, ddp, ddE.
__device__ __noinline__ void obs_derivs(const SysDev& P, double phi0, const double* y0, const double* yf, double tf,
                                        const double* dy0, const double* dyf, double dtf, const double* dq,
                                        double& dtheta, double& ddp, double& ddE)
{
    const double* v0 = y0 + 9;
    const double* vf = yf + 9;
    const double* dv0 = dy0 + 9;
    const double* dvf = dyf + 9;
    double c[3] = {v0[1] * vf[2] - v0[2] * vf[1], v0[2] * vf[0] - v0[0] * vf[2], v0[0] * vf[1] - v0[1] * vf[0]};
    double dc[3] = {dv0[1] * vf[2] - dv0[2] * vf[1] + v0[1] * dvf[2] - v0[2] * dvf[1],
                    dv0[2] * vf[0] - dv0[0] * vf[2] + v0[2] * dvf[0] - v0[0] * dvf[2],
                    dv0[0] * vf[1] - dv0[1] * vf[0] + v0[0] * dvf[1] - v0[1] * dvf[0]};
    const double C = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    const double D = v0[0] * vf[0] + v0[1] * vf[1] + v0[2] * vf[2];
    const double dC = C > 0.0 ? (c[0] * dc[0] + c[1] * dc[1] + c[2] * dc[2]) / C : 0.0;
    const double dD = dv0[0] * vf[0] + dv0[1] * vf[1] + dv0[2] * vf[2] + v0[0] * dvf[0] + v0[1] * dvf[1] + v0[2] * dvf[2];
    dtheta = (D * dC - C * dD) / (C * C + D * D);
    double u[3] = {vf[0] - v0[0], vf[1] - v0[1], vf[2] - v0[2]};
    const double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    ddp = un > 0.0 ? P.m_a * (u[0] * (dvf[0] - dv0[0]) + u[1] * (dvf[1] - dv0[1]) + u[2] * (dvf[2] - dv0[2])) / un : 0.0;
    // E_ion = m |v_i|^2 / 2 + sum_j (ua_j + uq_j cos(Omega t + phi0)) x_j^2
    const double cf = cos(P.Omega * tf + phi0), sf = sin(P.Omega * tf + phi0), c0 = cos(phi0);
    double e = 0.0;
    for (int j = 0; j < 3; ++j) {
        const double xf = yf[j], x0 = y0[j];
        e += P.m_i * (yf[3 + j] * dyf[3 + j] - y0[3 + j] * dy0[3 + j]);
        e += 2.0 * (P.ua[j] + P.uq[j] * cf) * xf * dyf[j] - 2.0 * (P.ua[j] + P.uq[j] * c0) * x0 * dy0[j];
        e += -P.uq[j] * P.Omega * sf * xf * xf * dtf;
        e += P.uq_per_q * dq[j] * (cf * xf * xf - c0 * x0 * x0);
    }
    ddE = e;
}

__device__ __forceinline__ int max_exp3(double a, double b, double c)
{
    const int ea = (__double2hiint(a) >> 20) & 0x7ff, eb = (__double2hiint(b) >> 20) & 0x7ff;
    const int ec = (__double2hiint(c) >> 20) & 0x7ff;
    return max(ea, max(eb, ec));
}

}  // namespace ia
