// ia_sample.cuh -- initial conditions drawn on the device from a counter-based generator.
//
// The paper's runs start from sampled initial conditions (arXiv 2509.15117):
//   - head-on runs: ion at rest at the trap centre; the atom on the r0 sphere moving radially inward
//     with E = m_a v0^2 / 2 (head-on paragraph), over the octant of Fig. 1;
//   - thermal runs: the ion Gaussian at T_ion in an isotropic harmonic trap of frequency
//     omega = q_x Omega / 2^(3/2); the atom uniform on the r0 sphere, velocity components Gaussian at T,
//     negated to point inward (thermal paragraph, Fig. 3 caption);
//   - a random rf phase Omega t0 mod 2 pi (Fig. 4 caption).
// Drawing them here removes the host sampling and the host-to-device copy of 104 bytes per trajectory
// for batches of 10^8 and more. Every trajectory draws from its own counter, so any index range can
// be generated alone (by chunks, or by ranks) and gives the same values as the whole batch.
//
// Generator: Philox4x64-10 (Salmon, Moraes, Dror & Shaw, SC'11). A round maps the counter words
// (c0, c1, c2, c3) under the key (k0, k1) to (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1,
// lo(M0 c0)). The key takes one Weyl increment before each round after the first. Ten rounds.
// The 64x64 -> 128-bit products use __umul64hi and the low 64-bit product.
//
// Draw layout, the contract that ia_sample_ics documents:
//   - block j = 0..3 of trajectory g is the counter (g, j, 0, 0) under the key (seed, kind);
//   - u[4j + w] = ((word_w >> 11) | 1) 2^-53, an exact odd multiple of 2^-53 in (0, 1);
//   - u[0]: rf phase; u[1], u[2]: direction or disk point; u[3]: unused;
//   - u[4..13]: five Box-Muller pairs giving Gaussians g[0..9]. g[0..2] are the atom velocity,
//     g[3..5] the ion's secular position, g[6..8] its secular velocity.
#pragma once

#include <cstdint>

namespace ia_sample {

constexpr unsigned long long PHILOX_M0 = 0xD2E7470EE14C6C93ull;
constexpr unsigned long long PHILOX_M1 = 0xCA5A826395121157ull;
constexpr unsigned long long PHILOX_W0 = 0x9E3779B97F4A7C15ull;  // 2^64 / golden ratio
constexpr unsigned long long PHILOX_W1 = 0xBB67AE8584CAA73Bull;  // 2^64 (sqrt(3) - 1)
constexpr int SAMPLE_THREADS = 256;

struct SampleParams {
    int kind;             // 0 head-on, 1 thermal sphere, 2 thermal disk
    int random_phase;
    int micromotion;
    int rf_sign;
    double r0, v0;        // head-on speed
    double sig_a;         // atom velocity standard deviation sqrt(kT/m_a)
    double sig_x, sig_v;  // ion secular position and velocity standard deviations
    double b_max, phase, Omega;
    double q[3];
    unsigned long long seed;
    long long first, n, ld;
    double* y0;
    double* phi0;
};

__device__ __forceinline__ void philox4x64_10(unsigned long long c[4], unsigned long long k0, unsigned long long k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        const unsigned long long hi0 = __umul64hi(PHILOX_M0, c[0]), lo0 = PHILOX_M0 * c[0];
        const unsigned long long hi1 = __umul64hi(PHILOX_M1, c[2]), lo1 = PHILOX_M1 * c[2];
        const unsigned long long n0 = hi1 ^ c[1] ^ k0;
        const unsigned long long n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

__device__ __forceinline__ double uniform01(unsigned long long x)
{
    return (double)((x >> 11) | 1ull) * 0x1p-53;
}

// Four uniforms of block j of trajectory g.
__device__ __forceinline__ void block_uniforms(unsigned long long seed, int kind, long long g, int j, double* u)
{
    unsigned long long c[4] = {(unsigned long long)g, (unsigned long long)j, 0ull, 0ull};
    philox4x64_10(c, seed, (unsigned long long)(unsigned)kind);
#pragma unroll
    for (int w = 0; w < 4; ++w) u[w] = uniform01(c[w]);
}

// Box-Muller pair from (u_r, u_a): rho = sqrt(-2 ln u_r), angle 2 pi u_a.
__device__ __forceinline__ void box_muller(double u_r, double u_a, double& z0, double& z1)
{
    const double rho = sqrt(-2.0 * log(u_r));
    double s, c;
    sincospi(2.0 * u_a, &s, &c);
    z0 = rho * c;
    z1 = rho * s;
}

__global__ void __launch_bounds__(SAMPLE_THREADS) k_sample(SampleParams p)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += stride) {
        const long long g = p.first + i;
        double u[16];
        block_uniforms(p.seed, p.kind, g, 0, u);
        const double ph = p.random_phase ? 2.0 * 3.14159265358979323846 * u[0] : p.phase;
        double y[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) y[c] = 0.0;

        if (p.kind == 0) {
            const double ct = u[1];
            const double st = sqrt((1.0 - ct) * (1.0 + ct));
            double sa, ca;
            sincospi(0.5 * u[2], &sa, &ca);
            const double xh[3] = {st * ca, st * sa, ct};
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                y[6 + j] = p.r0 * xh[j];
                y[9 + j] = -p.v0 * xh[j];
            }
        } else {
            block_uniforms(p.seed, p.kind, g, 1, u + 4);
            block_uniforms(p.seed, p.kind, g, 2, u + 8);
            block_uniforms(p.seed, p.kind, g, 3, u + 12);
            double gz[10];
#pragma unroll
            for (int q = 0; q < 5; ++q) box_muller(u[4 + 2 * q], u[5 + 2 * q], gz[2 * q], gz[2 * q + 1]);
            double v[3] = {p.sig_a * gz[0], p.sig_a * gz[1], p.sig_a * gz[2]};
            if (p.kind == 1) {
                const double ct = 2.0 * u[1] - 1.0;
                const double st = sqrt((1.0 - ct) * (1.0 + ct));
                double sa, ca;
                sincospi(2.0 * u[2], &sa, &ca);
                const double xh[3] = {st * ca, st * sa, ct};
                const double vr = v[0] * xh[0] + v[1] * xh[1] + v[2] * xh[2];
                if (vr >= 0.0) {
                    v[0] = -v[0];
                    v[1] = -v[1];
                    v[2] = -v[2];
                }
#pragma unroll
                for (int j = 0; j < 3; ++j) y[6 + j] = p.r0 * xh[j];
            } else {
                const double vn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
                const double vh[3] = {v[0] / vn, v[1] / vn, v[2] / vn};
                // e1 = unit(v_hat x r), r = z_hat unless v_hat is within ~26 degrees of the z axis
                const bool use_z = fabs(vh[2]) < 0.9;
                double e1[3];
                if (use_z) {
                    e1[0] = vh[1];
                    e1[1] = -vh[0];
                    e1[2] = 0.0;
                } else {
                    e1[0] = 0.0;
                    e1[1] = vh[2];
                    e1[2] = -vh[1];
                }
                const double n1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
                e1[0] /= n1;
                e1[1] /= n1;
                e1[2] /= n1;
                const double e2[3] = {vh[1] * e1[2] - vh[2] * e1[1], vh[2] * e1[0] - vh[0] * e1[2],
                                      vh[0] * e1[1] - vh[1] * e1[0]};
                const double b = p.b_max * sqrt(u[1]);
                double sp, cp;
                sincospi(2.0 * u[2], &sp, &cp);
                const double back = sqrt(p.r0 * p.r0 - b * b);
#pragma unroll
                for (int j = 0; j < 3; ++j) y[6 + j] = b * (cp * e1[j] + sp * e2[j]) - back * vh[j];
            }
#pragma unroll
            for (int j = 0; j < 3; ++j) y[9 + j] = v[j];
            double sph = 0.0, cph = 1.0;
            if (p.micromotion) sincos(ph, &sph, &cph);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const double X = p.sig_x * gz[3 + j];
                const double V = p.sig_v * gz[6 + j];
                if (p.micromotion) {
                    const double f = 1.0 + p.rf_sign * (0.5 * p.q[j]) * cph;
                    y[j] = X * f;
                    y[3 + j] = V * f - X * p.rf_sign * (0.5 * p.q[j] * p.Omega) * sph;
                } else {
                    y[j] = X;
                    y[3 + j] = V;
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 12; ++c) p.y0[(long long)c * p.ld + i] = y[c];
        p.phi0[i] = ph;
    }
}

// Raw blocks: block j has the counter (first + j, ctr1, 0, 0) under the key (key0, key1).
__global__ void __launch_bounds__(SAMPLE_THREADS) k_philox(unsigned long long key0, unsigned long long key1,
                                                           unsigned long long ctr1, long long first, long long n,
                                                           unsigned long long* out)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        unsigned long long c[4] = {(unsigned long long)(first + j), ctr1, 0ull, 0ull};
        philox4x64_10(c, key0, key1);
#pragma unroll
        for (int w = 0; w < 4; ++w) out[4 * j + w] = c[w];
    }
}

}  // namespace ia_sample
