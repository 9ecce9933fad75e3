/*
 * ia_sample_oracle.c -- CPU oracle of the counter-based initial-condition samplers.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE, like ia_oracle.c beside it: only the test suite and the
 * CPU legs of the benchmark load it. It shares no source with the CUDA library. Both sides implement
 * the same counter-based generator from its published definition and the same sampling recipe,
 * each in its own code, so that initial conditions drawn on the GPU can be checked one by one.
 *
 * Random numbers: Philox4x64-10 of Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3" (SC'11). The state is a counter of four 64-bit words and a key of two. One round
 * multiplies counter words 0 and 2 by two fixed odd constants into 128-bit products. The new
 * counter is (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)). The key is bumped
 * by two Weyl constants (the 64-bit golden ratio and sqrt(3) - 1) before every round but the first.
 * Ten rounds make one block of four 64-bit outputs.
 *
 * Uniform variates: u = (2 floor(x / 2^12) + 1) 2^-53 for an output word x. This is an odd multiple
 * of 2^-53, so u lies in the open interval (0, 1) and is exact in double precision.
 *
 * Draw layout of trajectory g (its global index) under seed s and sampler kind k:
 *   - Block j = 0..3 is Philox4x64-10 of counter (g, j, 0, 0) with key (s, k). Word w of block j is
 *     uniform u[4j + w].
 *   - u[0] gives the rf phase phi0 = 2 pi u[0] when the phase is random.
 *   - u[1] and u[2] give the direction or the point on the disk.
 *   - u[3] is unused.
 *   - Box and Muller (1958): the pair (u[4 + 2p], u[5 + 2p]), p = 0..4, gives
 *     g[2p] = rho cos(2 pi u[5 + 2p]) and g[2p + 1] = rho sin(2 pi u[5 + 2p]),
 *     with rho = sqrt(-2 ln u[4 + 2p]).
 *   - g[0..2] are the atom's velocity, g[3..5] the ion's secular position, g[6..8] the ion's
 *     secular velocity, each in units of its standard deviation. g[9] is unused.
 *
 * The samplers (arXiv 2509.15117):
 *   - Head-on runs (head-on paragraph, Fig. 1 caption). The ion is at rest at the centre. The atom
 *     starts at r0 x_hat and moves with velocity -v0 x_hat, v0 = sqrt(2E/m_a). The direction x_hat is
 *     uniform on the octant's surface: cos(theta) = u[1], phi = (pi/2) u[2].
 *   - Thermal runs (thermal paragraph, Fig. 3 caption). The atom position is uniform on the r0
 *     sphere, with cos(theta) = 2 u[1] - 1 and phi = 2 pi u[2]. Its velocity components are Gaussian
 *     with variance k_B T / m_a; the whole vector is negated when it does not point inward
 *     (v . x_hat >= 0). The ion is Gaussian at T_ion in an isotropic harmonic trap of frequency
 *     omega = |q_x| Omega / 2^(3/2). The position per axis has variance k_B T_ion / (m_i omega^2)
 *     and the velocity k_B T_ion / m_i.
 *   - The disk variant of the thermal runs. The atom velocity is as above. The impact parameter is
 *     b = b_max sqrt(u[1]) at azimuth psi = 2 pi u[2], in the plane perpendicular to v_hat spanned by
 *     e1 = unit(v_hat x r) and e2 = v_hat x e1, with r = z_hat if |v_hat_z| < 0.9, else x_hat. The atom
 *     starts at b (cos psi e1 + sin psi e2) - sqrt(r0^2 - b^2) v_hat, on the r0 sphere.
 *   - Optional micromotion of the thermal ion, the lowest-order Mathieu solution at the rf phase
 *     phi0 with the trap sign s:
 *       x_j = X_j (1 + s (q_j / 2) cos phi0),
 *       v_j = V_j (1 + s (q_j / 2) cos phi0) - X_j s (q_j Omega / 2) sin phi0.
 *
 * Compiled with -ffp-contract=off like ia_oracle.c: every operation is one IEEE-754 double operation
 * in source order.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define SMP_PI 3.14159265358979323846

/* Philox4x64-10 constants (Salmon et al., SC'11): round multipliers and Weyl key increments. */
static const uint64_t PHILOX_M0 = 0xD2E7470EE14C6C93ull;
static const uint64_t PHILOX_M1 = 0xCA5A826395121157ull;
static const uint64_t PHILOX_W0 = 0x9E3779B97F4A7C15ull;
static const uint64_t PHILOX_W1 = 0xBB67AE8584CAA73Bull;

/* One Philox4x64-10 block: out = bijection of ctr under key. */
void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        const unsigned __int128 p0 = (unsigned __int128)PHILOX_M0 * c0;
        const unsigned __int128 p1 = (unsigned __int128)PHILOX_M1 * c2;
        const uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        const uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* n consecutive blocks: block j has counter (first + j, ctr1, 0, 0) and key (key0, key1). */
void orc_philox4x64_stream(uint64_t key0, uint64_t key1, uint64_t ctr1, int64_t first, int64_t n, uint64_t* out)
{
    const uint64_t key[2] = {key0, key1};
    for (int64_t j = 0; j < n; ++j) {
        const uint64_t ctr[4] = {(uint64_t)(first + j), ctr1, 0, 0};
        orc_philox4x64(ctr, key, out + 4 * j);
    }
}

/* Open-interval uniform of one output word: an odd multiple of 2^-53. */
static double uniform01(uint64_t x) { return (double)((x >> 11) | 1u) * 0x1p-53; }

/* Sampler kinds (the oracle's numbering, the same values as the library's). */
enum { SMP_HEAD_ON = 0, SMP_SPHERE = 1, SMP_DISK = 2 };

typedef struct {
    int32_t kind;          /* SMP_HEAD_ON, SMP_SPHERE or SMP_DISK */
    int32_t random_phase;  /* 1: phi0 = 2 pi u[0]; 0: phi0 = phase */
    int32_t micromotion;   /* thermal kinds: add the ion's lowest-order micromotion */
    int32_t rf_sign;       /* s of the trap term */
    double m_ion, m_atom;  /* m_e */
    double Omega;          /* rad per a.u. of time */
    double q[3];           /* Mathieu q per axis */
    double r0;             /* a0 */
    double E;              /* head-on collision energy, E_h */
    double kT;             /* thermal: k_B T of the atom, E_h */
    double kT_ion;         /* thermal: k_B T of the ion, E_h */
    double b_max;          /* disk radius, a0 */
    double phase;          /* fixed rf phase */
    uint64_t seed;
} orc_sampler;

/* The sixteen uniforms of trajectory g. */
static void draw_uniforms(const orc_sampler* s, int64_t g, double u[16])
{
    const uint64_t key[2] = {s->seed, (uint64_t)(uint32_t)s->kind};
    for (int j = 0; j < 4; ++j) {
        const uint64_t ctr[4] = {(uint64_t)g, (uint64_t)j, 0, 0};
        uint64_t w[4];
        orc_philox4x64(ctr, key, w);
        for (int k = 0; k < 4; ++k) u[4 * j + k] = uniform01(w[k]);
    }
}

/* Box-Muller: ten standard normal variates from u[4..13]. */
static void gaussians(const double u[16], double gz[10])
{
    for (int p = 0; p < 5; ++p) {
        const double rho = sqrt(-2.0 * log(u[4 + 2 * p]));
        const double ang = 2.0 * SMP_PI * u[5 + 2 * p];
        gz[2 * p] = rho * cos(ang);
        gz[2 * p + 1] = rho * sin(ang);
    }
}

/* Initial state of trajectory g: y = [x_ion(3), v_ion(3), x_atom(3), v_atom(3)] and phi0. */
static void sample_one(const orc_sampler* s, int64_t g, double y[12], double* phi0)
{
    double u[16];
    draw_uniforms(s, g, u);
    const double ph = s->random_phase ? 2.0 * SMP_PI * u[0] : s->phase;
    *phi0 = ph;
    for (int c = 0; c < 12; ++c) y[c] = 0.0;

    if (s->kind == SMP_HEAD_ON) {
        const double ct = u[1];
        const double st = sqrt((1.0 - ct) * (1.0 + ct));
        const double az = 0.5 * SMP_PI * u[2];
        const double xh[3] = {st * cos(az), st * sin(az), ct};
        const double v0 = sqrt(2.0 * s->E / s->m_atom);
        for (int j = 0; j < 3; ++j) {
            y[6 + j] = s->r0 * xh[j];
            y[9 + j] = -v0 * xh[j];
        }
        return;
    }

    double gz[10];
    gaussians(u, gz);
    const double sig_a = sqrt(s->kT / s->m_atom);
    double v[3] = {sig_a * gz[0], sig_a * gz[1], sig_a * gz[2]};

    if (s->kind == SMP_SPHERE) {
        const double ct = 2.0 * u[1] - 1.0;
        const double st = sqrt((1.0 - ct) * (1.0 + ct));
        const double az = 2.0 * SMP_PI * u[2];
        const double xh[3] = {st * cos(az), st * sin(az), ct};
        const double vr = v[0] * xh[0] + v[1] * xh[1] + v[2] * xh[2];
        if (vr >= 0.0)
            for (int j = 0; j < 3; ++j) v[j] = -v[j];
        for (int j = 0; j < 3; ++j) y[6 + j] = s->r0 * xh[j];
    } else {
        const double vn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        const double vh[3] = {v[0] / vn, v[1] / vn, v[2] / vn};
        const double ref[3] = {fabs(vh[2]) < 0.9 ? 0.0 : 1.0, 0.0, fabs(vh[2]) < 0.9 ? 1.0 : 0.0};
        double e1[3] = {vh[1] * ref[2] - vh[2] * ref[1], vh[2] * ref[0] - vh[0] * ref[2],
                        vh[0] * ref[1] - vh[1] * ref[0]};
        const double n1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
        for (int j = 0; j < 3; ++j) e1[j] /= n1;
        const double e2[3] = {vh[1] * e1[2] - vh[2] * e1[1], vh[2] * e1[0] - vh[0] * e1[2],
                              vh[0] * e1[1] - vh[1] * e1[0]};
        const double b = s->b_max * sqrt(u[1]);
        const double psi = 2.0 * SMP_PI * u[2];
        const double back = sqrt(s->r0 * s->r0 - b * b);
        for (int j = 0; j < 3; ++j)
            y[6 + j] = b * (cos(psi) * e1[j] + sin(psi) * e2[j]) - back * vh[j];
    }
    for (int j = 0; j < 3; ++j) y[9 + j] = v[j];

    /* thermal ion in the isotropic secular trap, optionally with micromotion */
    const double omega = fabs(s->q[0]) * s->Omega / (2.0 * sqrt(2.0));
    const double sig_v = sqrt(s->kT_ion / s->m_ion);
    const double sig_x = s->kT_ion > 0.0 ? sig_v / omega : 0.0;
    for (int j = 0; j < 3; ++j) {
        const double X = sig_x * gz[3 + j];
        const double V = sig_v * gz[6 + j];
        if (s->micromotion) {
            const double f = 1.0 + s->rf_sign * (0.5 * s->q[j]) * cos(ph);
            y[j] = X * f;
            y[3 + j] = V * f - X * s->rf_sign * (0.5 * s->q[j] * s->Omega) * sin(ph);
        } else {
            y[j] = X;
            y[3 + j] = V;
        }
    }
}

/* n initial states of the trajectories first .. first + n - 1: y row-major n x 12, phi0 n.
 * Returns 0, or -1 when the sampler's parameters are out of range. */
int orc_sample_ics(const orc_sampler* s, int64_t first, int64_t n, double* y, double* phi0)
{
    if (s->kind < SMP_HEAD_ON || s->kind > SMP_DISK || first < 0 || n < 0) return -1;
    if (!(s->m_ion > 0.0) || !(s->m_atom > 0.0) || !(s->r0 > 0.0)) return -1;
    if (s->kind == SMP_HEAD_ON && !(s->E > 0.0)) return -1;
    if (s->kind != SMP_HEAD_ON) {
        if (!(s->kT > 0.0) || !(s->kT_ion >= 0.0)) return -1;
        if (s->kT_ion > 0.0 && !(fabs(s->q[0]) * s->Omega > 0.0)) return -1;
        if (s->kind == SMP_DISK && !(s->b_max >= 0.0 && s->b_max < s->r0)) return -1;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) sample_one(s, first + i, y + 12 * i, phi0 + i);
    return 0;
}
