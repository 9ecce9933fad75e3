// ia_stats.cuh -- batch statistics of the observables (ensemble step of the method).
//
// The paper turns its trajectory ensembles into complex-formation probabilities (Fig. 3, Fig. 4),
// bounce-count maps (Fig. 1c) and complex lifetime survival curves (Fig. 2). This reduction gives, per
// cell (any grouping of trajectories, e.g. one cell per system), exact integer counts and histograms
// and two floating-point sums, Sigma dE_ion and Sigma dE_ion^2, that are summed in a fixed order so a
// rerun gives the same bits:
//   pass 1: each block takes a contiguous range of trajectories; lanes of a warp that share a cell
//           are combined in lane order (match_any + shuffles), each warp keeps its own per-cell sums
//           in shared memory, and the block adds its warps in warp order into a per-block partial;
//   pass 2: one thread per cell adds the block partials in block order.
// Counts use integer atomics, which are exact whatever their order.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ia_traj.cuh"
#include "../../include/ionatom.h"

namespace ia {

constexpr int STATS_BLOCK = 256;
constexpr int STATS_MAX_CELLS = 1024;

__device__ __forceinline__ int bounce_bin(int nb)
{
    if (nb <= 0) return 0;
    int b = 1 + (31 - __clz(nb));  // 1: one bounce, 2: 2-3, 3: 4-7, ...
    return b < IA_STATS_BOUNCE_BINS ? b : IA_STATS_BOUNCE_BINS - 1;
}

// Complex lifetime t_last - t_first in a.u. of time, two bins per octave from 2^20 a.u. (~25 ps):
// bin = floor(2 (log2 tau - 20)), from the exponent and a comparison of the mantissa with sqrt(2).
__device__ __forceinline__ int lifetime_bin(double tau)
{
    if (!(tau > 0.0)) return 0;
    const long long bits = __double_as_longlong(tau);
    const int e = (int)((bits >> 52) & 0x7ff) - 1023;
    const int half = ((bits & 0xfffffffffffffLL) >= 0x6a09e667f3bcdLL) ? 1 : 0;  // mantissa >= sqrt(2)
    int b = 2 * (e - 20) + half;
    if (b < 0) b = 0;
    if (b >= IA_STATS_LIFETIME_BINS) b = IA_STATS_LIFETIME_BINS - 1;
    return b;
}

__global__ void __launch_bounds__(STATS_BLOCK) k_stats_pass1(ObsPtrs obs, long long n, const int32_t* __restrict__ cell,
                                                             int n_cells, ia_stats* __restrict__ st,
                                                             double* __restrict__ partial, long long chunk)
{
    extern __shared__ double sh[];  // [warps][n_cells][2]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int W = STATS_BLOCK / 32;
    for (int k = threadIdx.x; k < W * n_cells * 2; k += STATS_BLOCK) sh[k] = 0.0;
    __syncthreads();
    double* mine = sh + (size_t)warp * n_cells * 2;
    const long long lo = (long long)blockIdx.x * chunk;
    const long long hi = lo + chunk < n ? lo + chunk : n;
    for (long long base = lo + (long long)warp * 32; base < hi; base += STATS_BLOCK) {
        const long long i = base + lane;
        const bool in = i < hi;
        int c = -1;
        double dE = 0.0;
        if (in) {
            c = cell ? cell[i] : 0;
            if (c < 0 || c >= n_cells) c = -1;
        }
        if (c >= 0) {
            const uint32_t status = obs.status[i];
            const int nb = obs.n_bounce[i];
            ia_stats* s = st + c;
            atomicAdd((unsigned long long*)&s->n, 1ull);
            atomicAdd((unsigned long long*)&s->attempts,
                      (unsigned long long)((long long)obs.n_steps[i] + (long long)obs.n_rej[i]));
            if (nb >= 2) {
                atomicAdd((unsigned long long*)&s->n_complex, 1ull);
                atomicAdd((unsigned long long*)&s->lifetime_hist[lifetime_bin(obs.t_last[i] - obs.t_first[i])], 1ull);
            }
            atomicAdd((unsigned long long*)&s->bounce_hist[bounce_bin(nb)], 1ull);
            if ((status & 0xffu) == 0u) atomicAdd((unsigned long long*)&s->n_status[IA_STATS_EXIT_SLOT], 1ull);
#pragma unroll
            for (int b = 0; b < 6; ++b)
                if (status & (1u << b)) atomicAdd((unsigned long long*)&s->n_status[b], 1ull);
            dE = obs.dE_ion[i];
        }
        // lanes with the same cell: the lowest lane adds the group's values in lane order
        const unsigned same = __match_any_sync(FULL, c);
        double s1 = 0.0, s2 = 0.0;
        unsigned m = same;
        while (m) {
            const int src = __ffs(m) - 1;
            const double v = __shfl_sync(same, dE, src);
            s1 += v;
            s2 = fma(v, v, s2);
            m &= m - 1;
        }
        if (c >= 0 && lane == __ffs(same) - 1) {
            mine[2 * c] += s1;
            mine[2 * c + 1] += s2;
        }
        __syncwarp();
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n_cells * 2; k += STATS_BLOCK) {
        double a = 0.0;
        for (int w = 0; w < W; ++w) a += sh[(size_t)w * n_cells * 2 + k];
        partial[(size_t)blockIdx.x * n_cells * 2 + k] = a;
    }
}

__global__ void k_stats_pass2(const double* __restrict__ partial, int n_blocks, int n_cells, ia_stats* __restrict__ st)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    double a = 0.0, b = 0.0;
    for (int k = 0; k < n_blocks; ++k) {
        a += partial[(size_t)k * n_cells * 2 + 2 * c];
        b += partial[(size_t)k * n_cells * 2 + 2 * c + 1];
    }
    st[c].sum_dE = a;
    st[c].sum_dE2 = b;
}

}  // namespace ia
