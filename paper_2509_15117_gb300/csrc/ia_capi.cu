// ia_capi.cu -- kernels and the C ABI (include/ionatom.h) of the ion-atom trajectory engine.
//
// Kernels:
//   k_plain       one thread per trajectory; a warp runs until its longest trajectory ends.
//   k_sched       the fused persistent kernel (cooperative launch: all blocks resident).
//                 Lane phase: a lane that finishes stores its observables and, once `refill` lanes of
//                 its warp are idle, the warp claims that many queue positions with one atomic add.
//                 A trajectory that has used `budget` attempted steps is saved to a suspend record
//                 and its lane takes new work: lengths span 10^3 .. 10^7 steps (single passes against
//                 long-lived complexes).
//                 Tail phase: suspended trajectories run in group mode (G lanes each, about a third of
//                 the FP64 instructions per step of one lane, so ~2.5x lower latency). One block on each
//                 of the first `tail_sms` SMs is a tail worker from the start; every other warp joins
//                 once the queue is drained. The batch time is then the larger of the bulk work and
//                 the longest complex's latency, instead of their sum.
//   k_tail<G>     finishes records the fused kernel left (normally none).
//   k_fp64_fma    FP64 FMA throughput microbenchmark: the denominator of the integrator's roofline.
#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <cmath>
#include <mutex>
#include <map>
#include <new>
#include <utility>
#include <vector>
#include <cuda.h>
#include <cuda_runtime.h>

#include "ia_traj.cuh"
#include "ia_stats.cuh"
#include "ia_tangent.cuh"
#include "ia_adjoint.cuh"
#include "ia_sample.cuh"
#include "../../include/ionatom.h"

using namespace ia;

namespace {

// Work counters at the start of the scratch area; suspend-record ready flags and the records follow.
// The first group is cleared before every launch; the second holds the state a batch keeps between
// the launches of an ia_queue (suspend records and lane-mode carry records), cleared when a batch
// starts.
struct Counters {
    unsigned long long work;        // next queue position for the lane phase
    unsigned long long warps_done;  // warps that have left the lane phase
    unsigned long long errors;      // bounded waits that ran out (stays 0 in a healthy run)
    unsigned long long t_start;     // %globaltimer (ns) when the first block started
    unsigned long long t_lane_end;  // ... when the last warp left the lane phase
    unsigned long long t_end;       // ... when the last warp finished (fused and clean-up kernels)
    unsigned int sm_claim[192];     // blocks seen per SM, to give one block per reserved SM the tail role
    unsigned long long tc_taken;    // group-mode carry records of the previous part claimed so far
    // --- kept between the launches of one batch ---
    unsigned long long n_susp;      // suspend records taken by writers
    unsigned long long tail;        // next suspend record to resume
    unsigned long long carry_n[2];  // lane-mode carry records written into buffer 0 / 1
    unsigned long long tcarry_n[2]; // group-mode carry records written into buffer 0 / 1
};
constexpr size_t SCRATCH_HEAD = 1024;
static_assert(sizeof(Counters) <= SCRATCH_HEAD, "scratch head");
constexpr size_t PER_LAUNCH_BYTES = offsetof(Counters, n_susp);
// a test of the suspend-record overflow reads these two counters from a caller's scratch
static_assert(offsetof(Counters, errors) == 16 && offsetof(Counters, n_susp) == 824, "counter layout");
constexpr int MAX_TAIL_SMS = 192;

// The part of a batch one launch of the fused kernel works on. A single ia_launch is one part that
// is also the last: it starts queue positions 0..n-1 and finishes everything. The launches of an
// ia_queue split a batch into parts: each starts the next `count` queue positions after resuming,
// in lane mode, the trajectories the previous part left running; a part that is not the last ends as
// soon as its queue is exhausted, leaving its running lane-mode trajectories in carry records and its
// running group-mode trajectories in suspend records for the next part.
struct Part {
    long long first;                        // queue position of the part's first new trajectory
    long long count;                        // new trajectories of this part
    const Susp* carry_in;                   // lane-mode trajectories left by the previous part
    const unsigned long long* carry_in_n;   // how many (null: none)
    Susp* carry_out;                        // where this part leaves its running lane-mode trajectories
    unsigned long long* carry_out_n;
    long long carry_cap;                    // records per carry buffer
    const Susp* tcarry_in;                  // group-mode trajectories the previous part's tail was running:
    const unsigned long long* tcarry_in_n;  //   resumed by this part's tail before any suspend record
    Susp* tcarry_out;                       // where this part's tail leaves its running trajectories
    unsigned long long* tcarry_out_n;
    long long tcarry_cap;                   // records per group-mode carry buffer
    int last;                               // 1: finish every trajectory (no carry out)
    int lane_only;                          // 1: the lane phase alone (the autotuner's timing runs)
};

// Warps of a reserved SM's block that work on the tail by default: one per SM sub-partition, so that
// each tail warp has an FP64 unit to itself (the latency of one trajectory in group mode is its FP64
// instruction count per step); further warps of that block leave. At most MAX_TAIL_WARPS.
constexpr int TAIL_WARPS = 4;
constexpr int MAX_TAIL_WARPS = 8;

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__host__ __device__ constexpr size_t ready_bytes(long long cap) { return ((size_t)cap * 4u + 255u) & ~(size_t)255u; }

// Bounds of the waits in the fused kernel (each wait also sleeps, so these are seconds, not spins).
constexpr unsigned READY_SPIN_LIMIT = 1u << 22;  // record claimed but not yet published: ~0.3-1 s
constexpr unsigned IDLE_SPIN_LIMIT = 1u << 27;   // tail worker with nothing to do: minutes
constexpr unsigned CLAIM_BACKOFF = 64;           // attempts between claim polls of a partly busy warp


__global__ void __launch_bounds__(128) k_plain(const SysDev* __restrict__ tab, int n_sys, IcPtrs ic,
                                               ObsPtrs out, long long n)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int sid = ic.sys_id ? __ldg(ic.sys_id + i) : 0;
    if (sid < 0 || sid >= n_sys) {
        store_bad_sid(ic, out, tab, i);
        return;
    }
    const SysDev& P = tab[sid];
    Lane L;
    Final fin;
    if (!lane_init(P, ic, i, L, fin)) {
        store_result(P, ic, out, i, tally(L.s), fin, false);
        return;
    }
    while (lane_attempt(P, L, fin) == RUNNING) {
    }
    store_result(P, ic, out, i, tally(L.s), fin, true);
}

// Lane phase: each lane holds one trajectory at a time; idle lanes of a warp claim queue positions
// together with one atomic add; a trajectory that has used `budget` attempted steps is written to a
// suspend record (published by its ready flag) and the lane takes new work. With one_batch the warp
// claims once (32 positions) and returns when those are finished or suspended.
// The part's queue has n_virt = n_carry + part.count positions: positions below n_carry resume the
// carry records of the previous part, the others start trajectories part.first + (pos - n_carry) of
// the batch's queue. When the part is not the last, every lane leaves its trajectory in a carry record
// as soon as the queue is exhausted.
__device__ __forceinline__ void lane_phase(const SysDev* __restrict__ tab, int n_sys, const IcPtrs& ic,
                                           const ObsPtrs& out, const Part& part, long long n_virt,
                                           long long n_carry, Counters* __restrict__ ctr,
                                           unsigned* __restrict__ ready, Susp* __restrict__ susp, long long cap,
                                           int refill, int budget, bool one_batch = false)
{
    const int lane = threadIdx.x & 31;
    Lane L;
    Final fin;
    long long my = -1;     // trajectory index held by this lane, -1 = idle
    int sid = 0;
    bool can_suspend = false;
    bool drained = false;  // the queue has been seen empty by this warp
    const bool may_carry = !part.last;
    for (;;) {
        if (may_carry) {
            const bool exhausted = *(volatile unsigned long long*)&ctr->work >= (unsigned long long)n_virt;
            if (exhausted) {
                drained = true;
                if (my >= 0) {
                    const unsigned long long slot = atomicAdd(part.carry_out_n, 1ull);
                    if (slot < (unsigned long long)part.carry_cap) {
                        lane_suspend(L, my, sid, part.carry_out + slot);
                        my = -1;
                    }  // else (not expected: a buffer holds every lane of the grid) the lane finishes it
                }
            }
        }
        const unsigned idle = __ballot_sync(FULL, my < 0);
        const int n_idle = __popc(idle);
        if (!drained && (n_idle >= refill || n_idle == 32)) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(&ctr->work, (unsigned long long)n_idle);
            base = __shfl_sync(FULL, base, 0);
            // one_batch: a single claim of 32 positions, run to completion (a tail worker lending a hand)
            if (one_batch || base + (unsigned long long)n_idle >= (unsigned long long)n_virt) drained = true;
            if (my < 0) {
                const int rank = __popc(idle & ((1u << lane) - 1u));
                const unsigned long long pos = base + (unsigned long long)rank;
                if (pos < (unsigned long long)n_carry) {
                    lane_resume(part.carry_in + pos, L, my, sid);
                    can_suspend = budget > 0;
                } else if (pos < (unsigned long long)n_virt) {
                    const long long qp = part.first + (long long)pos - n_carry;
                    my = ic.order ? __ldg(ic.order + qp) : qp;
                    sid = ic.sys_id ? __ldg(ic.sys_id + my) : 0;
                    if (sid < 0 || sid >= n_sys) {
                        store_bad_sid(ic, out, tab, my);
                        my = -1;
                    } else if (!lane_init(tab[sid], ic, my, L, fin)) {
                        store_result(tab[sid], ic, out, my, tally(L.s), fin, false);
                        my = -1;
                    } else {
                        can_suspend = budget > 0;
                    }
                }
            }
        }
        if (__ballot_sync(FULL, my >= 0) == 0) {
            if (drained) break;
            continue;
        }
        if (my >= 0) {
            const SysDev& P = tab[sid];
            if (lane_attempt(P, L, fin) == FINISHED) {
                store_result(P, ic, out, my, tally(L.s), fin, true);
                my = -1;
            } else if (can_suspend && !L.s.retry && L.s.n_acc + L.s.n_rej >= budget) {
                const unsigned long long slot = atomicAdd(&ctr->n_susp, 1ull);
                if (slot < (unsigned long long)cap) {
                    lane_suspend(L, my, sid, susp + slot);
                    __threadfence();
                    atomicExch(ready + slot, 1u);
                    my = -1;
                } else {
                    can_suspend = false;  // no room: this lane finishes the trajectory itself
                }
            }
        }
    }
}

// Take the next published-or-being-published suspend record, if any (never beyond the writers).
__device__ __forceinline__ bool claim_record(Counters* ctr, long long cap, unsigned long long& k)
{
    unsigned long long t = *(volatile unsigned long long*)&ctr->tail;
    for (int it = 0; it < 64; ++it) {
        const unsigned long long ns = *(volatile unsigned long long*)&ctr->n_susp;
        const unsigned long long lim = ns < (unsigned long long)cap ? ns : (unsigned long long)cap;
        if (t >= lim) return false;
        const unsigned long long prev = atomicCAS(&ctr->tail, t, t + 1);
        if (prev == t) {
            k = t;
            return true;
        }
        t = prev;
    }
    return false;
}

// Tail phase (group mode): one suspended trajectory per group of G lanes until it ends.
// wait_ok: records may still be written by warps in the lane phase (all blocks co-resident,
// cooperative launch), so an idle group waits for them, boundedly; otherwise an idle group stops
// as soon as nothing is left to claim.
// help_n > 0: a worker with no trajectory and no record to take returns 1 while positions of the
// lane-phase queue (of length help_n) are left, so that its caller can run a batch of the lane phase
// (the reserved SMs then add to the bulk whenever the tail queue is empty); otherwise returns 0 when
// the tail is done.
// may_yield (a part of an ia_queue batch that is not the last): once every warp has left the lane
// phase, each group leaves its running trajectory in a new suspend record, published like the lane
// phase's, and the worker returns 0; the next part's tail resumes those records.
// The group-mode carry records of the previous part (part.tcarry_in, n_tc of them) are resumed before
// any suspend record: they hold the trajectories that part's tail was running, the oldest in the tail.
// A yield writes to part.tcarry_out, or, when that is full, appends a suspend record.
template <int G>
__device__ __forceinline__ int tail_phase(const SysDev* __restrict__ tab, const IcPtrs& ic, const ObsPtrs& out,
                                          Susp* __restrict__ susp, unsigned* __restrict__ ready,
                                          Counters* __restrict__ ctr, long long cap, bool wait_ok,
                                          unsigned long long total_warps, const Part& part, long long n_tc,
                                          long long help_n = 0, bool may_yield = false)
{
    constexpr int R = (N_COEF + G - 1) / G;  // coefficient rounds per lane
    const GroupLane<G> gl = group_lane<G>();
    double x = 0.0, v = 0.0, a1 = 0.0;
    Scal S;
    S.t = 0.0; S.h = 0.0; S.hmin = 0.0; S.phi0 = 0.0; S.rdot_prev = 0.0; S.t_first = 0.0; S.t_last = 0.0;
    S.n_acc = 0; S.n_rej = 0; S.n_bounce = 0; S.nofailed = true; S.retry = false;
    long long idx = -1;
    int sid = 0;
    bool active = false, drained = false;
    unsigned idle_spins = 0;
    unsigned claim_skip = 0;  // iterations without a claim attempt while other groups of the warp run
    bool yield_room = true;   // false once a yield found the record area full (warp-uniform)
    for (;;) {
        bool stop = false;
        if (may_yield && yield_room) {
            unsigned long long wd = 0;
            if ((threadIdx.x & 31) == 0) wd = *(volatile unsigned long long*)&ctr->warps_done;
            stop = __shfl_sync(FULL, wd, 0) >= total_warps;
        }
        if (stop) {
            unsigned long long slot = 0;
            int dest = 0;  // 1: group-mode carry record, 2: suspend record, 0: no room
            if (active && gl.c == 0) {
                slot = part.tcarry_out ? atomicAdd(part.tcarry_out_n, 1ull) : ~0ull;
                if (slot < (unsigned long long)part.tcarry_cap) {
                    dest = 1;
                } else {
                    slot = atomicAdd(&ctr->n_susp, 1ull);
                    dest = slot < (unsigned long long)cap ? 2 : 0;
                }
            }
            slot = __shfl_sync(FULL, slot, gl.base);
            dest = __shfl_sync(FULL, dest, gl.base);
            const bool room = active && dest != 0;
            if (room) {
                Susp* r = (dest == 1 ? part.tcarry_out : susp) + slot;
                if (gl.c < 6) {
                    r->x[gl.comp] = x;
                    r->v[gl.comp] = v;
                    r->a1[gl.comp] = a1;
                }
                if (gl.c == 0) {
                    r->t = S.t; r->h = S.h; r->phi0 = S.phi0; r->rdot_prev = S.rdot_prev;
                    r->t_first = S.t_first; r->t_last = S.t_last;
                    r->idx = idx; r->sid = sid;
                    r->n_acc = S.n_acc; r->n_rej = S.n_rej; r->n_bounce = S.n_bounce;
                    r->flags = (S.nofailed ? 1 : 0) | (S.retry ? 2 : 0);
                }
                __threadfence();
            }
            __syncwarp();
            if (room && dest == 2 && gl.c == 0) atomicExch(ready + slot, 1u);
            if (__any_sync(FULL, active && !room)) yield_room = false;  // no room (not expected): finish here
            if (room) active = false;
            drained = true;
            if (!__any_sync(FULL, active)) return 0;
        }
        const bool need = !active && !drained;
        bool poll = __any_sync(FULL, need);
        if (poll && claim_skip > 0 && __any_sync(FULL, active)) {
            // an idle group polls the record counters (global atomics, microseconds) only every
            // CLAIM_BACKOFF attempts while its warp still runs other trajectories
            --claim_skip;
            poll = false;
        }
        if (poll) {
            // the group's first lane claims; the claim is broadcast to the group
            int got = 0;
            unsigned long long k = 0;
            if (need && gl.c == 0 && n_tc > 0 &&
                *(volatile unsigned long long*)&ctr->tc_taken < (unsigned long long)n_tc) {
                k = atomicAdd(&ctr->tc_taken, 1ull);
                if (k < (unsigned long long)n_tc) got = 4;  // a trajectory the previous part's tail ran
            }
            if (need && gl.c == 0 && got == 0) {
                if (claim_record(ctr, cap, k)) {
                    got = 1;
                    unsigned spins = 0;
                    while (*(volatile const unsigned*)(ready + k) == 0u) {
                        if (++spins > READY_SPIN_LIMIT) {
                            atomicAdd(&ctr->errors, 1ull);
                            got = 0;
                            break;
                        }
                        __nanosleep(256);
                    }
                    __threadfence();
                } else {
                    const bool lane_work_left = wait_ok &&
                        *(volatile unsigned long long*)&ctr->warps_done < total_warps;
                    got = lane_work_left ? 2 : 3;  // 2: nothing yet, 3: nothing will come
                    if (got == 3 && claim_record(ctr, cap, k)) {
                        // a record published just before the last warp left the lane phase
                        got = 1;
                        unsigned spins = 0;
                        while (*(volatile const unsigned*)(ready + k) == 0u) {
                            if (++spins > READY_SPIN_LIMIT) {
                                atomicAdd(&ctr->errors, 1ull);
                                got = 0;
                                break;
                            }
                            __nanosleep(256);
                        }
                        __threadfence();
                    }
                }
            }
            got = __shfl_sync(FULL, got, gl.base);
            k = __shfl_sync(FULL, k, gl.base);
            if (!__any_sync(FULL, need && (got == 1 || got == 4))) claim_skip = CLAIM_BACKOFF;
            if (need) {
                if (got == 1 || got == 4) {
                    // written by another SM during this launch (or by the previous launch): read through L2
                    const Susp* r = (got == 4 ? part.tcarry_in : susp) + k;
                    x = __ldcg(&r->x[gl.comp]);
                    v = __ldcg(&r->v[gl.comp]);
                    a1 = __ldcg(&r->a1[gl.comp]);
                    S.t = __ldcg(&r->t); S.h = __ldcg(&r->h); S.phi0 = __ldcg(&r->phi0);
                    S.rdot_prev = __ldcg(&r->rdot_prev);
                    S.t_first = __ldcg(&r->t_first); S.t_last = __ldcg(&r->t_last);
                    S.n_acc = __ldcg(&r->n_acc); S.n_rej = __ldcg(&r->n_rej); S.n_bounce = __ldcg(&r->n_bounce);
                    const int flags = __ldcg(&r->flags);
                    S.nofailed = (flags & 1) != 0;
                    S.retry = (flags & 2) != 0;
                    S.hmin = hmin_at(S.t);
                    idx = __ldcg(&r->idx);
                    sid = __ldcg(&r->sid);
                    active = true;
                } else if (got == 3) {
                    drained = true;
                }
            }
        }
        if (!__any_sync(FULL, active)) {
            if (__all_sync(FULL, drained)) break;
            if (help_n > 0 && *(volatile unsigned long long*)&ctr->work < (unsigned long long)help_n) return 1;
            // nothing to run yet: wait for the lane phase to publish records
            if (++idle_spins > IDLE_SPIN_LIMIT) {
                if ((threadIdx.x & 31) == 0) atomicAdd(&ctr->errors, 1ull);
                break;  // a later launch of the tail kernel finishes what is left
            }
            __nanosleep(1000);
            continue;
        }

        const SysDev& P = tab[sid];
        uint32_t st = 0xffffffffu;
        if (active) st = attempt_begin(P, S);
        const double h = S.h, t = S.t;

        // step coefficients, spread over the group's lanes
        Coef K;
        K.h2 = h * h;
        double cv[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k = r * G + (gl.c < G ? gl.c : 0);
            const int kk = k < N_COEF ? k : N_COEF - 1;
            cv[r] = COEF_K[kk] * (COEF_H2[kk] ? K.h2 : h);
        }
        {
            double* kp = &K.c2;
#pragma unroll
            for (int k = 0; k < N_COEF; ++k) kp[k] = shfl(cv[k / G], gl.base + (k % G));
        }
        // rf phases of stages 2..6 (stage 7 shares stage 6's time), one per lane
        const double chsel = gl.c < 4 ? cv[0] : h;
        const double cl = cos(fma(P.Omega, t + chsel, S.phi0));
        const double cs2 = shfl(cl, gl.base + 0), cs3 = shfl(cl, gl.base + 1), cs4 = shfl(cl, gl.base + 2);
        const double cs5 = shfl(cl, gl.base + 3), cs67 = shfl(cl, gl.base + 4);

        const double kq = gl.comp >= 3 ? P.kq[gl.comp - 3] : 0.0;  // lanes 3-5: the ion's axis comp - 3
        const double ka = gl.comp >= 3 ? P.ka[gl.comp - 3] : 0.0;
        double r2, d3[3];
        const double a2 = accel_group<G>(P, gl, pos2(K, x, v), cs2, kq, ka, r2, d3);
        const double a3 = accel_group<G>(P, gl, pos3(K, x, v, a1), cs3, kq, ka, r2, d3);
        const double a4 = accel_group<G>(P, gl, pos4(K, x, v, a1, a2), cs4, kq, ka, r2, d3);
        const double a5 = accel_group<G>(P, gl, pos5(K, x, v, a1, a2, a3), cs5, kq, ka, r2, d3);
        const double a6 = accel_group<G>(P, gl, pos6(K, h, x, v, a1, a2, a3, a4), cs67, kq, ka, r2, d3);
        const double xn = pos7(K, h, x, v, a1, a3, a4, a5);
        double r2new, dn[3];
        const double a7 = accel_group<G>(P, gl, xn, cs67, kq, ka, r2new, dn);
        const double vn = vel_new(K, v, a1, a3, a4, a5, a6);

        bool okx, fx, okv, fv;
        float rx, rv;
        double aex, scx, aev, scv;
        err_check(P.rtol, P.atol_pos, x, xn, err_x(K, a1, a3, a4, a5, a6), okx, fx, rx, aex, scx);
        err_check(P.rtol, P.atol_vel, v, vn, err_v(K, a1, a3, a4, a5, a6, a7), okv, fv, rv, aev, scv);
        const bool real = gl.c < 6;
        const bool ok = !real || (okx && okv);
        const bool fi = !real || (fx && fv);
        const unsigned gmask = ((1u << G) - 1u) << gl.base;
        const bool accept = (__ballot_sync(FULL, !ok) & gmask) == 0;
        const bool finite = (__ballot_sync(FULL, !fi) & gmask) == 0;
        const ErrMeas em = group_err(gl.base, gl.c, real, rx, aex, scx, rv, aev, scv);
        // radial velocity sign at the step end: d . (v_a - v_i)
        const int j = gl.comp < 3 ? gl.comp : gl.comp - 3;
        const double wj = shfl(vn, gl.base + 3 + j) - shfl(vn, gl.base + j);
        const double w0 = shfl(wj, gl.base + 0), w1 = shfl(wj, gl.base + 1), w2 = shfl(wj, gl.base + 2);
        const double rd = fma(dn[0], w0, fma(dn[1], w1, dn[2] * w2));

        int res = 0;  // 0 running, 1 stopped, 2 exits in this step
        if (active) {
            if (st != 0xffffffffu) {
                res = 1;
            } else if (!finite) {
                res = 1;
                st = ST_NONFINITE;
            } else if (!accept) {
                st = on_reject(P, S, em);
                if (st != 0xffffffffu) res = 1;
            } else if (on_accept(P, S, rd, r2new)) {
                res = 2;
            } else {
                x = xn;
                v = vn;
                a1 = a7;
                on_commit(P, S, em);
            }
        }
        if (__any_sync(FULL, res != 0)) {
            Final fin;
            fin.t = S.t;
            fin.status = st;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                fin.xi[k] = shfl(x, gl.base + k);
                fin.xa[k] = shfl(x, gl.base + 3 + k);
                fin.vi[k] = shfl(v, gl.base + k);
                fin.va[k] = shfl(v, gl.base + 3 + k);
            }
            if (__any_sync(FULL, res == 2)) {
                StepData D;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    D.xi[k] = fin.xi[k]; D.xa[k] = fin.xa[k]; D.vi[k] = fin.vi[k]; D.va[k] = fin.va[k];
                    D.a1i[k] = shfl(a1, gl.base + k); D.a1a[k] = shfl(a1, gl.base + 3 + k);
                    D.a3i[k] = shfl(a3, gl.base + k); D.a3a[k] = shfl(a3, gl.base + 3 + k);
                    D.a4i[k] = shfl(a4, gl.base + k); D.a4a[k] = shfl(a4, gl.base + 3 + k);
                    D.a5i[k] = shfl(a5, gl.base + k); D.a5a[k] = shfl(a5, gl.base + 3 + k);
                    D.a6i[k] = shfl(a6, gl.base + k); D.a6a[k] = shfl(a6, gl.base + 3 + k);
                    D.a7i[k] = shfl(a7, gl.base + k); D.a7a[k] = shfl(a7, gl.base + 3 + k);
                    D.xni[k] = shfl(xn, gl.base + k); D.xna[k] = shfl(xn, gl.base + 3 + k);
                    D.vni[k] = shfl(vn, gl.base + k); D.vna[k] = shfl(vn, gl.base + 3 + k);
                }
                D.h = h;
                D.t = t;
                if (res == 2 && gl.c == 0) finish_exit(P, D, r2new, fin);
            }
            if (res != 0) {
                if (gl.c == 0) store_result(P, ic, out, idx, tally(S), fin, true);
                active = false;
            }
        }
    }
    return 0;
}

// ---------------------------------------------------------------------------------------------
// Paired tail phase. An FP64 instruction occupies a sub-partition's FP64 unit for its whole issue
// time whatever the number of active lanes, so the latency of one trajectory in group mode is its
// FP64 instruction count per step. Here the two warps of a pair -- on two sub-partitions, each with
// its own FP64 unit -- advance the same five trajectories together: the chain warp runs the serial
// part of every stage (the last term of the stage position and the force), the helper warp the rest
// (step coefficients, rf phases, ion trap coefficients, position partial sums, new velocity, error
// estimate, accept/reject decision, exit epilogue and result). Every value is formed with the
// expressions of the other layouts, so the results are bit-identical to them. The warps exchange
// data through shared memory, lane by lane: each lane reads only the slots of its counterpart lane,
// which publishes them with a per-lane sequence counter (release / acquire at block scope); every wait
// is bounded, and when one runs out both warps leave the tail phase and count an error (the clean-up
// kernel cannot resume a trajectory a pair held, so the host sees the error count).

struct __align__(16) PairShared {
    double a[8][32];    // chain -> helper: a_l of stage l
    double xp[8][32];   // helper -> chain: partial positions of stages 5..7 (slots 5..7)
    double kc[8][32];   // helper -> chain: ka_j + kq_j cos(Omega t_l + phi0) of stage l (ion lanes)
    double xn[32];      // chain -> helper: X7, the position at the step end
    double dn[3][32];   // chain -> helper: separation at X7
    double r2n[32];     // chain -> helper: its square
    double vn[32];      // helper -> chain: velocity at the step end
    double rd[32];      // helper -> chain: d . (v_a - v_i) at the step end
    long long ck[32];   // helper -> chain: claimed suspend record of the lane's group
    float errf[32];     // helper -> chain: FP32 error ratio of the lane's group
    double err_ae[32];  // helper -> chain: |e| and sc of the component that sets it
    double err_sc[32];
    int dec[32];        // helper -> chain: bit 0 accept, bit 1 finite
    int claim[32];      // helper -> chain: claim result of the lane's group (0..3, as in tail_phase)
    unsigned long long seq_h[32], seq_c[32];  // posts of the helper and of the chain warp, per lane
};

constexpr unsigned PAIR_SPIN_LIMIT = 1u << 26;  // a partner that stopped answering: seconds

__device__ __forceinline__ void st_release_cta(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.release.cta.shared::cta.u64 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "l"(v)
                 : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_cta(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.cta.shared::cta.u64 %0, [%1];"
                 : "=l"(v)
                 : "r"((unsigned)__cvta_generic_to_shared(p))
                 : "memory");
    return v;
}
// Each lane of the consumer reads only the slots its own lane of the producer wrote, so every lane
// synchronises with its counterpart directly: the producer lane writes its data, then its counter
// (release); the consumer lane waits for its counterpart's counter (acquire), then reads.
__device__ __forceinline__ void pair_post(unsigned long long* seq, unsigned long long& n)
{
    ++n;
    st_release_cta(seq + (threadIdx.x & 31), n);
}
// Consumer: false (in every lane) when a counterpart did not post within the bound.
__device__ __forceinline__ bool pair_wait(const unsigned long long* seq, unsigned long long& n)
{
    ++n;
    const unsigned long long* mine = seq + (threadIdx.x & 31);
    unsigned spins = 0;
    bool ok = true;
    while (ld_acquire_cta(mine) < n) {
        if (++spins > PAIR_SPIN_LIMIT) {
            ok = false;
            break;
        }
        if (spins > 256) __nanosleep(64);
    }
    return __all_sync(FULL, ok);
}

// Interaction part of a stage acceleration (everything of accel_group<6> but the ion trap term):
// returns gm d_j; the acceleration is fma(kc, p, returned value) with kc the trap coefficient.
__device__ __forceinline__ double chain_force(const SysDev& P, const GroupLane<6>& gl, double p, double& r2out,
                                              double d3[3])
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
    const int c = gl.c;
    const double ua = c == 0 ? s2 : (c == 1 ? P.ci8 : P.ca8);
    const double ub = c == 0 ? s : s2;
    const double uc = c == 0 ? 0.0 : (c == 1 ? -P.ci4 : -P.ca4);
    const double u = fma(ua, ub, uc);
    const double gm = shfl(u, gl.base + 0) * shfl(u, gl.base + (gl.comp < 3 ? 1 : 2));
    r2out = r2;
    d3[0] = d0;
    d3[1] = d1;
    d3[2] = d2;
    return gm * dj;
}

__device__ __forceinline__ void tail_phase_pair(const SysDev* __restrict__ tab, const IcPtrs& ic, const ObsPtrs& out,
                                                const Susp* __restrict__ susp, const unsigned* __restrict__ ready,
                                                Counters* __restrict__ ctr, long long cap,
                                                unsigned long long total_warps, PairShared* sh, bool helper)
{
    constexpr int G = 6;
    constexpr int R = (N_COEF + G - 1) / G;
    const GroupLane<G> gl = group_lane<G>();
    const int lane = threadIdx.x & 31;
    // idle groups keep a harmless state (unit separation) so that their arithmetic stays on the fast path
    double x = gl.comp < 3 ? 0.0 : 1.0, v = 0.0, a1 = 0.0;
    Scal S;
    S.t = 0.0; S.h = 1.0; S.hmin = 0.0; S.phi0 = 0.0; S.rdot_prev = 0.0; S.t_first = 0.0; S.t_last = 0.0;
    S.n_acc = 0; S.n_rej = 0; S.n_bounce = 0; S.nofailed = true; S.retry = false;
    long long idx = -1;
    int sid = 0;
    bool active = false, drained = false, broken = false;
    unsigned idle_spins = 0, claim_skip = 0;
    unsigned long long nh = 0, nc = 0;  // posts seen / made in each direction
    for (;;) {
        const bool need = !active && !drained;
        bool poll = __any_sync(FULL, need);
        if (poll && claim_skip > 0 && __any_sync(FULL, active)) {
            --claim_skip;
            poll = false;
        }
        if (poll) {
            // the helper claims for the idle groups and publishes; the chain warp acknowledges
            int got = 0;
            unsigned long long k = 0;
            if (helper) {
                if (need && gl.c == 0) {
                    if (claim_record(ctr, cap, k)) {
                        got = 1;
                        unsigned spins = 0;
                        while (*(volatile const unsigned*)(ready + k) == 0u) {
                            if (++spins > READY_SPIN_LIMIT) {
                                atomicAdd(&ctr->errors, 1ull);
                                got = 0;
                                break;
                            }
                            __nanosleep(256);
                        }
                        __threadfence();
                    } else {
                        const bool lane_work_left =
                            *(volatile unsigned long long*)&ctr->warps_done < total_warps;
                        got = lane_work_left ? 2 : 3;
                        if (got == 3 && claim_record(ctr, cap, k)) {
                            got = 1;
                            unsigned spins = 0;
                            while (*(volatile const unsigned*)(ready + k) == 0u) {
                                if (++spins > READY_SPIN_LIMIT) {
                                    atomicAdd(&ctr->errors, 1ull);
                                    got = 0;
                                    break;
                                }
                                __nanosleep(256);
                            }
                            __threadfence();
                        }
                    }
                }
                got = __shfl_sync(FULL, got, gl.base);
                k = __shfl_sync(FULL, k, gl.base);
                sh->claim[lane] = got;
                sh->ck[lane] = (long long)k;
                pair_post(sh->seq_h, nh);
                if (!pair_wait(sh->seq_c, nc)) broken = true;
            } else {
                if (!pair_wait(sh->seq_h, nh)) {
                    broken = true;
                } else {
                    got = sh->claim[lane];
                    k = (unsigned long long)sh->ck[lane];
                    pair_post(sh->seq_c, nc);
                }
            }
            if (broken) break;
            if (!__any_sync(FULL, need && got == 1)) claim_skip = CLAIM_BACKOFF;
            if (need) {
                if (got == 1) {
                    const Susp* r = susp + k;
                    x = __ldcg(&r->x[gl.comp]);
                    v = __ldcg(&r->v[gl.comp]);
                    a1 = __ldcg(&r->a1[gl.comp]);
                    S.t = __ldcg(&r->t); S.h = __ldcg(&r->h); S.phi0 = __ldcg(&r->phi0);
                    S.rdot_prev = __ldcg(&r->rdot_prev);
                    S.t_first = __ldcg(&r->t_first); S.t_last = __ldcg(&r->t_last);
                    S.n_acc = __ldcg(&r->n_acc); S.n_rej = __ldcg(&r->n_rej); S.n_bounce = __ldcg(&r->n_bounce);
                    const int flags = __ldcg(&r->flags);
                    S.nofailed = (flags & 1) != 0;
                    S.retry = (flags & 2) != 0;
                    S.hmin = hmin_at(S.t);
                    idx = __ldcg(&r->idx);
                    sid = __ldcg(&r->sid);
                    active = true;
                } else if (got == 3) {
                    drained = true;
                }
            }
        }
        if (!__any_sync(FULL, active)) {
            if (__all_sync(FULL, drained)) break;
            if (++idle_spins > IDLE_SPIN_LIMIT) {
                if (lane == 0 && helper) atomicAdd(&ctr->errors, 1ull);
                break;
            }
            __nanosleep(1000);
            continue;
        }

        const SysDev& P = tab[sid];
        uint32_t st = 0xffffffffu;
        if (active) st = attempt_begin(P, S);
        const double h = S.h, t = S.t;
        // values both warps hold at the end of the attempt
        double xn, vn, a7, r2new, rd;
        double a3 = 0.0, a4 = 0.0, a5 = 0.0, a6 = 0.0;  // helper: kept for the exit epilogue
        ErrMeas em;
        bool accept, finite;
        if (helper) {
            // rf phases first: the chain warp needs the ion trap coefficient of stage 2 soonest.
            // Lanes 0-3 form t + c_s h (s = 2..5; the products of the other layouts), lane 4 t + h.
            const int cidx = gl.c < 4 ? gl.c : 0;
            const double chsel = gl.c < 4 ? COEF_K[cidx] * h : h;
            const double cl = cos(fma(P.Omega, t + chsel, S.phi0));
            const double cs2 = shfl(cl, gl.base + 0), cs3 = shfl(cl, gl.base + 1), cs4 = shfl(cl, gl.base + 2);
            const double cs5 = shfl(cl, gl.base + 3), cs67 = shfl(cl, gl.base + 4);
            const double kqj = gl.comp < 3 ? P.kq[gl.comp] : 0.0;
            const double kaj = gl.comp < 3 ? P.ka[gl.comp] : 0.0;
            sh->kc[2][lane] = fma(kqj, cs2, kaj);
            sh->kc[3][lane] = fma(kqj, cs3, kaj);
            sh->kc[4][lane] = fma(kqj, cs4, kaj);
            sh->kc[5][lane] = fma(kqj, cs5, kaj);
            sh->kc[6][lane] = fma(kqj, cs67, kaj);
            pair_post(sh->seq_h, nh);                                     // H1: trap coefficients
            Coef K;
            K.h2 = h * h;
            double cv[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int kk = r * G + gl.c < N_COEF ? r * G + gl.c : N_COEF - 1;
                cv[r] = COEF_K[kk] * (COEF_H2[kk] ? K.h2 : h);
            }
            {
                double* kp = &K.c2;
#pragma unroll
                for (int k = 0; k < N_COEF; ++k) kp[k] = shfl(cv[k / G], gl.base + (k % G));
            }
            double p5 = fma(K.w51, a1, fma(K.c5, v, x));
            double p6 = fma(K.w61, a1, fma(h, v, x));
            double p7 = fma(K.w71, a1, fma(h, v, x));
            double vacc = fma(K.b1, a1, v);
            double ex = K.f1 * a1, ev = K.e1 * a1;
            bool ok = pair_wait(sh->seq_c, nc);                           // C1: a2
            const double a2 = sh->a[2][lane];
            p5 = fma(K.w52, a2, p5);
            sh->xp[5][lane] = p5;
            pair_post(sh->seq_h, nh);                                     // H2: stage 5 partial position
            p6 = fma(K.w62, a2, p6);
            ok = pair_wait(sh->seq_c, nc) && ok;                          // C2: a3
            a3 = sh->a[3][lane];
            p6 = fma(K.w63, a3, p6);
            sh->xp[6][lane] = p6;
            pair_post(sh->seq_h, nh);                                     // H3: stage 6 partial position
            p7 = fma(K.w73, a3, p7);
            vacc = fma(K.b3, a3, vacc);
            ex = fma(K.f3, a3, ex);
            ev = fma(K.e3, a3, ev);
            ok = pair_wait(sh->seq_c, nc) && ok;                          // C3: a4
            a4 = sh->a[4][lane];
            p7 = fma(K.w74, a4, p7);
            sh->xp[7][lane] = p7;
            pair_post(sh->seq_h, nh);                                     // H4: step-end partial position
            vacc = fma(K.b4, a4, vacc);
            ex = fma(K.f4, a4, ex);
            ev = fma(K.e4, a4, ev);
            ok = pair_wait(sh->seq_c, nc) && ok;                          // C4: a5, a6 and the step-end position
            a5 = sh->a[5][lane];
            a6 = sh->a[6][lane];
            xn = sh->xn[lane];
            vacc = fma(K.b5, a5, vacc);
            ex = fma(K.f5, a5, ex);
            ev = fma(K.e5, a5, ev);
            vn = fma(K.b6, a6, vacc);
            ex = fma(K.f6, a6, ex);
            ev = fma(K.e6, a6, ev);
            bool okx, fx, okv, fv;
            float rx, rv;
            double aex, scx, aev, scv;
            err_check(P.rtol, P.atol_pos, x, xn, ex, okx, fx, rx, aex, scx);  // while the chain warp forms a7
            const int j = gl.comp < 3 ? gl.comp : gl.comp - 3;
            const double wj = shfl(vn, gl.base + 3 + j) - shfl(vn, gl.base + j);
            const double w0 = shfl(wj, gl.base + 0), w1 = shfl(wj, gl.base + 1), w2 = shfl(wj, gl.base + 2);
            ok = pair_wait(sh->seq_c, nc) && ok;                          // C5: a7 and the step end
            a7 = sh->a[7][lane];
            r2new = sh->r2n[lane];
            const double dn0 = sh->dn[0][lane], dn1 = sh->dn[1][lane], dn2 = sh->dn[2][lane];
            ev = fma(K.e7, a7, ev);
            err_check(P.rtol, P.atol_vel, v, vn, ev, okv, fv, rv, aev, scv);
            const bool real = gl.c < 6;
            const bool okk = !real || (okx && okv);
            const bool fi = !real || (fx && fv);
            const unsigned gmask = ((1u << G) - 1u) << gl.base;
            accept = (__ballot_sync(FULL, !okk) & gmask) == 0;
            finite = (__ballot_sync(FULL, !fi) & gmask) == 0;
            em = group_err(gl.base, gl.c, real, rx, aex, scx, rv, aev, scv);
            rd = fma(dn0, w0, fma(dn1, w1, dn2 * w2));
            sh->vn[lane] = vn;
            sh->rd[lane] = rd;
            sh->errf[lane] = em.f;
            sh->err_ae[lane] = em.ae;
            sh->err_sc[lane] = em.sc;
            sh->dec[lane] = (accept ? 1 : 0) | (finite ? 2 : 0);
            pair_post(sh->seq_h, nh);                                     // H5: the decision
            if (!ok) broken = true;
        } else {
            // stage 2, and the step coefficients of this warp's own stage positions (the products
            // and the positions of the other layouts, bit for bit) while the helper forms the rf phases
            const double X2 = fma(COEF_K[0] * h, v, x);
            double r2, d3[3];
            const double q2 = chain_force(P, gl, X2, r2, d3);
            const double h2 = h * h;
            const double X3 = fma(COEF_K[4] * h2, a1, fma(COEF_K[1] * h, v, x));     // w31, c3
            const double p4 = fma(COEF_K[5] * h2, a1, fma(COEF_K[2] * h, v, x));     // w41, c4
            const double w42 = COEF_K[6] * h2, w53 = COEF_K[9] * h2;
            const double w64 = COEF_K[13] * h2, w75 = COEF_K[17] * h2;
            bool ok = pair_wait(sh->seq_h, nh);                           // H1
            const bool ion = gl.comp < 3;
            const double kc2 = ion ? sh->kc[2][lane] : 0.0, kc3 = ion ? sh->kc[3][lane] : 0.0;
            const double kc4 = ion ? sh->kc[4][lane] : 0.0, kc5 = ion ? sh->kc[5][lane] : 0.0;
            const double kc6 = ion ? sh->kc[6][lane] : 0.0;
            const double a2 = fma(kc2, X2, q2);
            sh->a[2][lane] = a2;
            pair_post(sh->seq_c, nc);                                     // C1
            // stage 3
            const double b3 = fma(kc3, X3, chain_force(P, gl, X3, r2, d3));
            sh->a[3][lane] = b3;
            pair_post(sh->seq_c, nc);                                     // C2
            // stage 4
            const double X4 = fma(w42, a2, p4);
            const double b4 = fma(kc4, X4, chain_force(P, gl, X4, r2, d3));
            sh->a[4][lane] = b4;
            pair_post(sh->seq_c, nc);                                     // C3
            // stage 5
            ok = pair_wait(sh->seq_h, nh) && ok;                          // H2
            const double X5 = fma(w53, b3, sh->xp[5][lane]);
            const double b5 = fma(kc5, X5, chain_force(P, gl, X5, r2, d3));
            // stage 6
            ok = pair_wait(sh->seq_h, nh) && ok;                          // H3
            const double X6 = fma(w64, b4, sh->xp[6][lane]);
            const double b6 = fma(kc6, X6, chain_force(P, gl, X6, r2, d3));
            // stage 7: the step end
            ok = pair_wait(sh->seq_h, nh) && ok;                          // H4
            xn = fma(w75, b5, sh->xp[7][lane]);
            sh->a[5][lane] = b5;
            sh->a[6][lane] = b6;
            sh->xn[lane] = xn;
            pair_post(sh->seq_c, nc);                                     // C4
            double dn[3];
            a7 = fma(kc6, xn, chain_force(P, gl, xn, r2new, dn));
            sh->a[7][lane] = a7;
            sh->r2n[lane] = r2new;
            sh->dn[0][lane] = dn[0];
            sh->dn[1][lane] = dn[1];
            sh->dn[2][lane] = dn[2];
            pair_post(sh->seq_c, nc);                                     // C5
            ok = pair_wait(sh->seq_h, nh) && ok;                          // H5: the decision
            vn = sh->vn[lane];
            rd = sh->rd[lane];
            em.f = sh->errf[lane];
            em.ae = sh->err_ae[lane];
            em.sc = sh->err_sc[lane];
            const int dec = sh->dec[lane];
            accept = (dec & 1) != 0;
            finite = (dec & 2) != 0;
            if (!ok) broken = true;
        }
        if (broken) break;

        int res = 0;  // 0 running, 1 stopped, 2 exits in this step
        if (active) {
            if (st != 0xffffffffu) {
                res = 1;
            } else if (!finite) {
                res = 1;
                st = ST_NONFINITE;
            } else if (!accept) {
                st = on_reject(P, S, em);
                if (st != 0xffffffffu) res = 1;
            } else if (on_accept(P, S, rd, r2new)) {
                res = 2;
            } else {
                x = xn;
                v = vn;
                a1 = a7;
                on_commit(P, S, em);
            }
        }
        if (__any_sync(FULL, res != 0)) {
            if (helper) {
                Final fin;
                fin.t = S.t;
                fin.status = st;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    fin.xi[k] = shfl(x, gl.base + k);
                    fin.xa[k] = shfl(x, gl.base + 3 + k);
                    fin.vi[k] = shfl(v, gl.base + k);
                    fin.va[k] = shfl(v, gl.base + 3 + k);
                }
                if (__any_sync(FULL, res == 2)) {
                    StepData D;
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        D.xi[k] = fin.xi[k]; D.xa[k] = fin.xa[k]; D.vi[k] = fin.vi[k]; D.va[k] = fin.va[k];
                        D.a1i[k] = shfl(a1, gl.base + k); D.a1a[k] = shfl(a1, gl.base + 3 + k);
                        D.a3i[k] = shfl(a3, gl.base + k); D.a3a[k] = shfl(a3, gl.base + 3 + k);
                        D.a4i[k] = shfl(a4, gl.base + k); D.a4a[k] = shfl(a4, gl.base + 3 + k);
                        D.a5i[k] = shfl(a5, gl.base + k); D.a5a[k] = shfl(a5, gl.base + 3 + k);
                        D.a6i[k] = shfl(a6, gl.base + k); D.a6a[k] = shfl(a6, gl.base + 3 + k);
                        D.a7i[k] = shfl(a7, gl.base + k); D.a7a[k] = shfl(a7, gl.base + 3 + k);
                        D.xni[k] = shfl(xn, gl.base + k); D.xna[k] = shfl(xn, gl.base + 3 + k);
                        D.vni[k] = shfl(vn, gl.base + k); D.vna[k] = shfl(vn, gl.base + 3 + k);
                    }
                    D.h = h;
                    D.t = t;
                    if (res == 2 && gl.c == 0) finish_exit(P, D, r2new, fin);
                }
                if (res != 0 && gl.c == 0) store_result(P, ic, out, idx, tally(S), fin, true);
            }
            if (res != 0) active = false;
        }
    }
    if (broken && lane == 0) atomicAdd(&ctr->errors, 1ull);
}

// Fused persistent kernel. Blocks on SMs with id < tail_sms (one block per such SM) are tail
// workers from the start, so long-lived complexes run in group mode on sub-partitions of their own
// while the rest of the GPU works through the queue; every other block runs the lane phase and then
// joins the tail phase. In a part of a batch that is not the last, the lane-phase warps leave once the
// part's queue is exhausted (their running trajectories go to carry records) and the tail workers
// then leave theirs in suspend records: the next part continues both.
template <int BLOCK, int MINB, int G>
__global__ void __launch_bounds__(BLOCK, MINB) k_sched(const SysDev* __restrict__ tab, int n_sys, IcPtrs ic,
                                                       ObsPtrs out, Part part, Counters* __restrict__ ctr,
                                                       unsigned* __restrict__ ready, Susp* __restrict__ susp,
                                                       long long cap, int refill, int budget, int tail_sms,
                                                       int wait_ok, int pair, int tail_warps)
{
    __shared__ int role;  // 0 lane phase first, 1 tail worker, 2 surplus block on a reserved SM
    __shared__ PairShared pair_sh[G == 6 ? BLOCK / 64 : 1];
    if (threadIdx.x == 0) {
        for (int k = 0; k < (G == 6 ? BLOCK / 64 : 1); ++k)
            for (int l = 0; l < 32; ++l) pair_sh[k].seq_h[l] = pair_sh[k].seq_c[l] = 0ull;
        atomicCAS(&ctr->t_start, 0ull, global_ns());
        int r = 0;
        if (budget > 0 && tail_sms > 0) {
            unsigned smid;
            asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
            if (smid < (unsigned)tail_sms && smid < (unsigned)MAX_TAIL_SMS)
                r = (atomicAdd(&ctr->sm_claim[smid], 1u) == 0u) ? 1 : 2;
        }
        role = r;
    }
    __syncthreads();
    // a reserved SM's block keeps tail_warps tail warps; its other warps leave (pairs need all of them)
    const int r = (role == 1 && !(G == 6 && pair && wait_ok) && (int)(threadIdx.x >> 5) >= tail_warps) ? 2 : role;
    const unsigned long long total_warps = (unsigned long long)gridDim.x * (BLOCK / 32);
    // carry records written by the previous part's launch (complete before this launch started)
    long long n_carry = 0, n_tc = 0;
    if (part.carry_in_n) {
        const unsigned long long c = *part.carry_in_n;
        n_carry = c < (unsigned long long)part.carry_cap ? (long long)c : part.carry_cap;
    }
    if (part.tcarry_in_n) {
        const unsigned long long c = *part.tcarry_in_n;
        n_tc = c < (unsigned long long)part.tcarry_cap ? (long long)c : part.tcarry_cap;
    }
    const long long n_virt = n_carry + part.count;
    if (r == 0) lane_phase(tab, n_sys, ic, out, part, n_virt, n_carry, ctr, ready, susp, cap, refill, budget);
    if ((threadIdx.x & 31) == 0) {
        __threadfence();
        if (atomicAdd(&ctr->warps_done, 1ull) + 1ull == total_warps) atomicMax(&ctr->t_lane_end, global_ns());
    }
    if (part.lane_only) {
        // timing runs of the lane phase: trajectories past the budget stay in their suspend records
    } else if (!part.last) {
        // only the reserved-SM workers stay: they work on the tail (and lend a hand to the lane phase)
        // until every lane-phase warp has left, then leave their trajectories for the next part
        if (r == 1 && budget > 0)
            while (tail_phase<G>(tab, ic, out, susp, ready, ctr, cap, wait_ok != 0, total_warps, part, n_tc, n_virt,
                                 true) == 1)
                lane_phase(tab, n_sys, ic, out, part, n_virt, n_carry, ctr, ready, susp, cap, refill, budget, true);
    } else if (G == 6 && r == 1 && pair && wait_ok) {
        // dedicated tail block: warps 2p and 2p+1 form pair p (chain and helper warp)
        const int w = threadIdx.x >> 5;
        tail_phase_pair(tab, ic, out, susp, ready, ctr, cap, total_warps, &pair_sh[G == 6 ? (w >> 1) : 0],
                        (w & 1) != 0);
    } else if (r != 2 && budget > 0) {
        // a reserved-SM worker that finds the tail queue empty runs batches of the lane phase meanwhile
        const long long help_n = r == 1 ? n_virt : 0;
        while (tail_phase<G>(tab, ic, out, susp, ready, ctr, cap, wait_ok != 0, total_warps, part, n_tc, help_n) == 1)
            lane_phase(tab, n_sys, ic, out, part, n_virt, n_carry, ctr, ready, susp, cap, refill, budget, true);
    }
    if ((threadIdx.x & 31) == 0) atomicMax(&ctr->t_end, global_ns());
}

// Finishes suspend records left by k_sched (normally none: its workers drain them).
template <int G>
__global__ void __launch_bounds__(128) k_tail(const SysDev* __restrict__ tab, IcPtrs ic, ObsPtrs out,
                                              Susp* __restrict__ susp, unsigned* __restrict__ ready,
                                              Counters* __restrict__ ctr, long long cap, Part part)
{
    long long n_tc = 0;
    if (part.tcarry_in_n) {
        const unsigned long long c = *part.tcarry_in_n;
        n_tc = c < (unsigned long long)part.tcarry_cap ? (long long)c : part.tcarry_cap;
    }
    tail_phase<G>(tab, ic, out, susp, ready, ctr, cap, false, 0ull, part, n_tc);
    if ((threadIdx.x & 31) == 0) atomicMax(&ctr->t_end, global_ns());
}


// Tangent kernel: one trajectory per warp (lane = direction x 6 + component); see ia_tangent.cuh.
__global__ void __launch_bounds__(128) k_tangent(const SysDev* __restrict__ tab, int n_sys, IcPtrs ic, ObsPtrs out,
                                                 long long n, TanIn tin, TanOut tout,
                                                 unsigned long long* __restrict__ work)
{
    const TLane tl = tlane();
    const int lane = threadIdx.x & 31;
    const int yi = tl.comp < 3 ? tl.comp : tl.comp + 3;  // position index in y
    const int yv = yi + 3;                              // velocity index
    const int dsel = tl.dir - 1;                         // tangent direction of this lane, -1: primal
    const bool used = tl.dir <= tin.ndir;
    for (;;) {
        unsigned long long claim = 0;
        if (lane == 0) claim = atomicAdd(work, 1ull);
        claim = __shfl_sync(FULL, claim, 0);
        if (claim >= (unsigned long long)n) break;
        const long long i = (long long)claim;
        const int sid = ic.sys_id ? __ldg(ic.sys_id + i) : 0;
        if (sid < 0 || sid >= n_sys) {
            if (lane == 0) store_bad_sid(ic, out, tab, i);
            if (lane < tin.ndir) {
                const long long o = (long long)lane * tout.ld + i;
                tout.d_theta[o] = 0.0; tout.d_dp[o] = 0.0; tout.d_dE[o] = 0.0; tout.d_tf[o] = 0.0;
            }
            if (tout.ftle && lane == 0) tout.ftle[i] = 0.0;
            continue;
        }
        const SysDev& P = tab[sid];
        double x, v;
        if (tl.dir == 0) {
            x = __ldg(ic.y0 + yi * ic.ld + i);
            v = __ldg(ic.y0 + yv * ic.ld + i);
        } else if (used) {
            x = __ldg(tin.dy0 + ((long long)dsel * 12 + yi) * tin.ld + i);
            v = __ldg(tin.dy0 + ((long long)dsel * 12 + yv) * tin.ld + i);
        } else {
            x = 0.0;
            v = 0.0;
        }
        Scal S;
        S.phi0 = __ldg(ic.phi0 + i);
        // the primal state must be usable (same test as lane mode)
        bool okl = tl.dir != 0 || (is_finite(x) && is_finite(v));
        const bool ok_state = __all_sync(FULL, okl) && is_finite(S.phi0);
        double xs[6], vs[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            xs[k] = shfl(x, k);
            vs[k] = shfl(v, k);
        }
        double dd0 = xs[3] - xs[0], dd1 = xs[4] - xs[1], dd2 = xs[5] - xs[2];
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
            if (lane < tin.ndir) {
                const long long o = (long long)lane * tout.ld + i;
                tout.d_theta[o] = 0.0; tout.d_dp[o] = 0.0; tout.d_dE[o] = 0.0; tout.d_tf[o] = 0.0;
            }
            if (tout.ftle && lane == 0) tout.ftle[i] = 0.0;
            continue;
        }
        // per-lane constants
        const double kq = tl.comp < 3 ? P.kq[tl.comp] : 0.0;
        const double ka = tl.comp < 3 ? P.ka[tl.comp] : 0.0;
        const double coef = tl.comp < 3 ? P.neg_inv_mi : P.inv_ma;
        double dq_lane = (tl.dir > 0 && used && tl.comp < 3) ? tin.dq[dsel][tl.comp] : 0.0;
        double dkq = P.kq_per_q * dq_lane;
        int scale_e = 0;
        // initial acceleration (FSAL) of primal and tangents, and the initial step of ode45
        double r2, d3[3];
        double a1 = tan_accel(P, tl, x, cos(S.phi0), kq, ka, dkq, coef, r2, d3);
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
        // |Y0| of direction 1 in the FTLE norm
        double ynorm0 = 0.0;
        {
            const double sx = x * P.inv_len, sv = v * P.inv_vel;
            double part = fma(sx, sx, sv * sv);
            double acc = 0.0;
#pragma unroll
            for (int k = 0; k < 6; ++k) acc += __shfl_sync(FULL, part, 6 + k);
            ynorm0 = sqrt(acc);
        }
        Final fin;
        fin.s_exit = -1.0;
        int res = 0;
        uint32_t st = 0xffffffffu;
        double h = 0.0, t = 0.0;
        double a3 = 0.0, a4 = 0.0, a5 = 0.0, a6 = 0.0, a7 = 0.0, xn = 0.0, vn = 0.0, r2new = 0.0, dn[3] = {0, 0, 0};
        Coef K;
        for (;;) {
            st = attempt_begin(P, S);
            if (st != 0xffffffffu) {
                res = 1;
                break;
            }
            h = S.h;
            t = S.t;
            K.h2 = h * h;
            // coefficients: lane k computes coefficient k (and k + 30 for lanes 0..3)
            const int k0 = lane < N_COEF ? lane : N_COEF - 1;
            const double cv0 = COEF_K[k0] * (COEF_H2[k0] ? K.h2 : h);
            const int k1 = lane + 32 < N_COEF ? lane + 32 : N_COEF - 1;
            const double cv1 = COEF_K[k1] * (COEF_H2[k1] ? K.h2 : h);
            {
                double* kp = &K.c2;
#pragma unroll
                for (int k = 0; k < N_COEF; ++k) kp[k] = k < 32 ? shfl(cv0, k) : shfl(cv1, k - 32);
            }
            const double chsel = lane < 4 ? cv0 : h;
            const double cl = cos(fma(P.Omega, t + chsel, S.phi0));
            const double cs2 = shfl(cl, 0), cs3 = shfl(cl, 1), cs4 = shfl(cl, 2), cs5 = shfl(cl, 3), cs67 = shfl(cl, 4);
            const double a2 = tan_accel(P, tl, pos2(K, x, v), cs2, kq, ka, dkq, coef, r2, d3);
            a3 = tan_accel(P, tl, pos3(K, x, v, a1), cs3, kq, ka, dkq, coef, r2, d3);
            a4 = tan_accel(P, tl, pos4(K, x, v, a1, a2), cs4, kq, ka, dkq, coef, r2, d3);
            a5 = tan_accel(P, tl, pos5(K, x, v, a1, a2, a3), cs5, kq, ka, dkq, coef, r2, d3);
            a6 = tan_accel(P, tl, pos6(K, h, x, v, a1, a2, a3, a4), cs67, kq, ka, dkq, coef, r2, d3);
            xn = pos7(K, h, x, v, a1, a3, a4, a5);
            a7 = tan_accel(P, tl, xn, cs67, kq, ka, dkq, coef, r2new, dn);
            vn = vel_new(K, v, a1, a3, a4, a5, a6);
            // error test on the primal lanes
            bool okx, fx, okv, fv;
            float rx, rv;
            double aex, scx, aev, scv;
            err_check(P.rtol, P.atol_pos, x, xn, err_x(K, a1, a3, a4, a5, a6), okx, fx, rx, aex, scx);
            err_check(P.rtol, P.atol_vel, v, vn, err_v(K, a1, a3, a4, a5, a6, a7), okv, fv, rv, aev, scv);
            const bool prim = tl.dir == 0;
            const bool accept = (__ballot_sync(FULL, prim && !(okx && okv)) & 0x3fu) == 0;
            const bool finite = (__ballot_sync(FULL, prim && !(fx && fv)) & 0x3fu) == 0;
            const ErrMeas em = group_err(0, lane, prim, rx, aex, scx, rv, aev, scv);
            const int jj = tl.comp < 3 ? tl.comp : tl.comp - 3;
            const double wj = shfl(vn, 3 + jj) - shfl(vn, jj);
            const double w0 = shfl(wj, 0), w1 = shfl(wj, 1), w2 = shfl(wj, 2);
            const double rd = fma(dn[0], w0, fma(dn[1], w1, dn[2] * w2));
            if (!finite) {
                st = ST_NONFINITE;
                res = 1;
                break;
            }
            if (!accept) {
                st = on_reject(P, S, em);
                if (st != 0xffffffffu) {
                    res = 1;
                    break;
                }
                continue;
            }
            if (on_accept(P, S, rd, r2new)) {
                res = 2;
                break;
            }
            x = xn;
            v = vn;
            a1 = a7;
            on_commit(P, S, em);
            // exact power-of-two rescaling of a tangent direction that left [2^-256, 2^256]
            int me = max_exp3(x, v, a1);
#pragma unroll
            for (int k = 1; k < 6; ++k) me = max(me, __shfl_sync(FULL, me, tl.base + ((tl.comp + k) % 6)));
            if (tl.dir > 0 && (me > 1023 + 256 || (me > 0 && me < 1023 - 256))) {
                const int sh = me > 1023 + 256 ? -256 : 256;
                const double f = sh < 0 ? 0x1p-256 : 0x1p+256;
                x *= f; v *= f; a1 *= f; dq_lane *= f; dkq *= f;
                scale_e -= sh;
            }
        }
        // final state of primal (lane 0 owns the epilogue) and of each tangent direction
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            fin.xi[k] = shfl(x, k); fin.xa[k] = shfl(x, 3 + k);
            fin.vi[k] = shfl(v, k); fin.va[k] = shfl(v, 3 + k);
        }
        fin.t = S.t;
        fin.status = st;
        double yfx = x, yfv = v;  // this lane's final component (stops: the current state)
        double dtf_lane = 0.0;
        if (res == 2) {
            StepData D;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                D.xi[k] = fin.xi[k]; D.xa[k] = fin.xa[k]; D.vi[k] = fin.vi[k]; D.va[k] = fin.va[k];
                D.a1i[k] = shfl(a1, k); D.a1a[k] = shfl(a1, 3 + k);
                D.a3i[k] = shfl(a3, k); D.a3a[k] = shfl(a3, 3 + k);
                D.a4i[k] = shfl(a4, k); D.a4a[k] = shfl(a4, 3 + k);
                D.a5i[k] = shfl(a5, k); D.a5a[k] = shfl(a5, 3 + k);
                D.a6i[k] = shfl(a6, k); D.a6a[k] = shfl(a6, 3 + k);
                D.a7i[k] = shfl(a7, k); D.a7a[k] = shfl(a7, 3 + k);
                D.xni[k] = shfl(xn, k); D.xna[k] = shfl(xn, 3 + k);
                D.vni[k] = shfl(vn, k); D.vna[k] = shfl(vn, 3 + k);
            }
            D.h = h;
            D.t = t;
            if (lane == 0) finish_exit(P, D, r2new, fin);
            fin.t = __shfl_sync(FULL, fin.t, 0);
            fin.s_exit = __shfl_sync(FULL, fin.s_exit, 0);
            fin.status = __shfl_sync(FULL, fin.status, 0);
            if (fin.s_exit >= 0.0) {
                // continuous extension at s* for every lane, and its s-derivative
                const double s = fin.s_exit, s2 = s * s, h2 = h * h, sh = s * h;
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
                const double qx = fma(px6, a6, fma(px5, a5, fma(px4, a4, fma(px3, a3, px1 * a1))));
                const double ux = fma(b7, a7, fma(b6, a6, fma(b5, a5, fma(b4, a4, fma(b3, a3, b1 * a1)))));
                yfx = fma(h2, qx, fma(sh, v, x));
                yfv = fma(h, ux, v);
                // d/ds of the extension (primal lanes use it)
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
                const double dqx = s * (dp1 * a1 + dp3 * a3 + dp4 * a4 + dp5 * a5 + dp6 * a6);
                const double dux = db1 * a1 + s * (db3 * a3 + db4 * a4 + db5 * a5 + db6 * a6 + db7 * a7);
                const double ysx = fma(h, v, h2 * dqx);  // dx/ds
                const double ysv = h * dux;              // dv/ds
                // primal separation and its s-derivative; this direction's separation tangent
                const int j = tl.comp < 3 ? tl.comp : tl.comp - 3;
                const double dprim = shfl(yfx, 3 + j) - shfl(yfx, j);
                const double dsep = shfl(ysx, 3 + j) - shfl(ysx, j);
                const double dtan = shfl(yfx, tl.base + 3 + j) - shfl(yfx, tl.base + j);
                const double num = shfl(dprim, 0) * shfl(dtan, tl.base + 0) + shfl(dprim, 1) * shfl(dtan, tl.base + 1) +
                                   shfl(dprim, 2) * shfl(dtan, tl.base + 2);
                const double den = shfl(dprim, 0) * shfl(dsep, 0) + shfl(dprim, 1) * shfl(dsep, 1) +
                                   shfl(dprim, 2) * shfl(dsep, 2);
                const double dsstar = tl.dir == 0 ? 0.0 : -num / den;
                const double pysx = shfl(ysx, tl.comp), pysv = shfl(ysv, tl.comp);
                if (tl.dir > 0) {
                    yfx = fma(pysx, dsstar, yfx);
                    yfv = fma(pysv, dsstar, yfv);
                }
                dtf_lane = h * dsstar;
            } else {
                yfx = xn;  // ends outside r0 without a crossing: the step end is final
                yfv = vn;
            }
        }
        // primal observables (lane 0) and the derivatives of direction k (lane 6k)
        double yf[12], dyf[12];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int pi = k < 3 ? k : k + 3;
            yf[pi] = shfl(yfx, k);
            yf[pi + 3] = shfl(yfv, k);
            dyf[pi] = shfl(yfx, tl.base + k);
            dyf[pi + 3] = shfl(yfv, tl.base + k);
        }
        if (lane == 0) store_result(P, ic, out, i, tally(S), fin, true);
        if (tl.dir > 0 && used && tl.comp == 0) {
            double y0v[12], dy0v[12], dqv[3];
            const double sc = ldexp(1.0, -scale_e);
            for (int c = 0; c < 12; ++c) {
                y0v[c] = __ldg(ic.y0 + c * ic.ld + i);
                dy0v[c] = sc * __ldg(tin.dy0 + ((long long)dsel * 12 + c) * tin.ld + i);
            }
            for (int c = 0; c < 3; ++c) dqv[c] = sc * tin.dq[dsel][c];
            double dth, ddp, dde;
            obs_derivs(P, S.phi0, y0v, yf, fin.t, dy0v, dyf, dtf_lane, dqv, dth, ddp, dde);
            const long long o = (long long)dsel * tout.ld + i;
            tout.d_theta[o] = ldexp(dth, scale_e);
            tout.d_dp[o] = ldexp(ddp, scale_e);
            tout.d_dE[o] = ldexp(dde, scale_e);
            tout.d_tf[o] = ldexp(dtf_lane, scale_e);
            if (tout.dy_final)
                for (int c = 0; c < 12; ++c) tout.dy_final[((long long)dsel * 12 + c) * tout.ld + i] = ldexp(dyf[c], scale_e);
            if (tout.ftle && dsel == 0) {
                double acc = 0.0;
                for (int c = 0; c < 12; ++c) {
                    const bool vel = (c % 6) >= 3;
                    const double z = dyf[c] * (vel ? P.inv_vel : P.inv_len);
                    acc = fma(z, z, acc);
                }
                const double lf = 0.5 * log(acc) + (double)scale_e * 0.69314718055994531;
                tout.ftle[i] = fin.t > 0.0 && ynorm0 > 0.0 ? (lf - log(ynorm0)) / fin.t : 0.0;
            }
        }
    }
}

__global__ void k_fp64_fma(double* out, int iters, double a, double b)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double x0 = 1.0 + 1e-9 * (double)g, x1 = x0 + 1e-3, x2 = x0 + 2e-3, x3 = x0 + 3e-3;
    double x4 = x0 + 4e-3, x5 = x0 + 5e-3, x6 = x0 + 6e-3, x7 = x0 + 7e-3;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    out[g] = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
}

__global__ void k_rcp_check(const double* x, double* y, long long n)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = rcp_nr(x[i]);
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// Host side

struct ia_system {
    int device;
    int n_sys;
    SysDev* d_tab;
    void* d_scratch;          // library-owned scratch of persistent launches (grown on demand)
    size_t scratch_bytes;
    void* d_stats_scratch;    // block partials of the statistics reduction
    size_t stats_scratch_bytes;
    void* d_adj_scratch;      // checkpoints and step buffers of adjoint launches (grown on demand)
    size_t adj_scratch_bytes;
    int num_sms;
};

struct ia_graph {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

struct ia_queue {
    ia_system* sys;
    int64_t n;                // trajectories of the batch
    ia_launch_opts opts;      // launch options fixed at creation
    void* scratch;            // counters, ready flags, suspend records, two carry buffers
    size_t bytes;
    size_t carry_off;         // byte offset of the carry buffers
    long long carry_cap;      // records per lane-mode carry buffer (one per lane of the grid)
    long long tcarry_cap;     // records per group-mode carry buffer
    int64_t started;          // queue positions handed to parts so far
    int64_t parts;            // parts launched since creation or the last reset
    const void* bound[18];    // the arrays of the batch, fixed by its first part
};

namespace {

bool aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

// SM count of the current device, which must be an sm_103 GPU.
int sample_device(int* sms)
{
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return IA_ERR_NO_DEVICE;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return IA_ERR_NO_DEVICE;
    return (major == 10 && minor == 3 && *sms > 0) ? IA_OK : IA_ERR_NO_DEVICE;
}

// Stability of one trap axis. With tau = (Omega t + phi0)/2 the ion's equation of motion along axis j
// (Eq. 1) is x'' + (a_j + 2 q_j cos 2 tau) x = 0, Mathieu's equation, whose solutions stay bounded when
// the trace of the monodromy matrix over one rf period (tau from 0 to pi) lies within [-2, 2]
// (Floquet). The trace is that of the two fundamental solutions, integrated with classical RK4 over
// 4096 steps (error ~1e-12 for |a|, |q| <= 1). An axis with a = q = 0 has trace exactly 2 (free
// motion: bounded velocity) and is accepted, as is any trace within 1e-8 of +-2.
constexpr int kMathieuSteps = 4096;

double mathieu_trace(double a, double q)
{
    static const std::vector<double> cos2 = [] {
        std::vector<double> c(2 * kMathieuSteps + 1);
        const double pi = 3.14159265358979323846;
        for (int i = 0; i <= 2 * kMathieuSteps; ++i)
            c[i] = std::cos(2.0 * (pi * (double)i / (2.0 * kMathieuSteps)));
        return c;
    }();
    const double h = 3.14159265358979323846 / kMathieuSteps;
    double tr = 0.0;
    for (int sol = 0; sol < 2; ++sol) {
        double x = sol == 0 ? 1.0 : 0.0, v = sol == 0 ? 0.0 : 1.0;
        for (int i = 0; i < kMathieuSteps; ++i) {
            const double w0 = a + 2.0 * q * cos2[2 * i];
            const double wm = a + 2.0 * q * cos2[2 * i + 1];
            const double w1 = a + 2.0 * q * cos2[2 * i + 2];
            const double k1x = v, k1v = -w0 * x;
            const double k2x = v + 0.5 * h * k1v, k2v = -wm * (x + 0.5 * h * k1x);
            const double k3x = v + 0.5 * h * k2v, k3v = -wm * (x + 0.5 * h * k2x);
            const double k4x = v + h * k3v, k4v = -w1 * (x + h * k3x);
            x += h / 6.0 * (k1x + 2.0 * k2x + 2.0 * k3x + k4x);
            v += h / 6.0 * (k1v + 2.0 * k2v + 2.0 * k3v + k4v);
        }
        tr += sol == 0 ? x : v;
    }
    return tr;
}

bool mathieu_stable(double a, double q)
{
    const double tr = mathieu_trace(a, q);
    return std::isfinite(tr) && std::fabs(tr) <= 2.0 + 1e-8;
}

bool valid_desc(const ia_system_desc& d)
{
    auto pos = [](double x) { return std::isfinite(x) && x > 0.0; };
    if (!pos(d.m_ion) || !pos(d.m_atom) || !pos(d.Omega) || !pos(d.r0) || !pos(d.t_max)) return false;
    if (!pos(d.rtol) || !pos(d.atol_pos) || !pos(d.atol_vel) || !pos(d.h_max)) return false;
    if (!std::isfinite(d.alpha) || d.alpha < 0.0) return false;
    if (d.alpha > 0.0 && !pos(d.De)) return false;
    for (int j = 0; j < 3; ++j)
        if (!std::isfinite(d.a[j]) || !std::isfinite(d.q[j])) return false;
    if (d.rf_sign != 1 && d.rf_sign != -1) return false;
    if (d.reserved != 0 || d.max_attempts <= 0 || d.max_attempts > 0x7fffffffLL) return false;
    for (int j = 0; j < 3; ++j)
        if (std::fabs(d.a[j]) > 16.0 || std::fabs(d.q[j]) > 16.0) return false;
    return true;
}

// Every axis of every row Mathieu-stable; each distinct (a, |q|) pair is integrated once (the sign of
// q shifts the rf phase by half a period and leaves the stability unchanged).
bool stable_traps(const ia_system_desc* desc, int n_sys)
{
    std::map<std::pair<double, double>, bool> seen;
    for (int k = 0; k < n_sys; ++k)
        for (int j = 0; j < 3; ++j) {
            const std::pair<double, double> key(desc[k].a[j], std::fabs(desc[k].q[j]));
            auto it = seen.find(key);
            if (it == seen.end()) it = seen.emplace(key, mathieu_stable(key.first, key.second)).first;
            if (!it->second) return false;
        }
    return true;
}

// Constants of one system (text after Eq. 1: C4 = alpha/2, C8 = C4^2/(4 De); Eq. 1's trap term).
SysDev derive(const ia_system_desc& d)
{
    SysDev P;
    std::memset(&P, 0, sizeof(P));
    const double C4 = 0.5 * d.alpha;
    const double C8 = C4 > 0.0 ? C4 * C4 / (4.0 * d.De) : 0.0;
    P.inv_mi = 1.0 / d.m_ion;
    P.inv_ma = 1.0 / d.m_atom;
    P.neg_inv_mi = -P.inv_mi;
    P.c8x8 = 8.0 * C8;
    P.c4x4 = 4.0 * C4;
    P.ci8 = P.c8x8 * P.neg_inv_mi;
    P.ci4 = P.c4x4 * P.neg_inv_mi;
    P.ca8 = P.c8x8 * P.inv_ma;
    P.ca4 = P.c4x4 * P.inv_ma;
    P.Omega = d.Omega;
    const double W2 = d.Omega * d.Omega;
    for (int j = 0; j < 3; ++j) {
        P.ka[j] = -(W2 / 4.0) * d.a[j];
        P.kq[j] = -(W2 / 4.0) * (2.0 * (double)d.rf_sign * d.q[j]);
        P.ua[j] = (d.m_ion * W2 / 8.0) * d.a[j];
        P.uq[j] = (d.m_ion * W2 / 8.0) * (2.0 * (double)d.rf_sign * d.q[j]);
    }
    P.m_i = d.m_ion;
    P.m_a = d.m_atom;
    P.r0sq = d.r0 * d.r0;
    P.t_max = d.t_max;
    P.h_max = d.h_max;
    P.rtol = d.rtol;
    P.atol_pos = d.atol_pos;
    P.atol_vel = d.atol_vel;
    P.thr_pos = d.atol_pos / d.rtol;
    P.thr_vel = d.atol_vel / d.rtol;
    P.hinit_den = 0.8 * std::pow(d.rtol, 0.2);
    P.max_attempts = (long long)d.max_attempts;
    P.kq_per_q = -(W2 / 4.0) * (2.0 * (double)d.rf_sign);
    P.uq_per_q = (d.m_ion * W2 / 8.0) * (2.0 * (double)d.rf_sign);
    const double mu = d.m_ion * d.m_atom / (d.m_ion + d.m_atom);
    P.inv_len = C4 > 0.0 ? 1.0 / std::pow(C4 / (2.0 * d.De), 0.25) : 1.0;
    P.inv_vel = C4 > 0.0 ? 1.0 / std::sqrt(2.0 * d.De / mu) : 1.0;
    return P;
}

struct Resolved {
    ia_launch_opts o;
    long long cap;  // suspend records
    size_t bytes;   // scratch bytes
};

constexpr int DEFAULT_BUDGET = 131072;
constexpr int DEFAULT_TAIL_SMS = 32;

int resolve(int64_t n, const ia_launch_opts* opts, Resolved& r)
{
    std::memset(&r.o, 0, sizeof(r.o));
    if (opts) r.o = *opts;
    ia_launch_opts& o = r.o;
    if (o.kernel != IA_KERNEL_PLAIN && o.kernel != IA_KERNEL_PERSISTENT) return IA_ERR_INVALID_ARG;
    if (o.tail_sms == 0) o.tail_sms = DEFAULT_TAIL_SMS;
    if (o.tail_sms < -1 || o.tail_sms > MAX_TAIL_SMS) return IA_ERR_INVALID_ARG;
    if (o.refill == 0) o.refill = 1;
    if (o.refill < 1 || o.refill > 32) return IA_ERR_INVALID_ARG;
    if (o.grid < 0 || o.blocks_per_sm < 0 || o.tail_blocks_per_sm < 0) return IA_ERR_INVALID_ARG;
    if (o.tail_pair < -1 || o.tail_pair > 1 || o.tail_warps < 0 || o.tail_warps > MAX_TAIL_WARPS)
        return IA_ERR_INVALID_ARG;
    if (o.slice_budget == 0) o.slice_budget = DEFAULT_BUDGET;
    if (o.slice_budget < -1) return IA_ERR_INVALID_ARG;
    if (o.tail_group == 0) o.tail_group = 6;
    if (o.tail_group != 6 && o.tail_group != 8) return IA_ERR_INVALID_ARG;
    if (o.tail_blocks_per_sm == 0) o.tail_blocks_per_sm = 1;
    if (o.tail_blocks_per_sm > 16) return IA_ERR_INVALID_ARG;
    if (o.regs_variant != 0 && o.regs_variant != 1 && o.regs_variant != 3) return IA_ERR_INVALID_ARG;
    if (o.suspend_capacity < 0) return IA_ERR_INVALID_ARG;
    r.cap = 0;
    if (o.kernel == IA_KERNEL_PERSISTENT && o.slice_budget > 0) {
        long long cap = o.suspend_capacity;
        if (cap == 0) {
            cap = n / 32;
            if (cap < 4096) cap = 4096;
            if (cap > n) cap = n;
        }
        r.cap = cap;
    }
    r.bytes = SCRATCH_HEAD + ready_bytes(r.cap) + (size_t)r.cap * sizeof(Susp);
    return IA_OK;
}

// Builds of the fused persistent kernel: (block, minimum resident blocks per SM, tail group size).
// The register cap of 3 x 128-thread blocks per SM (168 registers) is the only one that does not spill.
const void* sched_fn(int block, int minb, int g)
{
    if (block == 64) return (const void*)k_sched<64, 1, 6>;
    if (block == 256) return (const void*)k_sched<256, 1, 6>;
    if (minb == 3) return (const void*)k_sched<128, 3, 6>;
    if (g == 8) return (const void*)k_sched<128, 1, 8>;
    return (const void*)k_sched<128, 1, 6>;
}

// Launch configuration of the fused kernel for resolved options on the system's device.
struct SchedCfg {
    const void* fn;
    int block, grid, resident, budget, wait_ok, tail_sms, pair, refill, tail_warps;
};

int sched_config(const ia_system* sys, const Resolved& r, SchedCfg& c)
{
    const ia_launch_opts& o = r.o;
    c.block = o.block == 0 ? 128 : o.block;
    if (c.block != 64 && c.block != 128 && c.block != 256) return IA_ERR_INVALID_ARG;
    if (o.regs_variant != 0 && o.regs_variant != 1 && !(o.regs_variant == 3 && c.block == 128))
        return IA_ERR_INVALID_ARG;
    if (o.tail_group == 8 && (c.block != 128 || o.regs_variant == 3)) return IA_ERR_INVALID_ARG;
    const int minb = o.regs_variant == 3 ? 3 : 1;
    c.fn = sched_fn(c.block, minb, o.tail_group);
    c.resident = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.resident, c.fn, c.block, 0) != cudaSuccess ||
        c.resident <= 0)
        return IA_ERR_CUDA;
    c.grid = o.grid;
    if (c.grid == 0) {
        int nb = c.resident;
        if (o.blocks_per_sm > 0 && o.blocks_per_sm < nb) nb = o.blocks_per_sm;
        c.grid = nb * sys->num_sms;
    }
    // Waiting for records across blocks needs every block resident: a cooperative launch gives that.
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, sys->device);
    c.budget = o.slice_budget > 0 ? o.slice_budget : 0;
    c.wait_ok = (c.budget > 0 && coop && c.grid <= c.resident * sys->num_sms) ? 1 : 0;
    c.tail_sms = (c.wait_ok && o.tail_sms > 0) ? o.tail_sms : 0;
    if (c.tail_sms > sys->num_sms / 2) c.tail_sms = sys->num_sms / 2;
    c.pair = (o.tail_group != 8 && o.tail_pair == 1) ? 1 : 0;
    c.refill = o.refill;
    c.tail_warps = o.tail_warps == 0 ? std::min(TAIL_WARPS, c.block / 32) : o.tail_warps;
    if (c.tail_warps < 1 || c.tail_warps > MAX_TAIL_WARPS || c.tail_warps > c.block / 32) return IA_ERR_INVALID_ARG;
    return IA_OK;
}

// One launch of the fused kernel on `part` (plus, for the last part of a batch, the clean-up tail
// kernel). The scratch counters the launch needs at zero are cleared by the caller.
int launch_sched(const ia_system* sys, const SchedCfg& c, const Resolved& r, IcPtrs icp, ObsPtrs op, Part part,
                 char* scratch, cudaStream_t st)
{
    Counters* ctr = reinterpret_cast<Counters*>(scratch);
    unsigned* ready = reinterpret_cast<unsigned*>(scratch + SCRATCH_HEAD);
    Susp* susp = reinterpret_cast<Susp*>(scratch + SCRATCH_HEAD + ready_bytes(r.cap));
    long long cap = r.cap;
    int refill = c.refill, budget = c.budget, tail_sms = c.tail_sms, wait_ok = c.wait_ok, pair = c.pair;
    int tail_warps = c.tail_warps;
    int n_sys = sys->n_sys;
    const SysDev* tab = sys->d_tab;
    void* args[] = {(void*)&tab, (void*)&n_sys, (void*)&icp, (void*)&op, (void*)&part, (void*)&ctr, (void*)&ready,
                    (void*)&susp, (void*)&cap, (void*)&refill, (void*)&budget, (void*)&tail_sms, (void*)&wait_ok,
                    (void*)&pair, (void*)&tail_warps};
    cudaError_t e;
    if (wait_ok)
        e = cudaLaunchCooperativeKernel(c.fn, dim3(c.grid), dim3(c.block), args, 0, st);
    else
        e = cudaLaunchKernel(c.fn, dim3(c.grid), dim3(c.block), args, 0, st);
    if (e != cudaSuccess) return IA_ERR_CUDA;
    if (budget > 0 && part.last && !part.lane_only) {
        // records the fused kernel could not finish (normally none)
        const int tgrid = r.o.tail_blocks_per_sm * sys->num_sms;
        if (r.o.tail_group == 8)
            k_tail<8><<<tgrid, 128, 0, st>>>(tab, icp, op, susp, ready, ctr, cap, part);
        else
            k_tail<6><<<tgrid, 128, 0, st>>>(tab, icp, op, susp, ready, ctr, cap, part);
        if (cudaGetLastError() != cudaSuccess) return IA_ERR_CUDA;
    }
    return IA_OK;
}

// The whole batch as one part (ia_launch, ia_graph_create, ia_launch_static).
Part single_part(long long n)
{
    Part p;
    std::memset(&p, 0, sizeof(p));
    p.first = 0;
    p.count = n;
    p.last = 1;
    return p;
}

}  // namespace

extern "C" {

int ia_version(void) { return 200; }

const char* ia_error_string(int code)
{
    switch (code) {
        case IA_OK: return "ok";
        case IA_ERR_INVALID_ARG: return "invalid argument";
        case IA_ERR_BAD_DESC: return "system descriptor fails validation";
        case IA_ERR_CUDA: return "CUDA runtime error";
        case IA_ERR_ALIGNMENT: return "device pointer not 8-byte aligned (scratch: 256-byte)";
        case IA_ERR_NO_DEVICE: return "no usable CUDA device (sm_103 required)";
        case IA_ERR_TOO_LARGE: return "size beyond a documented limit";
        default: return "unknown error code";
    }
}

int ia_system_create(const ia_system_desc* desc, int32_t n_sys, ia_system** out)
{
    if (!desc || !out || n_sys < 1 || n_sys > 65536) return IA_ERR_INVALID_ARG;
    for (int k = 0; k < n_sys; ++k)
        if (!valid_desc(desc[k])) return IA_ERR_BAD_DESC;
    if (!stable_traps(desc, n_sys)) return IA_ERR_BAD_DESC;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return IA_ERR_NO_DEVICE;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return IA_ERR_NO_DEVICE;
    if (prop.major != 10 || prop.minor != 3) return IA_ERR_NO_DEVICE;
    SysDev* host = new (std::nothrow) SysDev[n_sys];
    if (!host) return IA_ERR_INVALID_ARG;
    for (int k = 0; k < n_sys; ++k) host[k] = derive(desc[k]);
    ia_system* s = new (std::nothrow) ia_system;
    if (!s) {
        delete[] host;
        return IA_ERR_INVALID_ARG;
    }
    s->device = dev;
    s->n_sys = n_sys;
    s->d_tab = nullptr;
    s->d_scratch = nullptr;
    s->scratch_bytes = 0;
    s->d_stats_scratch = nullptr;
    s->stats_scratch_bytes = 0;
    s->d_adj_scratch = nullptr;
    s->adj_scratch_bytes = 0;
    s->num_sms = prop.multiProcessorCount;
    if (cudaMalloc(&s->d_tab, sizeof(SysDev) * (size_t)n_sys) != cudaSuccess ||
        cudaMemcpy(s->d_tab, host, sizeof(SysDev) * (size_t)n_sys, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(s->d_tab);
        delete s;
        delete[] host;
        return IA_ERR_CUDA;
    }
    delete[] host;
    *out = s;
    return IA_OK;
}

int ia_system_destroy(ia_system* sys)
{
    if (!sys) return IA_OK;
    cudaFree(sys->d_tab);
    cudaFree(sys->d_scratch);
    cudaFree(sys->d_stats_scratch);
    cudaFree(sys->d_adj_scratch);
    delete sys;
    return IA_OK;
}

int ia_system_count(const ia_system* sys)
{
    if (!sys) return IA_ERR_INVALID_ARG;
    return sys->n_sys;
}

int64_t ia_scratch_bytes(int64_t n, const ia_launch_opts* opts)
{
    if (n < 0) return IA_ERR_INVALID_ARG;
    Resolved r;
    int rc = resolve(n, opts, r);
    if (rc != IA_OK) return rc;
    return (int64_t)r.bytes;
}

int ia_reserve(ia_system* sys, int64_t n, const ia_launch_opts* opts)
{
    if (!sys || n < 0) return IA_ERR_INVALID_ARG;
    Resolved r;
    int rc = resolve(n, opts, r);
    if (rc != IA_OK) return rc;
    if (r.bytes <= sys->scratch_bytes) return IA_OK;
    void* p = nullptr;
    if (cudaMalloc(&p, r.bytes) != cudaSuccess) return IA_ERR_CUDA;
    cudaFree(sys->d_scratch);
    sys->d_scratch = p;
    sys->scratch_bytes = r.bytes;
    return IA_OK;
}

int ia_launch(ia_system* sys, const ia_ic_soa* ic, int64_t n, const ia_obs_soa* out,
              const ia_launch_opts* opts, void* stream)
{
    if (!sys || !ic || !out || n < 0) return IA_ERR_INVALID_ARG;
    if (n == 0) return IA_OK;
    if (!ic->y0 || !ic->phi0 || ic->ld < n) return IA_ERR_INVALID_ARG;
    if (!out->theta_s || !out->dp || !out->dE_ion || !out->t_final || !out->t_first_bounce ||
        !out->t_last_bounce || !out->n_bounce || !out->status || !out->n_steps || !out->n_rej)
        return IA_ERR_INVALID_ARG;
    if (out->y_final && out->ld < n) return IA_ERR_INVALID_ARG;
    if (!aligned8(ic->y0) || !aligned8(ic->phi0) || !aligned8(out->theta_s) || !aligned8(out->dp) ||
        !aligned8(out->dE_ion) || !aligned8(out->t_final) || !aligned8(out->t_first_bounce) ||
        !aligned8(out->t_last_bounce) || (out->y_final && !aligned8(out->y_final)))
        return IA_ERR_ALIGNMENT;
    Resolved r;
    int rc = resolve(n, opts, r);
    if (rc != IA_OK) return rc;
    const ia_launch_opts& o = r.o;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

    IcPtrs icp{ic->y0, ic->phi0, ic->sys_id, reinterpret_cast<const long long*>(ic->order), (long long)ic->ld};
    if (ic->order && !aligned8(ic->order)) return IA_ERR_ALIGNMENT;
    ObsPtrs op{out->theta_s, out->dp, out->dE_ion, out->t_final, out->t_first_bounce, out->t_last_bounce,
               out->n_bounce, out->status, out->n_steps, out->n_rej, out->y_final,
               (long long)(out->y_final ? out->ld : 0)};

    if (o.kernel == IA_KERNEL_PLAIN) {
        if (o.block != 0 && o.block != 128) return IA_ERR_INVALID_ARG;
        const int block = 128;
        const long long blocks = (n + block - 1) / block;
        if (blocks > 0x7fffffffLL) return IA_ERR_TOO_LARGE;
        k_plain<<<(unsigned)blocks, block, 0, st>>>(sys->d_tab, sys->n_sys, icp, op, (long long)n);
        return cudaGetLastError() == cudaSuccess ? IA_OK : IA_ERR_CUDA;
    }

    SchedCfg cfg;
    rc = sched_config(sys, r, cfg);
    if (rc != IA_OK) return rc;
    // scratch: caller's, else the system's own (grown here if needed: not inside a stream capture)
    char* scratch = nullptr;
    if (o.scratch) {
        if ((size_t)o.scratch_bytes < r.bytes) return IA_ERR_TOO_LARGE;
        if ((reinterpret_cast<uintptr_t>(o.scratch) & 255u) != 0) return IA_ERR_ALIGNMENT;
        scratch = static_cast<char*>(o.scratch);
    } else {
        rc = ia_reserve(sys, n, opts);
        if (rc != IA_OK) return rc;
        scratch = static_cast<char*>(sys->d_scratch);
    }
    if (cudaMemsetAsync(scratch, 0, SCRATCH_HEAD + ready_bytes(r.cap), st) != cudaSuccess) return IA_ERR_CUDA;
    return launch_sched(sys, cfg, r, icp, op, single_part((long long)n), scratch, st);
}

// ---------------------------------------------------------------------------------------------
// A batch integrated over several launches (ia_queue)

int ia_queue_create(ia_system* sys, int64_t n, const ia_launch_opts* opts, ia_queue** q)
{
    if (!sys || !q || n < 1) return IA_ERR_INVALID_ARG;
    ia_launch_opts o;
    std::memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (o.kernel == IA_KERNEL_PLAIN) o.kernel = IA_KERNEL_PERSISTENT;
    if (o.scratch != nullptr || o.scratch_bytes != 0 || o.tail_pair == 1) return IA_ERR_INVALID_ARG;
    Resolved r;
    int rc = resolve(n, &o, r);
    if (rc != IA_OK) return rc;
    SchedCfg cfg;
    rc = sched_config(sys, r, cfg);
    if (rc != IA_OK) return rc;
    // every block must be resident (the parts end on a grid-wide condition)
    if (cfg.grid > cfg.resident * sys->num_sms) return IA_ERR_INVALID_ARG;
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, sys->device);
    if (!coop) return IA_ERR_NO_DEVICE;
    const long long carry_cap = (long long)cfg.grid * cfg.block;  // one record per lane of the grid
    // one group-mode record per trajectory the reserved SMs' tail warps can hold
    const long long tcarry_cap = (long long)(cfg.tail_sms > 0 ? cfg.tail_sms : 1) * cfg.tail_warps * 5;
    const size_t carry_off = r.bytes;
    const size_t bytes = carry_off + 2 * (size_t)(carry_cap + tcarry_cap) * sizeof(Susp);
    ia_queue* Q = new (std::nothrow) ia_queue;
    if (!Q) return IA_ERR_INVALID_ARG;
    Q->scratch = nullptr;
    if (cudaMalloc(&Q->scratch, bytes) != cudaSuccess) {
        delete Q;
        return IA_ERR_CUDA;
    }
    Q->sys = sys;
    Q->n = n;
    Q->opts = o;
    Q->bytes = bytes;
    Q->carry_off = carry_off;
    Q->carry_cap = carry_cap;
    Q->tcarry_cap = tcarry_cap;
    Q->started = 0;
    Q->parts = 0;
    std::memset(Q->bound, 0, sizeof(Q->bound));
    *q = Q;
    return IA_OK;
}

int ia_queue_launch(ia_queue* q, const ia_ic_soa* ic, const ia_obs_soa* out, int64_t count, void* stream)
{
    if (!q || !ic || !out || count < 0) return IA_ERR_INVALID_ARG;
    ia_system* sys = q->sys;
    const int64_t n = q->n;
    if (q->started >= n || count > n - q->started) return IA_ERR_INVALID_ARG;
    if (!ic->y0 || !ic->phi0 || ic->ld < n) return IA_ERR_INVALID_ARG;
    if (!out->theta_s || !out->dp || !out->dE_ion || !out->t_final || !out->t_first_bounce ||
        !out->t_last_bounce || !out->n_bounce || !out->status || !out->n_steps || !out->n_rej)
        return IA_ERR_INVALID_ARG;
    if (out->y_final && out->ld < n) return IA_ERR_INVALID_ARG;
    if (!aligned8(ic->y0) || !aligned8(ic->phi0) || !aligned8(out->theta_s) || !aligned8(out->dp) ||
        !aligned8(out->dE_ion) || !aligned8(out->t_final) || !aligned8(out->t_first_bounce) ||
        !aligned8(out->t_last_bounce) || (out->y_final && !aligned8(out->y_final)) ||
        (ic->order && !aligned8(ic->order)))
        return IA_ERR_ALIGNMENT;
    // the records of running trajectories hold batch indices: every part sees the same arrays
    const void* ptrs[18] = {ic->y0, ic->phi0, ic->sys_id, ic->order, (const void*)(intptr_t)ic->ld,
                            out->theta_s, out->dp, out->dE_ion, out->t_final, out->t_first_bounce,
                            out->t_last_bounce, out->n_bounce, out->status, out->n_steps, out->n_rej,
                            out->y_final, (const void*)(intptr_t)(out->y_final ? out->ld : 0), nullptr};
    if (q->parts == 0) {
        std::memcpy(q->bound, ptrs, sizeof(ptrs));
    } else if (std::memcmp(q->bound, ptrs, sizeof(ptrs)) != 0) {
        return IA_ERR_INVALID_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != sys->device) return IA_ERR_INVALID_ARG;
    Resolved r;
    int rc = resolve(n, &q->opts, r);
    if (rc != IA_OK) return rc;
    SchedCfg cfg;
    rc = sched_config(sys, r, cfg);
    if (rc != IA_OK) return rc;
    if ((long long)cfg.grid * cfg.block > q->carry_cap) return IA_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char* scratch = static_cast<char*>(q->scratch);
    Counters* ctr = reinterpret_cast<Counters*>(scratch);
    Susp* carry = reinterpret_cast<Susp*>(scratch + q->carry_off);
    const int in = q->parts & 1, outb = in ^ 1;
    Susp* tcarry = carry + 2 * (size_t)q->carry_cap;
    if (q->parts == 0) {
        if (cudaMemsetAsync(scratch, 0, SCRATCH_HEAD + ready_bytes(r.cap), st) != cudaSuccess) return IA_ERR_CUDA;
    } else {
        if (cudaMemsetAsync(scratch, 0, PER_LAUNCH_BYTES, st) != cudaSuccess ||
            cudaMemsetAsync(&ctr->carry_n[outb], 0, sizeof(unsigned long long), st) != cudaSuccess ||
            cudaMemsetAsync(&ctr->tcarry_n[outb], 0, sizeof(unsigned long long), st) != cudaSuccess)
            return IA_ERR_CUDA;
    }
    Part part;
    part.first = (long long)q->started;
    part.count = (long long)count;
    part.carry_in = carry + (size_t)in * (size_t)q->carry_cap;
    part.carry_in_n = q->parts == 0 ? nullptr : &ctr->carry_n[in];
    part.last = q->started + count == n ? 1 : 0;
    part.carry_out = part.last ? nullptr : carry + (size_t)outb * (size_t)q->carry_cap;
    part.carry_out_n = part.last ? nullptr : &ctr->carry_n[outb];
    part.carry_cap = q->carry_cap;
    part.tcarry_in = tcarry + (size_t)in * (size_t)q->tcarry_cap;
    part.tcarry_in_n = q->parts == 0 ? nullptr : &ctr->tcarry_n[in];
    part.tcarry_out = part.last ? nullptr : tcarry + (size_t)outb * (size_t)q->tcarry_cap;
    part.tcarry_out_n = part.last ? nullptr : &ctr->tcarry_n[outb];
    part.tcarry_cap = q->tcarry_cap;
    part.lane_only = 0;
    IcPtrs icp{ic->y0, ic->phi0, ic->sys_id, reinterpret_cast<const long long*>(ic->order), (long long)ic->ld};
    ObsPtrs op{out->theta_s, out->dp, out->dE_ion, out->t_final, out->t_first_bounce, out->t_last_bounce,
               out->n_bounce, out->status, out->n_steps, out->n_rej, out->y_final,
               (long long)(out->y_final ? out->ld : 0)};
    rc = launch_sched(sys, cfg, r, icp, op, part, scratch, st);
    if (rc != IA_OK) return rc;
    q->started += count;
    q->parts += 1;
    return IA_OK;
}

int ia_queue_reset(ia_queue* q)
{
    if (!q) return IA_ERR_INVALID_ARG;
    q->started = 0;
    q->parts = 0;
    std::memset(q->bound, 0, sizeof(q->bound));
    return IA_OK;
}

int ia_queue_state(const ia_queue* q, int64_t* started, int64_t* parts, int64_t* n)
{
    if (!q) return IA_ERR_INVALID_ARG;
    if (started) *started = q->started;
    if (parts) *parts = q->parts;
    if (n) *n = q->n;
    return IA_OK;
}

int ia_queue_phases(const ia_queue* q, double* lane_ms, double* total_ms, int64_t* errors)
{
    if (!q || q->parts == 0) return IA_ERR_INVALID_ARG;
    return ia_launch_phases(q->sys, q->scratch, lane_ms, total_ms, errors);
}

int ia_queue_destroy(ia_queue* q)
{
    if (!q) return IA_OK;
    cudaFree(q->scratch);
    delete q;
    return IA_OK;
}

// ---------------------------------------------------------------------------------------------
// Batch statistics

namespace {
int stats_grid(const ia_system* sys, int64_t n)
{
    long long g = (n + STATS_BLOCK - 1) / STATS_BLOCK;
    const long long gmax = 4LL * sys->num_sms;
    if (g > gmax) g = gmax;
    if (g < 1) g = 1;
    return (int)g;
}
}  // namespace

int ia_reserve_stats(ia_system* sys, int64_t n, int32_t n_cells)
{
    if (!sys || n < 0 || n_cells < 1 || n_cells > IA_STATS_MAX_CELLS) return IA_ERR_INVALID_ARG;
    const size_t need = (size_t)stats_grid(sys, n) * (size_t)n_cells * 2 * sizeof(double);
    if (need <= sys->stats_scratch_bytes) return IA_OK;
    void* p = nullptr;
    if (cudaMalloc(&p, need) != cudaSuccess) return IA_ERR_CUDA;
    cudaFree(sys->d_stats_scratch);
    sys->d_stats_scratch = p;
    sys->stats_scratch_bytes = need;
    return IA_OK;
}

int ia_reduce_stats(ia_system* sys, const ia_obs_soa* obs, int64_t n, const int32_t* cell_id, int32_t n_cells,
                    ia_stats* stats, void* stream)
{
    if (!sys || !obs || !stats || n < 0 || n_cells < 1 || n_cells > IA_STATS_MAX_CELLS) return IA_ERR_INVALID_ARG;
    if (n > 0 && (!obs->status || !obs->n_bounce || !obs->n_steps || !obs->n_rej || !obs->dE_ion ||
                  !obs->t_first_bounce || !obs->t_last_bounce))
        return IA_ERR_INVALID_ARG;
    if (!aligned8(stats) || (n > 0 && !aligned8(obs->dE_ion))) return IA_ERR_ALIGNMENT;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(stats, 0, sizeof(ia_stats) * (size_t)n_cells, st) != cudaSuccess) return IA_ERR_CUDA;
    const int grid = stats_grid(sys, n);
    int rc = ia_reserve_stats(sys, n, n_cells);
    if (rc != IA_OK) return rc;
    double* partial = static_cast<double*>(sys->d_stats_scratch);
    long long chunk = (n + grid - 1) / grid;
    chunk = (chunk + 31) / 32 * 32;
    const size_t shmem = (size_t)(STATS_BLOCK / 32) * n_cells * 2 * sizeof(double);
    if (shmem > 48 * 1024 &&
        cudaFuncSetAttribute(k_stats_pass1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem) != cudaSuccess)
        return IA_ERR_CUDA;
    ObsPtrs op{obs->theta_s, obs->dp, obs->dE_ion, obs->t_final, obs->t_first_bounce, obs->t_last_bounce,
               obs->n_bounce, obs->status, obs->n_steps, obs->n_rej, nullptr, 0};
    k_stats_pass1<<<grid, STATS_BLOCK, shmem, st>>>(op, (long long)n, cell_id, n_cells, stats, partial, chunk);
    k_stats_pass2<<<(n_cells + 127) / 128, 128, 0, st>>>(partial, grid, n_cells, stats);
    return cudaGetLastError() == cudaSuccess ? IA_OK : IA_ERR_CUDA;
}

// ---------------------------------------------------------------------------------------------
// CUDA graph of one batch

int ia_graph_create(ia_system* sys, const ia_ic_soa* ic, int64_t n, const ia_obs_soa* out,
                    const ia_launch_opts* opts, const int32_t* cell_id, int32_t n_cells, ia_stats* stats,
                    void* stream, ia_graph** graph)
{
    if (!sys || !ic || !out || !graph || !stream || n < 1) return IA_ERR_INVALID_ARG;
    ia_launch_opts o;
    std::memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    o.kernel = IA_KERNEL_PERSISTENT;
    int rc = IA_OK;
    if (!o.scratch) rc = ia_reserve(sys, n, &o);
    if (rc == IA_OK && stats) rc = ia_reserve_stats(sys, n, n_cells);
    if (rc != IA_OK) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return IA_ERR_CUDA;
    rc = ia_launch(sys, ic, n, out, &o, stream);
    if (rc == IA_OK && stats) rc = ia_reduce_stats(sys, out, n, cell_id, n_cells, stats, stream);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(st, &g);
    if (rc != IA_OK || ec != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        return rc != IA_OK ? rc : IA_ERR_CUDA;
    }
    cudaGraphExec_t ex = nullptr;
    if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        return IA_ERR_CUDA;
    }
    ia_graph* G = new (std::nothrow) ia_graph;
    if (!G) {
        cudaGraphExecDestroy(ex);
        cudaGraphDestroy(g);
        return IA_ERR_INVALID_ARG;
    }
    G->graph = g;
    G->exec = ex;
    *graph = G;
    return IA_OK;
}

int ia_graph_launch(ia_graph* graph, void* stream)
{
    if (!graph) return IA_ERR_INVALID_ARG;
    return cudaGraphLaunch(graph->exec, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? IA_OK : IA_ERR_CUDA;
}

int ia_graph_destroy(ia_graph* graph)
{
    if (!graph) return IA_OK;
    cudaGraphExecDestroy(graph->exec);
    cudaGraphDestroy(graph->graph);
    delete graph;
    return IA_OK;
}

// ---------------------------------------------------------------------------------------------
// Autotuner of the lane phase

int ia_autotune(ia_system* sys, const ia_ic_soa* ic, int64_t n, int32_t attempt_cap, const ia_launch_opts* base,
                ia_launch_opts* best, double* best_ms, void* stream)
{
    if (!sys || !ic || !best || !best_ms || n < 1 || attempt_cap < 64 || attempt_cap > (1 << 20))
        return IA_ERR_INVALID_ARG;
    if (!ic->y0 || !ic->phi0 || ic->ld < n) return IA_ERR_INVALID_ARG;
    if (!aligned8(ic->y0) || !aligned8(ic->phi0) || (ic->order && !aligned8(ic->order))) return IA_ERR_ALIGNMENT;
    ia_launch_opts b0;
    std::memset(&b0, 0, sizeof(b0));
    if (base) b0 = *base;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // throw-away outputs and a suspend area with room for every trajectory (each stops at the cap)
    const size_t nn = (size_t)n;
    const size_t obs_bytes = nn * (6 * sizeof(double) + 4 * sizeof(int32_t));
    const long long cap = (long long)n;
    const size_t scr_bytes = SCRATCH_HEAD + ready_bytes(cap) + (size_t)cap * sizeof(Susp);
    char* obuf = nullptr;
    char* scr = nullptr;
    if (cudaMalloc(&obuf, obs_bytes) != cudaSuccess) return IA_ERR_CUDA;
    if (cudaMalloc(&scr, scr_bytes) != cudaSuccess) {
        cudaFree(obuf);
        return IA_ERR_CUDA;
    }
    ObsPtrs op;
    op.theta_s = (double*)obuf;
    op.dp = op.theta_s + nn;
    op.dE_ion = op.dp + nn;
    op.t_final = op.dE_ion + nn;
    op.t_first = op.t_final + nn;
    op.t_last = op.t_first + nn;
    op.n_bounce = (int32_t*)(op.t_last + nn);
    op.status = (uint32_t*)(op.n_bounce + nn);
    op.n_steps = (int32_t*)(op.status + nn);
    op.n_rej = op.n_steps + nn;
    op.y_final = nullptr;
    op.ld_out = 0;
    IcPtrs icp{ic->y0, ic->phi0, ic->sys_id, reinterpret_cast<const long long*>(ic->order), (long long)ic->ld};
    Counters* ctr = reinterpret_cast<Counters*>(scr);
    unsigned* ready = reinterpret_cast<unsigned*>(scr + SCRATCH_HEAD);
    Susp* susp = reinterpret_cast<Susp*>(scr + SCRATCH_HEAD + ready_bytes(cap));
    struct Cand { int block, minb, refill; };
    const Cand cands[] = {{128, 1, 1}, {128, 1, 4}, {128, 1, 16}, {64, 1, 1}, {64, 1, 4},
                          {256, 1, 1}, {256, 1, 4}, {128, 3, 1}, {128, 3, 4}};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = IA_OK;
    constexpr int NC = (int)(sizeof(cands) / sizeof(cands[0]));
    constexpr int PASSES = 2;  // every candidate timed twice, interleaved; its time is the shorter
    double cand_t[NC];
    for (int c = 0; c < NC; ++c) cand_t[c] = 1e300;
    for (int it = -1; it < PASSES * NC && rc == IA_OK; ++it) {
        const int c = it < 0 ? 0 : it % NC;  // it = -1: warm-up of the first candidate
        const Cand cd = cands[c];
        const void* fn = sched_fn(cd.block, cd.minb, 6);
        int resident = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, fn, cd.block, 0) != cudaSuccess || resident <= 0) {
            rc = IA_ERR_CUDA;
            break;
        }
        int grid = resident * sys->num_sms;
        long long nn_ = (long long)n;
        int refill = cd.refill, budget = attempt_cap, tail_sms = 0, wait_ok = 0, pair = 0, n_sys = sys->n_sys;
        int tail_warps = TAIL_WARPS;
        long long capv = cap;
        const SysDev* tab = sys->d_tab;
        Part part = single_part(nn_);
        part.lane_only = 1;  // every trajectory stops at the cap (its suspend record is never resumed)
        void* args[] = {(void*)&tab, (void*)&n_sys, (void*)&icp, (void*)&op, (void*)&part, (void*)&ctr,
                        (void*)&ready, (void*)&susp, (void*)&capv, (void*)&refill, (void*)&budget,
                        (void*)&tail_sms, (void*)&wait_ok, (void*)&pair, (void*)&tail_warps};
        if (cudaMemsetAsync(scr, 0, SCRATCH_HEAD + ready_bytes(cap), st) != cudaSuccess) rc = IA_ERR_CUDA;
        cudaEventRecord(e0, st);
        // budget > 0 with no tail workers: the kernel stops every trajectory at the cap
        if (rc == IA_OK && cudaLaunchKernel(fn, dim3(grid), dim3(cd.block), args, 0, st) != cudaSuccess) rc = IA_ERR_CUDA;
        cudaEventRecord(e1, st);
        if (rc == IA_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = IA_ERR_CUDA;
        float ms = 0.0f;
        if (rc == IA_OK) cudaEventElapsedTime(&ms, e0, e1);
        if (it >= 0 && rc == IA_OK && ms < cand_t[c]) cand_t[c] = ms;
    }
    // Candidates within 1 % of the fastest are treated as equal, and the smallest refill among them
    // wins (then the fastest). The sample's trajectories all stop at the same cap, so lanes fall idle
    // together and a lazier refill costs nothing there; in a whole batch lengths spread, and refilling
    // each lane at once keeps warps fuller.
    double best_t = 1e300;
    for (int c = 0; c < NC; ++c) best_t = cand_t[c] < best_t ? cand_t[c] : best_t;
    Cand win = cands[0];
    double win_t = 1e300;
    for (int c = 0; c < NC; ++c) {
        if (cand_t[c] > best_t * 1.01) continue;
        if (win_t == 1e300 || cands[c].refill < win.refill || (cands[c].refill == win.refill && cand_t[c] < win_t)) {
            win = cands[c];
            win_t = cand_t[c];
        }
    }
    best_t = win_t;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(obuf);
    cudaFree(scr);
    if (rc != IA_OK) return rc;
    *best = b0;
    best->kernel = IA_KERNEL_PERSISTENT;
    best->block = win.block;
    best->regs_variant = win.minb;
    best->refill = win.refill;
    *best_ms = best_t;
    return IA_OK;
}


// ---------------------------------------------------------------------------------------------
// Tangent launch

int ia_launch_tangent(ia_system* sys, const ia_ic_soa* ic, int64_t n, const ia_obs_soa* out,
                      const ia_tangent_in* tin, const ia_tangent_out* tout, void* stream)
{
    if (!sys || !ic || !out || !tin || !tout || n < 0) return IA_ERR_INVALID_ARG;
    if (n == 0) return IA_OK;
    if (!ic->y0 || !ic->phi0 || ic->ld < n) return IA_ERR_INVALID_ARG;
    if (!out->theta_s || !out->dp || !out->dE_ion || !out->t_final || !out->t_first_bounce ||
        !out->t_last_bounce || !out->n_bounce || !out->status || !out->n_steps || !out->n_rej)
        return IA_ERR_INVALID_ARG;
    if (out->y_final && out->ld < n) return IA_ERR_INVALID_ARG;
    if (!aligned8(ic->y0) || !aligned8(ic->phi0) || !aligned8(out->theta_s) || !aligned8(out->dp) ||
        !aligned8(out->dE_ion) || !aligned8(out->t_final) || !aligned8(out->t_first_bounce) ||
        !aligned8(out->t_last_bounce) || (out->y_final && !aligned8(out->y_final)))
        return IA_ERR_ALIGNMENT;
    if (tin->ndir < 1 || tin->ndir > 4 || !tin->dy0 || tin->ld < n || tin->reserved != 0) return IA_ERR_INVALID_ARG;
    if (!tout->d_theta_s || !tout->d_dp || !tout->d_dE_ion || !tout->d_t_final || tout->ld < n)
        return IA_ERR_INVALID_ARG;
    if (!aligned8(tin->dy0) || !aligned8(tout->d_theta_s) || !aligned8(tout->d_dp) || !aligned8(tout->d_dE_ion) ||
        !aligned8(tout->d_t_final) || (tout->dy_final && !aligned8(tout->dy_final)) ||
        (tout->ftle && !aligned8(tout->ftle)))
        return IA_ERR_ALIGNMENT;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // a 64-bit work counter in the system's scratch
    int rc = ia_reserve(sys, 0, nullptr);
    if (rc != IA_OK) return rc;
    unsigned long long* work = reinterpret_cast<unsigned long long*>(sys->d_scratch);
    if (cudaMemsetAsync(work, 0, sizeof(unsigned long long), st) != cudaSuccess) return IA_ERR_CUDA;
    IcPtrs icp{ic->y0, ic->phi0, ic->sys_id, nullptr, (long long)ic->ld};
    ObsPtrs op{out->theta_s, out->dp, out->dE_ion, out->t_final, out->t_first_bounce, out->t_last_bounce,
               out->n_bounce, out->status, out->n_steps, out->n_rej, out->y_final,
               (long long)(out->y_final ? out->ld : 0)};
    TanIn ti;
    ti.dy0 = tin->dy0;
    for (int k = 0; k < 4; ++k)
        for (int j = 0; j < 3; ++j) ti.dq[k][j] = tin->dq[k][j];
    ti.ndir = tin->ndir;
    ti.ld = (long long)tin->ld;
    TanOut to{tout->d_theta_s, tout->d_dp, tout->d_dE_ion, tout->d_t_final, tout->dy_final, tout->ftle,
              (long long)tout->ld};
    int resident = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_tangent, 128, 0) != cudaSuccess || resident <= 0)
        return IA_ERR_CUDA;
    const long long warps = n;  // one warp per trajectory
    long long grid = (long long)resident * sys->num_sms;
    if (grid * 4 > warps) grid = (warps + 3) / 4;
    k_tangent<<<(unsigned)grid, 128, 0, st>>>(sys->d_tab, sys->n_sys, icp, op, (long long)n, ti, to, work);
    return cudaGetLastError() == cudaSuccess ? IA_OK : IA_ERR_CUDA;
}

// ---------------------------------------------------------------------------------------------
// Adjoint launch

namespace {

constexpr int ADJ_DEFAULT_SEG = 10000;
constexpr int ADJ_DEFAULT_CKPT = 64;
constexpr size_t ADJ_HEAD = 256;

struct AdjResolved {
    long long warps;
    int seg, max_ckpt;
    size_t bytes;
};

int adj_resolve(const ia_system* sys, int64_t n, const ia_adjoint_opts* opts, AdjResolved& r)
{
    ia_adjoint_opts o;
    std::memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (n < 0 || o.seg < 0 || o.max_ckpt < 0 || o.warps < 0 || o.scratch_bytes < 0) return IA_ERR_INVALID_ARG;
    r.seg = o.seg ? o.seg : ADJ_DEFAULT_SEG;
    r.max_ckpt = o.max_ckpt ? o.max_ckpt : ADJ_DEFAULT_CKPT;
    if (r.seg < 16 || r.seg > 1000000 || r.max_ckpt < 2 || r.max_ckpt > 1048576 || (r.max_ckpt & 1))
        return IA_ERR_INVALID_ARG;
    long long w = o.warps;
    if (w == 0) {
        if (!sys) return IA_ERR_INVALID_ARG;
        int resident = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_adjoint, 128, 0) != cudaSuccess ||
            resident <= 0)
            return IA_ERR_CUDA;
        w = (long long)resident * sys->num_sms * ADJ_WARPS;
    }
    if (w > n) w = n;
    if (w < 1) w = 1;
    if (w > (1ll << 24)) return IA_ERR_TOO_LARGE;
    r.warps = w;
    const size_t per = (size_t)r.max_ckpt * CK_DOUBLES * 8u + (size_t)r.seg * SR_DOUBLES * 8u;
    r.bytes = ADJ_HEAD + (size_t)w * per;
    return IA_OK;
}

}  // namespace

int64_t ia_adjoint_scratch_bytes(const ia_system* sys, int64_t n, const ia_adjoint_opts* opts)
{
    AdjResolved r;
    const int rc = adj_resolve(sys, n, opts, r);
    if (rc != IA_OK) return rc;
    return (int64_t)r.bytes;
}

int ia_launch_adjoint(ia_system* sys, const ia_ic_soa* ic, int64_t n, const ia_obs_soa* out,
                      const ia_tangent_in* seeds, const ia_adjoint_out* aout, const ia_adjoint_opts* opts,
                      void* stream)
{
    if (!sys || !ic || !out || !aout || n < 0) return IA_ERR_INVALID_ARG;
    if (n == 0) return IA_OK;
    if (!ic->y0 || !ic->phi0 || ic->ld < n) return IA_ERR_INVALID_ARG;
    if (!out->theta_s || !out->dp || !out->dE_ion || !out->t_final || !out->t_first_bounce ||
        !out->t_last_bounce || !out->n_bounce || !out->status || !out->n_steps || !out->n_rej)
        return IA_ERR_INVALID_ARG;
    if (out->y_final && out->ld < n) return IA_ERR_INVALID_ARG;
    if (!aligned8(ic->y0) || !aligned8(ic->phi0) || !aligned8(out->theta_s) || !aligned8(out->dp) ||
        !aligned8(out->dE_ion) || !aligned8(out->t_final) || !aligned8(out->t_first_bounce) ||
        !aligned8(out->t_last_bounce) || (out->y_final && !aligned8(out->y_final)))
        return IA_ERR_ALIGNMENT;
    const int ndir = seeds ? seeds->ndir : 0;
    if (seeds && (ndir < 1 || ndir > 4 || !seeds->dy0 || seeds->ld < n || seeds->reserved != 0))
        return IA_ERR_INVALID_ARG;
    if (!aout->grad_y0 && !aout->grad_q && ndir == 0) return IA_ERR_INVALID_ARG;
    if ((aout->grad_y0 || aout->grad_q || ndir > 0) && aout->ld < n) return IA_ERR_INVALID_ARG;
    if (ndir > 0 && (!aout->d_theta_s || !aout->d_dp || !aout->d_dE_ion || !aout->d_t_final))
        return IA_ERR_INVALID_ARG;
    if ((aout->grad_y0 && !aligned8(aout->grad_y0)) || (aout->grad_q && !aligned8(aout->grad_q)) ||
        (ndir > 0 && (!aligned8(seeds->dy0) || !aligned8(aout->d_theta_s) || !aligned8(aout->d_dp) ||
                      !aligned8(aout->d_dE_ion) || !aligned8(aout->d_t_final))))
        return IA_ERR_ALIGNMENT;
    AdjResolved r;
    int rc = adj_resolve(sys, n, opts, r);
    if (rc != IA_OK) return rc;
    void* scratch = opts ? opts->scratch : nullptr;
    if (scratch) {
        if ((reinterpret_cast<uintptr_t>(scratch) & 255u) != 0) return IA_ERR_ALIGNMENT;
        if ((size_t)opts->scratch_bytes < r.bytes) return IA_ERR_INVALID_ARG;
    } else {
        if (r.bytes > sys->adj_scratch_bytes) {
            void* p = nullptr;
            if (cudaMalloc(&p, r.bytes) != cudaSuccess) return IA_ERR_CUDA;
            cudaFree(sys->d_adj_scratch);
            sys->d_adj_scratch = p;
            sys->adj_scratch_bytes = r.bytes;
        }
        scratch = sys->d_adj_scratch;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    unsigned char* base = static_cast<unsigned char*>(scratch);
    if (cudaMemsetAsync(base, 0, ADJ_HEAD, st) != cudaSuccess) return IA_ERR_CUDA;
    AdjBuf buf;
    buf.work = reinterpret_cast<unsigned long long*>(base);
    buf.errors = reinterpret_cast<unsigned long long*>(base + 8);
    buf.ckpt = reinterpret_cast<double*>(base + ADJ_HEAD);
    buf.steps = buf.ckpt + (size_t)r.warps * r.max_ckpt * CK_DOUBLES;
    buf.warps = r.warps;
    buf.max_ckpt = r.max_ckpt;
    buf.seg = r.seg;
    IcPtrs icp{ic->y0, ic->phi0, ic->sys_id, nullptr, (long long)ic->ld};
    ObsPtrs op{out->theta_s, out->dp, out->dE_ion, out->t_final, out->t_first_bounce, out->t_last_bounce,
               out->n_bounce, out->status, out->n_steps, out->n_rej, out->y_final,
               (long long)(out->y_final ? out->ld : 0)};
    AdjIn ai;
    std::memset(&ai, 0, sizeof(ai));
    ai.ndir = ndir;
    if (ndir > 0) {
        ai.dy0 = seeds->dy0;
        for (int k = 0; k < 4; ++k)
            for (int j = 0; j < 3; ++j) ai.dq[k][j] = seeds->dq[k][j];
        ai.ld = (long long)seeds->ld;
    }
    AdjOut ao{aout->grad_y0, aout->grad_q, aout->d_theta_s, aout->d_dp, aout->d_dE_ion, aout->d_t_final,
              (long long)aout->ld};
    const long long grid = (r.warps + ADJ_WARPS - 1) / ADJ_WARPS;
    k_adjoint<<<(unsigned)grid, 128, 0, st>>>(sys->d_tab, sys->n_sys, icp, op, (long long)n, ai, ao, buf);
    return cudaGetLastError() == cudaSuccess ? IA_OK : IA_ERR_CUDA;
}

int ia_launch_phases(ia_system* sys, const void* scratch, double* lane_ms, double* total_ms, int64_t* errors)
{
    if (!sys || !lane_ms || !total_ms) return IA_ERR_INVALID_ARG;
    const void* base = scratch ? scratch : sys->d_scratch;
    if (!base) return IA_ERR_INVALID_ARG;
    Counters c;
    if (cudaMemcpy(&c, base, sizeof(Counters), cudaMemcpyDeviceToHost) != cudaSuccess) return IA_ERR_CUDA;
    if (c.t_start == 0 || c.t_end < c.t_start) return IA_ERR_INVALID_ARG;
    *lane_ms = c.t_lane_end >= c.t_start ? 1e-6 * (double)(c.t_lane_end - c.t_start) : 0.0;
    *total_ms = 1e-6 * (double)(c.t_end - c.t_start);
    if (errors) *errors = (int64_t)c.errors;
    return IA_OK;
}

int ia_philox4x64(uint64_t key0, uint64_t key1, uint64_t ctr1, int64_t first, int64_t n_blocks, uint64_t* out,
                  void* stream)
{
    if (n_blocks < 0 || first < 0 || first > INT64_MAX - n_blocks) return IA_ERR_INVALID_ARG;
    if (n_blocks == 0) return IA_OK;
    if (!out) return IA_ERR_INVALID_ARG;
    if (!aligned8(out)) return IA_ERR_ALIGNMENT;
    if (n_blocks > INT64_MAX / 4) return IA_ERR_TOO_LARGE;
    int sms = 0;
    if (sample_device(&sms) != IA_OK) return IA_ERR_NO_DEVICE;
    const long long grid = std::min<long long>((n_blocks + ia_sample::SAMPLE_THREADS - 1) / ia_sample::SAMPLE_THREADS,
                                               8LL * sms);
    ia_sample::k_philox<<<(unsigned)grid, ia_sample::SAMPLE_THREADS, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        key0, key1, ctr1, (long long)first, (long long)n_blocks, reinterpret_cast<unsigned long long*>(out));
    return cudaGetLastError() == cudaSuccess ? IA_OK : IA_ERR_CUDA;
}

int ia_sample_ics(const ia_sampler* s, int64_t first, int64_t n, double* y0, double* phi0, int64_t ld, void* stream)
{
    if (!s || n < 0 || first < 0 || first > INT64_MAX - n) return IA_ERR_INVALID_ARG;
    if (n == 0) return IA_OK;
    if (!y0 || !phi0 || ld < n || ld > INT64_MAX / 12) return IA_ERR_INVALID_ARG;
    if (!aligned8(y0) || !aligned8(phi0)) return IA_ERR_ALIGNMENT;
    auto pos = [](double x) { return std::isfinite(x) && x > 0.0; };
    if (s->kind < IA_SAMPLE_HEAD_ON || s->kind > IA_SAMPLE_DISK) return IA_ERR_INVALID_ARG;
    if ((s->random_phase != 0 && s->random_phase != 1) || (s->micromotion != 0 && s->micromotion != 1) ||
        (s->rf_sign != 1 && s->rf_sign != -1))
        return IA_ERR_INVALID_ARG;
    if (!pos(s->m_ion) || !pos(s->m_atom) || !pos(s->r0) || !std::isfinite(s->Omega) ||
        (!s->random_phase && !std::isfinite(s->phase)))
        return IA_ERR_INVALID_ARG;
    for (int j = 0; j < 3; ++j)
        if (!std::isfinite(s->q[j])) return IA_ERR_INVALID_ARG;
    ia_sample::SampleParams p{};
    p.kind = s->kind;
    p.random_phase = s->random_phase;
    p.micromotion = s->micromotion;
    p.rf_sign = s->rf_sign;
    p.r0 = s->r0;
    p.phase = s->random_phase ? 0.0 : s->phase;
    p.Omega = s->Omega;
    for (int j = 0; j < 3; ++j) p.q[j] = s->q[j];
    if (s->kind == IA_SAMPLE_HEAD_ON) {
        if (!pos(s->E)) return IA_ERR_INVALID_ARG;
        p.v0 = std::sqrt(2.0 * s->E / s->m_atom);
    } else {
        if (!pos(s->kT) || !std::isfinite(s->kT_ion) || s->kT_ion < 0.0) return IA_ERR_INVALID_ARG;
        const double omega = std::fabs(s->q[0]) * s->Omega / (2.0 * std::sqrt(2.0));
        if (s->kT_ion > 0.0 && !pos(omega)) return IA_ERR_INVALID_ARG;
        if (s->kind == IA_SAMPLE_DISK && !(std::isfinite(s->b_max) && s->b_max >= 0.0 && s->b_max < s->r0))
            return IA_ERR_INVALID_ARG;
        p.sig_a = std::sqrt(s->kT / s->m_atom);
        p.sig_v = std::sqrt(s->kT_ion / s->m_ion);
        p.sig_x = s->kT_ion > 0.0 ? p.sig_v / omega : 0.0;
        p.b_max = s->b_max;
    }
    p.seed = s->seed;
    p.first = first;
    p.n = n;
    p.ld = ld;
    p.y0 = y0;
    p.phi0 = phi0;
    int sms = 0;
    if (sample_device(&sms) != IA_OK) return IA_ERR_NO_DEVICE;
    const long long grid = std::min<long long>((n + ia_sample::SAMPLE_THREADS - 1) / ia_sample::SAMPLE_THREADS,
                                               8LL * sms);
    ia_sample::k_sample<<<(unsigned)grid, ia_sample::SAMPLE_THREADS, 0, reinterpret_cast<cudaStream_t>(stream)>>>(p);
    return cudaGetLastError() == cudaSuccess ? IA_OK : IA_ERR_CUDA;
}

int ia_rcp_check(const double* x, double* y, int64_t n, void* stream)
{
    if (!x || !y || n < 0) return IA_ERR_INVALID_ARG;
    if (n == 0) return IA_OK;
    if (!aligned8(x) || !aligned8(y)) return IA_ERR_ALIGNMENT;
    const long long blocks = (n + 255) / 256;
    k_rcp_check<<<(unsigned)blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(x, y, (long long)n);
    return cudaGetLastError() == cudaSuccess ? IA_OK : IA_ERR_CUDA;
}

int ia_fp64_peak(int32_t blocks_per_sm, int32_t iters, void* stream, double* flops)
{
    if (!flops || blocks_per_sm < 1 || blocks_per_sm > 64 || iters < 1) return IA_ERR_INVALID_ARG;
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
        return IA_ERR_NO_DEVICE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int block = 256;
    const int grid = blocks_per_sm * prop.multiProcessorCount;
    double* buf = nullptr;
    if (cudaMalloc(&buf, sizeof(double) * (size_t)grid * block) != cudaSuccess) return IA_ERR_CUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fp64_fma<<<grid, block, 0, st>>>(buf, 16, 0.999999, 1e-6);  // warm-up
    cudaEventRecord(e0, st);
    k_fp64_fma<<<grid, block, 0, st>>>(buf, iters, 0.999999, 1e-6);
    cudaEventRecord(e1, st);
    int rc = IA_OK;
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = IA_ERR_CUDA;
    float ms = 0.0f;
    if (rc == IA_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = IA_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (rc != IA_OK) return rc;
    *flops = 2.0 * 8.0 * (double)iters * (double)grid * (double)block / (1e-3 * (double)ms);
    return IA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Allocation-free launch: the persistent launch with its scratch in a fixed device array.
//
// Some callers cannot allocate device memory at the time they launch: code that records a CUDA
// graph (cudaMalloc is not allowed during stream capture), plug-ins running inside a host program
// that owns the whole device-memory budget through its own pool, and real-time loops that forbid
// allocation after start-up. ia_launch_static serves them with scratch that exists from the moment
// the library's device code is loaded on a GPU until the process exits.

namespace {

static __device__ __align__(256) unsigned char g_ia_static_scratch[IA_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_addr[kMaxDevices] = {};
unsigned long long g_static_ctx[kMaxDevices] = {};

// Identity of the calling thread's current CUDA context (unique for the life of the process), or 0
// when it cannot be told. A device reset destroys the context that loaded the library's device code;
// the array then lives at a new address in the next context, so the cached address is keyed on this.
// The driver functions are reached through the runtime's entry-point query (no link to the driver).
unsigned long long current_context_id()
{
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
    }
    if (!get_current || !get_id) return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of g_ia_static_scratch on the current device: looked up once per device and context
// (again after a device reset; every call when the context cannot be identified).
int static_scratch_address(int dev, void** out)
{
    if (dev < 0 || dev >= kMaxDevices) return IA_ERR_NO_DEVICE;
    std::lock_guard<std::mutex> lock(g_static_mu);
    const unsigned long long ctx = current_context_id();
    if (!g_static_addr[dev] || ctx == 0 || g_static_ctx[dev] != ctx) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_ia_static_scratch) != cudaSuccess || !p) return IA_ERR_CUDA;
        g_static_addr[dev] = p;
        g_static_ctx[dev] = ctx;
    }
    *out = g_static_addr[dev];
    return IA_OK;
}

}  // namespace

extern "C" int ia_launch_static(ia_system* sys, const ia_ic_soa* ic, int64_t n, const ia_obs_soa* out,
                                const ia_launch_opts* opts, void* stream)
{
    if (!sys || n < 0) return IA_ERR_INVALID_ARG;
    ia_launch_opts o;
    std::memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (o.kernel != IA_KERNEL_PERSISTENT || o.scratch != nullptr || o.scratch_bytes != 0) return IA_ERR_INVALID_ARG;
    const int64_t need = ia_scratch_bytes(n, &o);
    if (need < 0) return (int)need;
    if (need > (int64_t)IA_STATIC_SCRATCH_BYTES) return IA_ERR_TOO_LARGE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return IA_ERR_NO_DEVICE;
    if (dev != sys->device) return IA_ERR_INVALID_ARG;
    void* p = nullptr;
    const int rc = static_scratch_address(dev, &p);
    if (rc != IA_OK) return rc;
    o.scratch = p;
    o.scratch_bytes = (int64_t)IA_STATIC_SCRATCH_BYTES;
    return ia_launch(sys, ic, n, out, &o, stream);
}

extern "C" int ia_static_phases(ia_system* sys, double* lane_ms, double* total_ms, int64_t* errors)
{
    if (!sys || !lane_ms || !total_ms) return IA_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return IA_ERR_NO_DEVICE;
    if (dev != sys->device) return IA_ERR_INVALID_ARG;
    // the counters sit at the start of the array; read them by symbol (no device address needed)
    Counters c;
    if (cudaMemcpyFromSymbol(&c, g_ia_static_scratch, sizeof(Counters), 0, cudaMemcpyDeviceToHost) != cudaSuccess)
        return IA_ERR_CUDA;
    if (c.t_start == 0 || c.t_end < c.t_start) return IA_ERR_INVALID_ARG;
    *lane_ms = c.t_lane_end >= c.t_start ? 1e-6 * (double)(c.t_lane_end - c.t_start) : 0.0;
    *total_ms = 1e-6 * (double)(c.t_end - c.t_start);
    if (errors) *errors = (int64_t)c.errors;
    return IA_OK;
}
