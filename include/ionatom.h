/*
 * ionatom.h -- C ABI of the GB300 (sm_103a) engine for classical ion-atom trajectories.
 *
 * Method: arXiv 2509.15117, "Chaotic scattering and heating in cold ion-atom collisions".
 *   - Eq. 1 (Hamiltonian): one ion in a Paul trap with the per-axis term
 *     (a_j + 2 q_j cos(Omega t)) m_i Omega^2 / 8 x_j^2, one atom, interaction V(|x_a - x_i|);
 *     read with x_j the ion's Cartesian coordinate, and generalised to s cos(Omega t + phi0) with an
 *     rf phase phi0 per trajectory and a sign s (rf_sign, +1 = Eq. 1 as printed).
 *   - Text after Eq. 1: V(r) = C8/r^8 - C4/r^4, C4 = alpha/2; C8 is fixed by the well depth D_e,
 *     C8 = C4^2/(4 D_e). The equations for the twelve variables are integrated with the adaptive
 *     Dormand-Prince 5(4) pair (Dormand & Prince 1980; Shampine & Reichelt 1997, i.e. ode45).
 *   - Head-on paragraph: trajectories start on the sphere of radius r0 and end when the ion-atom
 *     separation crosses r0 outward (or at t_max).
 *   - Fig. 1 caption: observables -- scattering angle between the atom's initial and final velocity,
 *     number of bounces (short-range collisions), momentum transfer |p_f - p_i| of the atom; the
 *     text adds the ion energy change (heating) and complex formation (more than one bounce).
 *
 * Conventions for every entry point:
 *   - Units are atomic units (a0, E_h, m_e, a.u. of time).
 *   - State layout: y = [x_ion(3), v_ion(3), x_atom(3), v_atom(3)].
 *   - Device arrays are structure-of-arrays: component c of trajectory i sits at p[c * ld + i].
 *     Every device pointer must be 8-byte aligned; ld >= n.
 *   - The caller owns every device buffer it passes and the CUDA stream; calls are asynchronous on
 *     that stream (results are valid after the caller synchronises it). The library owns only what
 *     ia_system_create allocates (the parameter table and a work counter), freed by
 *     ia_system_destroy.
 *   - Functions return IA_OK (0) or a negative IA_ERR_* code; no exception crosses the ABI.
 *     ia_error_string() names a code. A CUDA launch failure is reported as IA_ERR_CUDA.
 *   - Per-trajectory failures are not errors of the call: they are status bits in the output.
 */
#ifndef IONATOM_H
#define IONATOM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define IA_OK 0
#define IA_ERR_INVALID_ARG (-1)   /* NULL pointer, n < 0, ld < n, bad option value */
#define IA_ERR_BAD_DESC (-2)      /* a system descriptor fails validation */
#define IA_ERR_CUDA (-3)          /* a CUDA runtime call failed */
#define IA_ERR_ALIGNMENT (-4)     /* a device pointer is not 8-byte aligned */
#define IA_ERR_NO_DEVICE (-5)     /* no CUDA device, or not an sm_103 device */
#define IA_ERR_TOO_LARGE (-6)     /* size beyond a documented limit */

/* ---- per-trajectory status bits (ia_obs_soa.status) ---- */
#define IA_ST_EXIT 0u                 /* separation crossed r0 outward; observables at the crossing */
#define IA_ST_TMAX (1u << 0)          /* reached t_max; observables at t_max */
#define IA_ST_MAX_STEPS (1u << 1)     /* attempted-step cap reached */
#define IA_ST_H_UNDERFLOW (1u << 2)   /* step fell to 16 eps(t) and was still rejected */
#define IA_ST_NONFINITE (1u << 3)     /* a stage produced inf/nan; observables at the last good state */
#define IA_ST_BAD_IC (1u << 4)        /* non-finite initial state, zero separation, bad sys_id */
#define IA_ST_EXIT_OUTSIDE (1u << 5)  /* moving outward beyond r0 with no crossing inside the step */
#define IA_ST_COMPLEX (1u << 8)       /* n_bounce >= 2 (complex formed) */

/* ---- kernels ---- */
#define IA_KERNEL_PLAIN 0       /* one thread per trajectory, one launch per batch */
#define IA_KERNEL_PERSISTENT 1  /* resident grid; finished lanes refill from an atomic work queue */

/* One physical system with its integration settings. */
typedef struct ia_system_desc {
    double m_ion, m_atom;   /* masses, m_e (> 0) */
    double alpha;           /* static dipole polarisability of the atom, a.u. (>= 0); C4 = alpha/2 */
    double De;              /* well depth, E_h (> 0 if alpha > 0); C8 = C4^2 / (4 De) */
    double Omega;           /* rf angular frequency, rad per a.u. of time (> 0) */
    double a[3], q[3];      /* Mathieu parameters per axis */
    double r0;              /* start sphere and exit radius, a0 (> 0) */
    double t_max;           /* a.u. of time (> 0) */
    double rtol;            /* relative tolerance (> 0) */
    double atol_pos;        /* absolute tolerance of positions, a0 (> 0) */
    double atol_vel;        /* absolute tolerance of velocities, a.u. (> 0) */
    double h_max;           /* largest step, a.u. of time (> 0) */
    int32_t rf_sign;        /* +1 (Eq. 1 as printed) or -1 */
    int32_t reserved;       /* must be 0 */
    int64_t max_attempts;   /* cap on attempted steps per trajectory (> 0) */
} ia_system_desc;

typedef struct ia_system ia_system; /* opaque */

/* Initial conditions (device pointers). */
typedef struct ia_ic_soa {
    const double* y0;       /* 12 x ld: initial state at t = 0 */
    const double* phi0;     /* n: rf phase at t = 0 */
    const int32_t* sys_id;  /* n: row of the system table, or NULL for row 0 */
    const int64_t* order;   /* n: persistent launches take trajectories in this order (a permutation of
                               0..n-1, e.g. longest expected first), or NULL for 0..n-1 */
    int64_t ld;             /* leading dimension of y0 (>= n) */
} ia_ic_soa;

/* Observables (device pointers, written for every trajectory). */
typedef struct ia_obs_soa {
    double* theta_s;        /* angle between initial and final atom velocity, rad */
    double* dp;             /* |p_f - p_i| of the atom, a.u. */
    double* dE_ion;         /* E_ion(t_f) - E_ion(0), E_ion = kinetic + trap term of Eq. 1, E_h */
    double* t_final;        /* time of the crossing (or of the stop), a.u. */
    double* t_first_bounce; /* end time of the step containing the first pericentre (0 if none) */
    double* t_last_bounce;  /* same for the last pericentre */
    int32_t* n_bounce;      /* pericentre passages: d.(v_a - v_i) from < 0 to >= 0 */
    uint32_t* status;       /* IA_ST_* bits */
    int32_t* n_steps;       /* accepted steps */
    int32_t* n_rej;         /* rejected steps */
    double* y_final;        /* 12 x ld final state, or NULL */
    int64_t ld;             /* leading dimension of y_final (>= n) */
} ia_obs_soa;

/* Launch options; zero-initialised means defaults. */
typedef struct ia_launch_opts {
    int32_t kernel;             /* IA_KERNEL_PLAIN (default) or IA_KERNEL_PERSISTENT */
    int32_t block;              /* persistent: threads per block, 64, 128 or 256; 0 = 128 (plain: 128) */
    int32_t grid;               /* persistent: blocks; 0 = resident blocks per SM x SMs */
    int32_t refill;             /* persistent: idle lanes in a warp before it claims work, 1..32; 0 = 1 */
    int32_t blocks_per_sm;      /* persistent: resident blocks per SM to use when grid = 0; 0 = max */
    int32_t regs_variant;       /* persistent: 1 = no register cap (default, 0 means 1); 3 = build capped
                                   for 3 resident 128-thread blocks per SM (block must be 128) */
    int32_t slice_budget;       /* persistent: attempted steps after which a trajectory is handed to the
                                   group-mode tail; 0 = 131072; -1 = never (no tail) */
    int32_t tail_group;         /* lanes per trajectory in the tail kernel: 6 or 8; 0 = 6 */
    int32_t tail_blocks_per_sm; /* blocks (128 threads) per SM of the clean-up tail kernel, 1..16; 0 = 1 */
    int32_t tail_sms;           /* persistent: SMs whose single block works on suspended trajectories from
                                   the start, 1..192 (at most half the SMs are used); 0 = 32; -1 = none */
    int32_t tail_pair;          /* persistent, tail_group 6: 1 = on the reserved SMs, two warps on two sub-
                                   partitions advance the same trajectories together (a single long
                                   trajectory steps 1.3x faster, but each SM holds half as many;
                                   bit-identical results); 0 or -1 = off (default) */
    int32_t tail_warps;         /* persistent: warps of each reserved SM's block that work on the tail, 1..8
                                   and at most block/32; 0 = 4 (one per SM sub-partition: a long
                                   trajectory's latency in group mode is its FP64 instruction count, so a
                                   tail warp steps fastest with an FP64 unit to itself; 8 trades latency
                                   for tail throughput). Further warps of that block leave */
    int64_t suspend_capacity;   /* suspend records; 0 = min(n, max(4096, n/32)). A trajectory that finds
                                   no free record is finished by its lane. */
    void* scratch;              /* persistent: caller's device scratch (256-byte aligned), or NULL to use
                                   the system's own, grown by ia_launch when needed */
    int64_t scratch_bytes;      /* size of `scratch`; at least ia_scratch_bytes(n, opts) */
} ia_launch_opts;

/*
 * Create a table of n_sys systems on the current CUDA device (copied to device memory).
 * Validation per row: masses, Omega, r0, t_max, tolerances, h_max > 0; alpha >= 0; De > 0 when
 * alpha > 0; rf_sign = +-1; max_attempts > 0; reserved = 0; |a_j|, |q_j| <= 16, and every axis
 * Mathieu-stable: with tau = (Omega t + phi0)/2, Eq. 1 gives x'' + (a_j + 2 q_j cos 2 tau) x = 0 per
 * axis, whose monodromy matrix over one rf period must have a trace within [-2, 2] (to 1e-8; the free
 * axis a_j = q_j = 0 has trace 2 and is accepted). Returns IA_ERR_BAD_DESC on failure and writes
 * nothing to *out. The checks run before any CUDA call. n_sys must be 1..65536.
 * Derived constants (text after Eq. 1): C4 = alpha/2, C8 = C4^2/(4 De).
 */
int ia_system_create(const ia_system_desc* desc, int32_t n_sys, ia_system** out);

/* Free a system table. NULL is accepted. The caller must make sure no launch using it is in flight. */
int ia_system_destroy(ia_system* sys);

/* Number of rows of a system table, or a negative code. */
int ia_system_count(const ia_system* sys);

/*
 * Scratch bytes a persistent launch of n trajectories with these options needs (counters and the
 * suspend records of trajectories moved to the tail kernel), or a negative code.
 */
int64_t ia_scratch_bytes(int64_t n, const ia_launch_opts* opts);

/*
 * Grow the system's own scratch to what a launch of n trajectories with opts needs (cudaMalloc;
 * synchronous). Call it before capturing ia_launch into a CUDA graph when opts->scratch is NULL.
 */
int ia_reserve(ia_system* sys, int64_t n, const ia_launch_opts* opts);

/*
 * Integrate n trajectories and write their observables (Eq. 1 with V, DP5(4), exit at r0, the
 * Fig. 1 observables). Asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream).
 * n = 0 is a no-op. opts may be NULL (defaults).
 * Persistent launches: a trajectory that has used opts->slice_budget attempted steps is saved to a
 * suspend record and finished by tail workers that give each such trajectory a group of lanes, which
 * run its steps ~2.2x faster; tail workers start at once on opts->tail_sms SMs and every other warp
 * joins them once the queue is drained (one cooperative launch, every wait bounded). Results are
 * bit-identical to the plain kernel.
 * Concurrency: persistent launches that share the system's own scratch must not overlap; pass a
 * distinct opts->scratch to run them concurrently.
 */
int ia_launch(ia_system* sys, const ia_ic_soa* ic, int64_t n, const ia_obs_soa* out,
              const ia_launch_opts* opts, void* stream);

/*
 * Allocation-free variant of the persistent launch (no counterpart in the paper; it exists for
 * callers that cannot allocate device memory when they launch: code recording a CUDA graph, where
 * cudaMalloc is not allowed during capture; plug-ins inside a host program that owns all device
 * memory through its own pool; real-time loops that forbid allocation after start-up).
 *
 * Same arguments, results and asynchrony as ia_launch with opts->kernel = IA_KERNEL_PERSISTENT
 * (required; opts->scratch must be NULL and scratch_bytes 0). Its scratch is a fixed device array of
 * IA_STATIC_SCRATCH_BYTES in the library, which every GPU that loads the library keeps until the
 * process exits. It calls no cudaMalloc or cudaFree.
 *   - Limit: ia_scratch_bytes(n, opts) must not exceed IA_STATIC_SCRATCH_BYTES (room for the counters
 *     and 16128 suspend records); otherwise IA_ERR_TOO_LARGE and nothing runs. For large batches set
 *     opts->suspend_capacity <= 16128 (trajectories that find no record finish in their lanes).
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with that
 *     device current; make that first call before any stream capture. A device reset (cudaDeviceReset)
 *     moves the array: the first call after it looks the address up again, so it too must come before
 *     any capture. The current device must be the one the system table was created on (else
 *     IA_ERR_INVALID_ARG).
 *   - Every call shares the one array and leaves its contents behind; the counters it needs at zero
 *     are cleared on the stream at the start of each call. Calls whose work overlaps on the GPU
 *     (other streams, other host threads) race on the array: serialise them.
 */
#define IA_STATIC_SCRATCH_BYTES (4u << 20)
int ia_launch_static(ia_system* sys, const ia_ic_soa* ic, int64_t n, const ia_obs_soa* out,
                     const ia_launch_opts* opts, void* stream);

/*
 * ia_launch_phases for the allocation-free launch (no counterpart in the paper): the phase times and
 * the count of bounded waits that ran out (*errors, if not NULL; 0 in a healthy run, otherwise some
 * trajectories may have no result) of the last ia_launch_static on the current device, read from the
 * library's fixed array. Synchronous (call it after that launch completed); allocates nothing.
 * IA_ERR_INVALID_ARG if the current device is not the system's or the array holds no completed launch.
 */
int ia_static_phases(ia_system* sys, double* lane_ms, double* total_ms, int64_t* errors);

/* ---- one batch integrated over several launches ---- */

/*
 * A work queue of one batch of n trajectories, integrated by a sequence of persistent launches
 * ("parts"). Trajectory lengths in a batch are heavy-tailed: most atoms leave after one bounce,
 * while complexes live up to the run's t_max (Fig. 2 passage: complexes alive past 600 us; the text
 * after Eq. 1 puts the average at ~3e5 steps). A single launch over a large batch therefore lasts as
 * long as its longest trajectory. A queue lets each launch do a bounded share of the batch instead:
 *   - part k starts the next `count` queue positions (in ic->order, or 0..n-1);
 *   - first it resumes, in lane mode, the trajectories the previous part left running;
 *   - trajectories past opts->slice_budget attempted steps go to suspend records and run in group mode
 *     on the reserved SMs, across parts, exactly as in ia_launch;
 *   - a part that does not take the last queue positions ends as soon as its queue is exhausted: every
 *     running trajectory is saved (lane mode: a lane-mode carry record; group mode: a group-mode carry
 *     record, or a suspend record when those are full) and the next part continues it where it
 *     stopped, its group-mode carry records before any suspend record;
 *   - the part that takes the last positions finishes every trajectory before it returns.
 * Results are bit-identical to ia_launch (the plain kernel) whatever the split. A trajectory's
 * observables are written by the part in which it ends; after the last part all n are written.
 *
 * ia_queue_create: fixes the launch options (kernel persistent; opts->scratch must be NULL and
 *   opts->tail_pair not 1: the paired tail is not available here) and allocates the queue's device
 *   scratch (cudaMalloc, synchronous): counters, suspend records as in ia_scratch_bytes(n, opts), two
 *   lane-mode carry buffers of one 256-byte record per lane of the grid, and two group-mode carry
 *   buffers of 5 records per tail warp. Every block of the grid must be
 *   resident (cooperative launch); otherwise IA_ERR_INVALID_ARG (a grid too large) or IA_ERR_NO_DEVICE.
 *   n >= 1.
 * ia_queue_launch: launches the next part on `stream` (asynchronous). ic and out describe the whole
 *   batch (n trajectories, ld >= n) and must be the same arrays in every part of a batch (else
 *   IA_ERR_INVALID_ARG); their contents may be written between parts (e.g. the inputs of the next
 *   part's positions copied in), but the inputs of a trajectory that has started must not change until
 *   its result is written. 0 <= count <= n - started; count = 0 continues the running trajectories
 *   only. The part whose count reaches n is the last. A complete batch takes no further part until
 *   ia_queue_reset. Parts of one queue must run in order on one stream (each reads what the previous
 *   wrote).
 * ia_queue_reset: starts a new batch of the same size and options (host state only; the next part
 *   clears the device counters on its stream). No part of the queue may be in flight on another stream.
 * ia_queue_state: queue positions started so far, parts launched, and n (any pointer may be NULL).
 * ia_queue_phases: as ia_launch_phases, for the latest part (synchronous).
 * ia_queue_destroy: frees the queue (NULL accepted); no part may be in flight.
 */
typedef struct ia_queue ia_queue; /* opaque */
int ia_queue_create(ia_system* sys, int64_t n, const ia_launch_opts* opts, ia_queue** q);
int ia_queue_launch(ia_queue* q, const ia_ic_soa* ic, const ia_obs_soa* out, int64_t count, void* stream);
int ia_queue_reset(ia_queue* q);
int ia_queue_state(const ia_queue* q, int64_t* started, int64_t* parts, int64_t* n);
int ia_queue_phases(const ia_queue* q, double* lane_ms, double* total_ms, int64_t* errors);
int ia_queue_destroy(ia_queue* q);

/*
 * Phase times of the last persistent launch whose scratch is `scratch` (NULL: the system's own
 * scratch), from the device clock: *lane_ms = from the first block's start until the last warp left
 * the lane phase (every trajectory had started and had either finished or been handed to the tail
 * phase), *total_ms = until the last warp finished. *errors (if not NULL) = bounded waits of that
 * launch that ran out (0 in a healthy run; otherwise some trajectories may have no result).
 * Synchronous (copies the launch's counters from the device; call it after the launch completed).
 * A diagnostic of how a batch's time splits between the bulk of short trajectories and the
 * long-lived complexes; no counterpart in the paper. IA_ERR_INVALID_ARG if that scratch holds no
 * completed persistent launch.
 */
int ia_launch_phases(ia_system* sys, const void* scratch, double* lane_ms, double* total_ms, int64_t* errors);

/*
 * FP64 FMA throughput microbenchmark (no counterpart in the paper: it measures the roofline
 * denominator of the integrator). Runs `blocks_per_sm` x SMs blocks of 256 threads, each thread
 * `iters` iterations of 8 independent fused multiply-add chains, on `stream`, timed with CUDA
 * events around the launch; synchronises the stream. *flops = 2 * 8 * iters * threads / seconds.
 */
int ia_fp64_peak(int32_t blocks_per_sm, int32_t iters, void* stream, double* flops);

/* ---- batch statistics ---- */
#define IA_STATS_BOUNCE_BINS 32
#define IA_STATS_LIFETIME_BINS 64
#define IA_STATS_EXIT_SLOT 6
#define IA_STATS_MAX_CELLS 1024

/* Per-cell ensemble statistics: the quantities of the paper's Fig. 3 and Fig. 4 (probability of
 * complex formation), Fig. 1c (bounce counts) and Fig. 2 (complex lifetimes), plus ion heating. */
typedef struct ia_stats {
    int64_t n;                 /* trajectories in the cell */
    int64_t n_complex;         /* trajectories with n_bounce >= 2 */
    int64_t attempts;          /* attempted steps (accepted + rejected) */
    int64_t n_status[8];       /* [b], b = 0..5: trajectories with status bit b (IA_ST_TMAX .. IA_ST_EXIT_OUTSIDE);
                                  [IA_STATS_EXIT_SLOT]: clean exits (low status byte 0); [7]: 0 */
    int64_t bounce_hist[IA_STATS_BOUNCE_BINS];     /* [0]: no bounce; [k >= 1]: 2^(k-1) <= n_bounce < 2^k
                                                      (last bin open-ended) */
    int64_t lifetime_hist[IA_STATS_LIFETIME_BINS]; /* complexes by tau = t_last_bounce - t_first_bounce:
                                                      bin k = floor(2 (log2 tau - 20)), clamped to 0..63 */
    double sum_dE;             /* sum of dE_ion, added in a fixed order (bit-reproducible) */
    double sum_dE2;            /* sum of dE_ion^2, same order */
} ia_stats;

/*
 * Reduce the observables of n trajectories into n_cells ia_stats records (device array `stats`,
 * caller-owned, overwritten). cell_id: device array of n cell indices in 0..n_cells-1 (others are
 * skipped), or NULL to put every trajectory in cell 0. n_cells: 1..IA_STATS_MAX_CELLS. Uses the
 * system's scratch (grown synchronously when too small; call ia_reserve_stats before a capture).
 * Asynchronous on `stream`.
 */
int ia_reduce_stats(ia_system* sys, const ia_obs_soa* obs, int64_t n, const int32_t* cell_id, int32_t n_cells,
                    ia_stats* stats, void* stream);

/* Grow the system's statistics scratch for n trajectories and n_cells cells (synchronous). */
int ia_reserve_stats(ia_system* sys, int64_t n, int32_t n_cells);

/* ---- CUDA graph of one batch ---- */
typedef struct ia_graph ia_graph; /* opaque */

/*
 * Capture one persistent launch (ia_launch with opts, kernel forced to IA_KERNEL_PERSISTENT) followed,
 * if stats is not NULL, by ia_reduce_stats into a CUDA graph on `stream` (a stream created by the
 * caller; the legacy default stream cannot be captured), and instantiate it. Scratch is reserved
 * first. All pointers are baked into the graph: replays read the same input buffers and write the same
 * outputs, so the caller refills the inputs between replays. Nothing runs until ia_graph_launch.
 */
int ia_graph_create(ia_system* sys, const ia_ic_soa* ic, int64_t n, const ia_obs_soa* out,
                    const ia_launch_opts* opts, const int32_t* cell_id, int32_t n_cells, ia_stats* stats,
                    void* stream, ia_graph** graph);
/* Replay the captured batch on `stream`. */
int ia_graph_launch(ia_graph* graph, void* stream);
/* Free a graph (NULL accepted); no replay may be in flight. */
int ia_graph_destroy(ia_graph* graph);

/*
 * Autotuner of the persistent kernel's lane phase (block size, register cap, refill grain). Each
 * candidate integrates the n trajectories of `ic` (a sample of the batch to tune for) with every
 * trajectory stopped after `attempt_cap` attempted steps (no tail phase, outputs not written), timed
 * with CUDA events on `stream`, twice (interleaved with the other candidates; the shorter time counts);
 * every candidate does the same arithmetic, so the fastest has the highest lane-phase throughput.
 * Candidates within 1 % of the fastest count as equal, and among them the smallest refill grain wins
 * (then the fastest): in the sample every trajectory stops at the same cap, which hides what a lazier
 * refill costs in a batch of spread lengths.
 * Writes the winner into *best (other fields copied from *base, which may be NULL) and its time in
 * *best_ms. Synchronous. attempt_cap: 64..1048576.
 */
int ia_autotune(ia_system* sys, const ia_ic_soa* ic, int64_t n, int32_t attempt_cap, const ia_launch_opts* base,
                ia_launch_opts* best, double* best_ms, void* stream);

/* ---- tangent (forward-mode) differentiation and FTLE ---- */

/* Tangent seeds: up to 4 directions p_k, each given by d y0 / d p_k per trajectory and by the
 * derivative of the trap's q vector (same for every trajectory of the launch). */
typedef struct ia_tangent_in {
    const double* dy0;      /* device, ndir x 12 x ld: d y0[c] / d p_k of trajectory i at dy0[(k*12 + c)*ld + i] */
    double dq[4][3];        /* d q_j / d p_k (host values) */
    int32_t ndir;           /* 1..4 */
    int32_t reserved;       /* must be 0 */
    int64_t ld;             /* >= n */
} ia_tangent_in;

/* Tangent results (device pointers), direction k of trajectory i at [k*ld + i]. */
typedef struct ia_tangent_out {
    double* d_theta_s;      /* d theta_s / d p_k */
    double* d_dp;           /* d |p_f - p_i| / d p_k */
    double* d_dE_ion;       /* d dE_ion / d p_k */
    double* d_t_final;      /* d t_final / d p_k */
    double* dy_final;       /* ndir x 12 x ld: d y_final / d p_k, or NULL */
    double* ftle;           /* ld: finite-time Lyapunov exponent along direction 0, per a.u. of time, in the
                               norm with positions in units of r_e and velocities in sqrt(2 D_e/mu);
                               or NULL */
    int64_t ld;             /* >= n */
} ia_tangent_out;

/*
 * Integrate n trajectories (as ia_launch, same primal results bit for bit) together with the
 * discrete tangent of the DP5(4) map along up to four directions: step sizes and accept/reject
 * decisions of the primal are held fixed; the exit time gets its own sensitivity from the
 * continuous extension (d s_star / d p = -(d . dd/dp) / (d . dd/ds)). Derivatives of theta_s, dp, dE_ion and
 * t_final follow by the chain rule. No counterpart in the paper's text, which measures chaos through
 * fractal maps and lifetimes; the FTLE output gives the finite-time Lyapunov exponent for those maps.
 * One warp per trajectory. Asynchronous on `stream`; uses the system's scratch for a work counter.
 */
int ia_launch_tangent(ia_system* sys, const ia_ic_soa* ic, int64_t n, const ia_obs_soa* out,
                      const ia_tangent_in* tin, const ia_tangent_out* tout, void* stream);

/* ---- adjoint (reverse-mode) differentiation ---- */

/* Options of ia_launch_adjoint; zero-initialised means defaults. */
typedef struct ia_adjoint_opts {
    int32_t seg;            /* committed steps between checkpoints, and the length of a recomputed block;
                               16..1000000; 0 = 10000 */
    int32_t max_ckpt;       /* checkpoints kept per trajectory, even, 2..1048576; 0 = 64. A trajectory
                               longer than seg x max_ckpt steps drops every other checkpoint and doubles
                               the spacing (memory fixed, recomputation grows) */
    int64_t warps;          /* trajectories in flight, one warp each; 0 = resident warps; capped at n */
    void* scratch;          /* device scratch (256-byte aligned) of at least ia_adjoint_scratch_bytes, or
                               NULL to use the system's own, grown by the launch when needed */
    int64_t scratch_bytes;  /* size of `scratch` */
} ia_adjoint_opts;

/* Adjoint results (device pointers). Objectives J_m: m = 0 theta_s, 1 |p_f - p_i|, 2 dE_ion, 3 t_final. */
typedef struct ia_adjoint_out {
    double* grad_y0;        /* 4 x 12 x ld: d J_m / d y0[c] of trajectory i at [(m*12 + c)*ld + i], or NULL */
    double* grad_q;         /* 4 x 3 x ld: d J_m / d q_j at [(m*3 + j)*ld + i], or NULL */
    double* d_theta_s;      /* ndir x ld: the gradients projected on the seeds (as ia_tangent_out);   */
    double* d_dp;           /*   required when seeds are given, ignored otherwise                     */
    double* d_dE_ion;
    double* d_t_final;
    int64_t ld;             /* >= n */
} ia_adjoint_out;

/*
 * Device scratch an adjoint launch of n trajectories needs: 256 bytes of counters, then per warp in
 * flight max_ckpt checkpoints of 256 bytes and a step buffer of seg x 128 bytes. sys may be NULL when
 * opts->warps > 0. Returns the size or a negative code.
 */
int64_t ia_adjoint_scratch_bytes(const ia_system* sys, int64_t n, const ia_adjoint_opts* opts);

/*
 * Integrate n trajectories (as ia_launch, same primal observables bit for bit) and compute, by a
 * reverse sweep, the gradients of theta_s, |p_f - p_i|, dE_ion and t_final with respect to the initial
 * state and the trap's q vector. The map differentiated is the one ia_launch_tangent differentiates
 * (step sizes and decisions held fixed; exit-time sensitivity from the continuous extension), so
 * for any direction p, grad . (dy0/dp, dq/dp) equals the tangent's derivative up to rounding. The
 * paper has no counterpart: it studies the sensitivity of these observables to the initial
 * conditions through fractal maps; the gradients give that sensitivity per trajectory.
 * Method: the forward pass keeps checkpoints of the complete controller state every opts->seg
 * committed steps; the reverse pass restores the checkpoint below each block of seg steps, replays
 * the primal (same decisions) to record the block, and pulls the adjoint back through each DP5 step.
 * Cost: about four primal integrations (forward, replay, adjoint stages).
 * seeds (may be NULL): up to 4 directions (ia_tangent_in) whose projections are written to
 * d_theta_s .. d_t_final. At least one of grad_y0, grad_q or seeds is required.
 * A trajectory whose replay does not reproduce its forward pass (not expected: the arithmetic is
 * deterministic) gets NaN derivatives; one with a bad initial state or sys_id gets zeros.
 * Scratch: opts->scratch, else the system's own (cudaMalloc when it must grow: synchronous).
 * One warp per trajectory. Asynchronous on `stream`; launches sharing the system's own adjoint
 * scratch must not overlap.
 */
int ia_launch_adjoint(ia_system* sys, const ia_ic_soa* ic, int64_t n, const ia_obs_soa* out,
                      const ia_tangent_in* seeds, const ia_adjoint_out* aout, const ia_adjoint_opts* opts,
                      void* stream);

/* ---- initial conditions drawn on the device ---- */

#define IA_SAMPLE_HEAD_ON 0  /* head-on runs: ion at rest at the centre; atom at r0 x_hat moving at -v0 x_hat,
                                E = m_a v0^2 / 2, x_hat uniform on the octant's surface (cos theta = u1,
                                phi = (pi/2) u2) */
#define IA_SAMPLE_SPHERE 1   /* thermal runs as the paper draws them: atom uniform on the r0 sphere
                                (cos theta = 2 u1 - 1, phi = 2 pi u2), velocity components Gaussian with
                                variance kT/m_a, the vector negated where v . x_hat >= 0; thermal ion */
#define IA_SAMPLE_DISK 2     /* thermal runs with the impact parameter uniform over a disk: atom velocity as
                                above; b = b_max sqrt(u1) at azimuth psi = 2 pi u2 about v_hat, measured from
                                e1 = unit(v_hat x r) (r = z_hat if |v_hat_z| < 0.9, else x_hat) toward
                                e2 = v_hat x e1; x_a = b (cos psi e1 + sin psi e2) - sqrt(r0^2 - b^2) v_hat;
                                thermal ion */

/* Parameters of a sampler. The masses, Omega, q, r0 and rf_sign are those of the system the
 * trajectories will be integrated in. */
typedef struct ia_sampler {
    int32_t kind;          /* IA_SAMPLE_* */
    int32_t random_phase;  /* 1: phi0 = 2 pi u0, uniform on (0, 2 pi) (Fig. 4 caption); 0: phi0 = phase */
    int32_t micromotion;   /* thermal kinds, 0 or 1: add the ion's lowest-order micromotion at phi0,
                              x_j = X_j (1 + s q_j/2 cos phi0), v_j = V_j (1 + s q_j/2 cos phi0)
                              - X_j s (q_j Omega/2) sin phi0 */
    int32_t rf_sign;       /* s: +1 or -1 */
    double m_ion, m_atom;  /* m_e (> 0) */
    double Omega;          /* rad per a.u. of time */
    double q[3];           /* Mathieu q per axis */
    double r0;             /* start sphere, a0 (> 0) */
    double E;              /* head-on: collision energy, E_h (> 0) */
    double kT;             /* thermal kinds: k_B T of the atom, E_h (> 0) */
    double kT_ion;         /* thermal kinds: k_B T of the ion, E_h (>= 0; 0 = at rest at the centre). The
                              secular position X_j and velocity V_j are Gaussian with variances
                              kT_ion/(m_ion omega^2) and kT_ion/m_ion, omega = |q_x| Omega / 2^(3/2) (> 0
                              when kT_ion > 0) */
    double b_max;          /* disk: radius, a0, 0 <= b_max < r0 */
    double phase;          /* phi0 when random_phase = 0 */
    uint64_t seed;         /* word 0 of the generator's key (word 1 is the kind) */
} ia_sampler;

/*
 * Raw generator (no counterpart in the paper): Philox4x64-10 (Salmon, Moraes, Dror & Shaw, SC'11).
 * Block j, j = 0 .. n_blocks - 1, is the ten-round map of the counter (first + j, ctr1, 0, 0) under the
 * key (key0, key1); its four words go to out[4j .. 4j + 3] (device array, 8-byte aligned).
 * first >= 0 and first + n_blocks must not overflow (else IA_ERR_INVALID_ARG). Asynchronous on `stream`.
 */
int ia_philox4x64(uint64_t key0, uint64_t key1, uint64_t ctr1, int64_t first, int64_t n_blocks, uint64_t* out,
                  void* stream);

/*
 * Draw the initial conditions of trajectories first .. first + n - 1 on the device: y0 (12 x ld, the
 * layout of ia_ic_soa.y0) and phi0 (n) get the state at t = 0 and the rf phase of trajectory
 * first + i in column i. Initial conditions as the paper's runs draw them (head-on paragraph, thermal
 * paragraph, Fig. 3 and Fig. 4 captions); see IA_SAMPLE_*.
 * Random numbers: trajectory g uses the Philox4x64-10 blocks of the counters (g, j, 0, 0), j = 0..3,
 * under the key (seed, kind). Word w of block j gives u[4j + w] = ((word >> 11) | 1) 2^-53, in (0, 1).
 *   - u0 is the rf phase, u1 and u2 the direction or the disk point;
 *   - u4 .. u13 are five Box-Muller pairs g[2p] = sqrt(-2 ln u[4+2p]) cos(2 pi u[5+2p]), g[2p+1] the sine;
 *   - g0..g2 scale to the atom velocity, g3..g5 to the ion's secular position, g6..g8 to its secular
 *     velocity.
 * A trajectory's values depend only on its index, the seed and the kind: any index range can be drawn
 * alone (in chunks, or one range per rank) and matches the whole batch. n = 0 is a no-op.
 * IA_ERR_INVALID_ARG for a parameter out of the ranges above, or when ld < n; IA_ERR_ALIGNMENT for
 * unaligned pointers; IA_ERR_NO_DEVICE when the current device is not an sm_103 GPU. Nothing is written
 * when a check fails. Asynchronous on `stream`.
 */
int ia_sample_ics(const ia_sampler* s, int64_t first, int64_t n, double* y0, double* phi0, int64_t ld,
                  void* stream);

/*
 * Test hook (no counterpart in the paper): y[i] = 1/x[i] computed as the integrator computes 1/r^2
 * (Newton-Raphson from an FP32 seed). x, y: device arrays of n doubles, x[i] > 0. Asynchronous.
 */
int ia_rcp_check(const double* x, double* y, int64_t n, void* stream);

/* Static description of a return code (never NULL). */
const char* ia_error_string(int code);

/* Library version, e.g. 100 for 0.1.0. */
int ia_version(void);

#ifdef __cplusplus
}
#endif

#endif /* IONATOM_H */
