"""Benchmark: trajectories/s and RHS evaluations/s of the ion-atom trajectory engine (FP64, rtol 1e-10).

Workload: the head-on species x energy sweep (Yb+ with Li, Na, K, Rb, Cs; 8 energies log-spaced from
1 uK to 1 mK; D_e = 1 K, q = 0.1, a = 0, t_max = 1 ms) on the cell-centred 1024 x 1024 (theta, phi)
octant grid. One step integrates one batch: by default (stride 1) the whole configuration, 41,943,040
trajectories of all 40 (species, energy) systems; with --stride S every S-th grid point in each
direction, the grid offset advancing every step so that successive steps see different trajectories. Trajectory lengths differ by 10-100x, so the persistent kernel with work-queue
refill is the timed path; the plain one-thread-per-trajectory kernel is timed on a subsample of the
same batch for the speedup. Each timed step copies its inputs from pinned host memory, flushes L2,
launches (device-timed with CUDA events: `value`) and copies the observables back (the whole step:
`e2e`).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--stride S]
Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2509_15117_gb300 import inputs as I  # noqa: E402

METRIC = "trajectories/s and RHS evals/s at rtol 1e-10 FP64, plain vs batched/adjoint"
UNIT = "trajectories/s"
GRID = 1024

# FP64 floating-point operations per attempted DP5 step of the one-lane-per-trajectory arithmetic
# (fused multiply-add = 2), counted by ncu's per-thread FP64 instruction counters (2 dfma + dmul + dadd,
# predicated-on threads) on the persistent kernel's lane phase (the bulk-only profile case, where no
# trajectory reaches the tail), divided by the attempted steps of that launch; the cos and reciprocal
# instruction sequences are included. The tail phase spreads one trajectory over six lanes and
# executes more FP64 instructions in total, so this is the useful work per attempt.
FLOPS_PER_ATTEMPT = 884.0
# DRAM bytes per trajectory of the persistent kernel (read + write, ncu dram__bytes on the 512 x 512
# bulk-only profile case: 39.0 MB for 262,144 trajectories): initial conditions in, observables out.
DRAM_BYTES_PER_TRAJECTORY = 148.8


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--stride", type=int, default=1, help="grid stride of the batch (1: the whole sweep)")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--order", choices=("cost", "threshold"), default="cost",
                   help="queue order of the sweep's systems: cost (sqrt(m_a)/v0 descending) or threshold "
                        "(E / W0^3D ascending: the complex-forming systems first)")
    p.add_argument("--dump-long", default="",
                   help="write the queue position, system and attempted steps of every trajectory above "
                        "2^17 attempts, with the part bounds and device times, to this .npz file")
    p.add_argument("--last-part", type=float, default=0.0,
                   help="fraction of the queue in the last part (0: equal parts)")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--block", type=int, default=0)
    p.add_argument("--refill", type=int, default=0)
    p.add_argument("--blocks-per-sm", type=int, default=0)
    p.add_argument("--regs-variant", type=int, default=0)
    p.add_argument("--slice-budget", type=int, default=0)
    p.add_argument("--tail-group", type=int, default=0)
    p.add_argument("--tail-blocks-per-sm", type=int, default=0)
    p.add_argument("--tail-sms", type=int, default=0)
    p.add_argument("--tail-warps", type=int, default=0)
    p.add_argument("--diff-sample", type=int, default=16384,
                   help="trajectories of the differentiation workload timed through the tangent and adjoint "
                        "kernels (0: skip)")
    p.add_argument("--diff-cap", type=int, default=1 << 16,
                   help="attempted steps after which each trajectory of that side measurement stops (0: none)")
    p.add_argument("--workload-cap", type=int, default=0,
                   help="with --workload diff: attempted steps after which each trajectory stops (0: none)")
    p.add_argument("--workload", default="sweep",
                   choices=["sweep", "thermal", "mixed-graph", "ftle", "diff", "sampler", "energy-scan",
                            "thermal-sweep", "lifetimes"],
                   help="sweep: the species x energy step (the bench line); thermal: the Monte Carlo bath; "
                        "mixed-graph: the 250-cell parameter sweep replayed as one CUDA graph with statistics; "
                        "ftle: the tangent kernel on the FTLE grid; diff: tangent and adjoint kernels on the "
                        "differentiation workload (uncapped); sampler: initial conditions drawn on the "
                        "device; energy-scan: the collision-energy scan with device-drawn initial conditions, "
                        "per-cell statistics and the threshold fit; thermal-sweep: the species x T x D_e "
                        "thermal runs with the paper's sphere sampler on the device; lifetimes: complex "
                        "lifetimes per species and the fit of their tail")
    p.add_argument("--scale", type=float, default=0.0, help="size factor of the secondary workloads")
    p.add_argument("--sampler-sample", type=int, default=1 << 24,
                   help="trajectories whose initial conditions are drawn on the device, per sampler kind, "
                        "in a timed side measurement (0: skip)")
    p.add_argument("--profile-case", action="store_true",
                   help="run the persistent and plain kernels once on a small batch (for ncu) and exit")
    p.add_argument("--profile-grid", type=int, default=64,
                   help="(theta, phi) grid points per direction of the profile case")
    return p.parse_args(argv)


def profile_case(n_grid: int = 64):
    """Small fixed case for ncu captures: head-on Rb trajectories at 1 mK on an n_grid x n_grid octant
    grid (short, single-bounce dominated; 64 x 64 = 4096 leaves most lanes idle and shows the latency
    of one wave, 512 x 512 = 262144 fills every lane several times and shows the bulk phase), run by
    the persistent kernel (default budget: its tail phase gets no work), by the persistent kernel with
    a 300-step budget (the tail phase finishes almost every trajectory) and by the plain kernel."""
    import torch
    from paper_2509_15117_gb300 import binding as Bd
    systems = I.c2_systems()
    rb_hot = [s for (sp, E, s) in systems if sp == "Rb"][-1]
    th, ph = I.octant_grid(n_grid)
    v0 = I.speed_for_energy(I.kelvin(I.C2_ENERGIES_K[-1]), rb_hot.m_atom)
    y0 = I.head_on(th, ph, rb_hot.r0, v0)
    with Bd.System([rb_hot.as_dict()]) as S:
        for kernel, kw in ((Bd.IA_KERNEL_PERSISTENT, {}), (Bd.IA_KERNEL_PERSISTENT, {"slice_budget": 300}),
                           (Bd.IA_KERNEL_PLAIN, {})):
            out = S.run(y0, np.zeros(len(y0)), None, kernel=kernel, **kw)
    torch.cuda.synchronize()
    n = int(out["n_steps"].sum().item() + out["n_rej"].sum().item())
    print(json.dumps({"profile_case": f"Rb 1 mK head-on {n_grid}x{n_grid}", "trajectories": len(y0),
                      "attempted_steps": n}))


def diff_bench(n: int, flush, cap: int = 0):
    """Tangent (4 seeds + FTLE) and adjoint (4 objectives, projected on the same seeds) launches on the
    first n trajectories of the differentiation workload (Yb+-Rb head-on, 1.5 uK, (theta, phi) uniform
    on the octant, seed 5), each timed with CUDA events after a warm-up launch on 64 of them, next to
    the persistent primal launch on the same trajectories. cap > 0 stops every trajectory after that
    many attempted steps (the same in all three launches), so that the measurement is bounded by
    throughput rather than by the few longest complexes."""
    import torch
    from paper_2509_15117_gb300 import binding as Bd
    sysd, y0, phi0, seeds, dq = I.c5_workload(n)
    dy0 = np.concatenate([seeds, np.zeros((n, 1, 12))], axis=1)
    stream = torch.cuda.current_stream()
    res = {}
    desc = sysd.as_dict()
    if cap > 0:
        desc["max_attempts"] = int(cap)
    with Bd.System([desc]) as S:
        def run(kind, m):
            y, p, _ = Bd.to_device_soa(y0[:m], phi0[:m], None)
            dyd = torch.from_numpy(np.ascontiguousarray(np.transpose(dy0[:m], (1, 2, 0)))).cuda()
            out = Bd.alloc_obs(m)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if kind == "tangent":
                tan = Bd.alloc_tangent(m, 4)
                flush.zero_()
                e0.record(stream)
                Bd.ia_launch_tangent(S.handle, y, p, None, out, dyd, dq, tan)
            elif kind == "adjoint":
                adj = Bd.alloc_adjoint(m, 4)
                flush.zero_()
                e0.record(stream)
                Bd.ia_launch_adjoint(S.handle, y, p, None, out, adj, dyd, dq)
            else:
                flush.zero_()
                e0.record(stream)
                Bd.ia_launch(S.handle, y, p, None, out)
            e1.record(stream)
            torch.cuda.synchronize()
            att = int((out["n_steps"].to(torch.int64) + out["n_rej"].to(torch.int64)).sum().item())
            return e0.elapsed_time(e1), att
        for kind in ("primal", "tangent", "adjoint"):
            run(kind, 64)
            ms, att = run(kind, n)
            res[kind] = (ms, att)
    wl = ("Yb+-Rb head-on, E = 1.5 uK, D_e = 1 K, q = 0.1, t_max = 1 ms, (theta, phi) uniform on the "
          f"octant (seed 5), first {n} trajectories" + (f", each stopped after at most {cap} attempted steps"
                                                        if cap > 0 else ""))
    base = {"unit": UNIT, "trajectories": n, "workload": wl,
            "attempted_steps_per_trajectory": res["primal"][1] / n,
            "primal_persistent_ms_same_sample": res["primal"][0]}
    tan = dict(base, value=n / (res["tangent"][0] / 1e3), ms=res["tangent"][0], directions=4, ftle=True,
               attempted_steps_per_s=res["tangent"][1] / (res["tangent"][0] / 1e3),
               cost_vs_primal=res["tangent"][0] / res["primal"][0])
    adj = dict(base, value=n / (res["adjoint"][0] / 1e3), ms=res["adjoint"][0], objectives=4, seeds=4,
               attempted_steps_per_s=res["adjoint"][1] / (res["adjoint"][0] / 1e3),
               checkpoint_every=10000, cost_vs_primal=res["adjoint"][0] / res["primal"][0])
    return tan, adj


def secondary(args):
    """One timed launch of a secondary workload after W warm-up launches on its first 2048 trajectories;
    prints one JSON line (trajectories/s, device-timed, inputs resident)."""
    import torch
    from paper_2509_15117_gb300 import binding as Bd
    from paper_2509_15117_gb300 import schedule as Sch
    if args.workload == "energy-scan":
        energy_scan(args)
        return
    if args.workload == "thermal-sweep":
        thermal_sweep(args)
        return
    if args.workload == "lifetimes":
        lifetimes(args)
        return
    if args.workload == "diff":
        n = int(args.scale) if args.scale > 0 else 1 << 20
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
        tan, adj = diff_bench(n, flush, args.workload_cap)
        print(json.dumps({"metric": METRIC, "workload": "diff", "tangent": tan, "adjoint": adj,
                          "gpu_launches": 6, "dtype": "f64", "data": "synthetic"}), flush=True)
        return
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    if args.workload == "sampler":
        n = int(args.scale * (1 << 20)) if args.scale > 0 else 1 << 24
        print(json.dumps({"workload": "sampler", "ic_sampler": sampler_bench(n, flush), "dtype": "f64",
                          "data": "synthetic"}), flush=True)
        return
    extra = {}
    if args.workload == "thermal":
        n_per = int(args.scale * 1e7) if args.scale > 0 else 10_000_000
        systems, y0, phi0, sid = I.c3_workload(n_per)
        desc = (f"Yb+-Rb Monte Carlo bath, disk sampler b_max 2000 a0, T = 10 uK, 100 uK, 1 mK, {n_per} "
                f"trajectories each (seeds 3001-3003), random rf phase, ion at 10 uK with micromotion")
    elif args.workload == "mixed-graph":
        scale = args.scale if args.scale > 0 else 1.0
        systems, y0, phi0, sid = I.c4_workload(scale=scale)
        desc = (f"250 cells D_e x q x a x species, 4096..262144 trajectories per cell x {scale}, head-on at "
                f"1.5 uK, random rf phase; launch + per-cell statistics replayed as one CUDA graph")
    else:
        sysd, y0, phi0, seeds = I.c5_ftle_grid(int(args.scale) if args.scale > 0 else 2048)
        systems, sid = [sysd], np.zeros(len(phi0), dtype=np.int32)
        desc = (f"tangent kernel (1 direction + FTLE) on the {int(round(len(phi0) ** 0.5))}^2 cell-centred "
                f"octant grid, Yb+-Rb head-on 1.5 uK, rf phase 0")
    descs = [s_.as_dict() for s_ in systems]
    n = len(phi0)
    with Bd.System(descs) as S:
        y, p, d = Bd.to_device_soa(y0, phi0, sid)
        out = Bd.alloc_obs(n)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if args.workload == "ftle":
            dyd = torch.from_numpy(np.ascontiguousarray(np.transpose(seeds, (1, 2, 0)))).cuda()
            tan = Bd.alloc_tangent(n, 1)
            for _ in range(args.warmup):
                m = min(n, 2048)
                Bd.ia_launch_tangent(S.handle, y[:, :m].contiguous(), p[:m].contiguous(), None,
                                     Bd.alloc_obs(m), dyd[:, :, :m].contiguous(), np.zeros((1, 3)), Bd.alloc_tangent(m, 1))
            torch.cuda.synchronize()
            flush.zero_()
            e0.record(stream)
            Bd.ia_launch_tangent(S.handle, y, p, None, out, dyd, np.zeros((1, 3)), tan)
            e1.record(stream)
            launches = 1
        else:
            # queue order: slow and heavy systems first (the velocity tolerance is 1e-10 x the speed scale)
            speeds = [s_.atol_vel / 1e-10 for s_ in systems]
            order = torch.from_numpy(Sch.order_by_cost(sid, Sch.system_cost(systems, speeds))).cuda()
            for _ in range(args.warmup):
                m = min(n, 2048)
                Bd.ia_launch(S.handle, y[:, :m].contiguous(), p[:m].contiguous(), d[:m].contiguous(), Bd.alloc_obs(m))
            torch.cuda.synchronize()
            if args.workload == "mixed-graph":
                st = Bd.alloc_stats(len(descs))
                gstream = torch.cuda.Stream()
                with torch.cuda.stream(gstream):
                    G = Bd.Graph(S.handle, y, p, d, out, gstream, order=order, cell_id=d, n_cells=len(descs), stats=st)
                gstream.synchronize()
                flush.zero_()
                torch.cuda.synchronize()
                e0.record(gstream)
                G.launch(gstream)
                e1.record(gstream)
                gstream.synchronize()
                stats = Bd.stats_to_numpy(st)
                extra["cells"] = len(descs)
                extra["p_complex_range"] = [float((stats["n_complex"] / np.maximum(stats["n"], 1)).min()),
                                            float((stats["n_complex"] / np.maximum(stats["n"], 1)).max())]
                G.close()
                launches = 4  # persistent kernel, clean-up kernel, two statistics passes
            else:
                flush.zero_()
                e0.record(stream)
                Bd.ia_launch(S.handle, y, p, d, out, order=order)
                e1.record(stream)
                launches = 2
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        att = int((out["n_steps"].to(torch.int64) + out["n_rej"].to(torch.int64)).sum().item())
        mx = int((out["n_steps"] + out["n_rej"]).max().item())
    print(json.dumps({"metric": METRIC, "workload": args.workload, "value": n / (ms / 1e3), "unit": UNIT,
                      "ms": ms, "trajectories": n, "rhs_evals_per_s": (6 * att + n) / (ms / 1e3),
                      "attempted_steps_per_trajectory": att / n, "max_attempted_steps": mx,
                      "gpu_launches": launches, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": desc, "rtol": 1e-10}, **extra}), flush=True)


def hbm_peak_gbs():
    """Measured copy bandwidth of this GPU type (generated file), else the earlier measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


IC_BYTES = 13 * 8  # y0 (12 doubles) and phi0 written per trajectory


def sampler_bench(n: int, flush, seed: int = 7):
    """ia_sample_ics for each kind on n trajectories (a warm-up launch, then one launch timed with CUDA
    events after an L2 flush), against the pinned host-to-device copy of the same bytes."""
    import torch
    from paper_2509_15117_gb300 import binding as Bd
    stream = torch.cuda.current_stream()
    d = I.make_system("Rb").as_dict()
    kinds = {"head_on": (Bd.IA_SAMPLE_HEAD_ON, dict(E=I.kelvin(1.5e-6))),
             "sphere": (Bd.IA_SAMPLE_SPHERE, dict(kT=I.kelvin(1e-4), kT_ion=I.kelvin(1e-5))),
             "disk": (Bd.IA_SAMPLE_DISK, dict(kT=I.kelvin(1e-3), kT_ion=I.kelvin(1e-5), b_max=2000.0,
                                              micromotion=True))}
    y = torch.empty((12, n), dtype=torch.float64, device="cuda")
    ph = torch.empty((n,), dtype=torch.float64, device="cuda")
    peak, src = hbm_peak_gbs()
    res = {}
    for name, (kind, kw) in kinds.items():
        smp = Bd.make_sampler(kind, d, seed, **kw)
        Bd.ia_sample_ics(smp, 0, y, ph)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        flush.zero_()
        e0.record(stream)
        Bd.ia_sample_ics(smp, 0, y, ph)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        gbs = n * IC_BYTES / (ms / 1e3) / 1e9
        res[name] = {"ms": ms, "value": n / (ms / 1e3), "unit": "initial conditions/s", "write_GBps": gbs,
                     "write_frac_of_hbm": gbs / peak}
    host = torch.empty((13, n), dtype=torch.float64).pin_memory()
    dev = torch.empty((13, n), dtype=torch.float64, device="cuda")
    dev.copy_(host, non_blocking=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    dev.copy_(host, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    h2d_ms = e0.elapsed_time(e1)
    del y, ph, host, dev
    return {"trajectories": n, "bytes_per_trajectory": IC_BYTES, "kinds": res,
            "h2d_copy_same_bytes_ms": h2d_ms, "hbm_peak_GBps": peak, "hbm_peak_source": src,
            "generator": "Philox4x64-10, 4 blocks per thermal trajectory (1 for head-on), Box-Muller"}


def energy_scan(args):
    """Fig. 4 workload: device-drawn head-on initial conditions with a random rf phase for every
    (species, energy) cell, one persistent launch over all cells, per-cell statistics; then the
    threshold fit of P_complex(E) per species against W0^3D. Timed on the device from the first
    sampler launch to the end of the statistics."""
    import torch
    from paper_2509_15117_gb300 import binding as Bd
    from paper_2509_15117_gb300 import schedule as Sch
    from paper_2509_15117_gb300 import statistics as St
    scale = args.scale if args.scale > 0 else 0.1
    n_per = max(1, int(round(scale * 10_000)))
    systems, energies, names = I.energy_scan_systems()
    descs = [s_.as_dict() for s_ in systems]
    n_cells = len(descs)
    n = n_per * n_cells
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    y = torch.empty((12, n), dtype=torch.float64, device="cuda")
    ph = torch.empty((n,), dtype=torch.float64, device="cuda")
    sid = torch.arange(n_cells, dtype=torch.int32, device="cuda").repeat_interleave(n_per)
    speeds = [s_.atol_vel / 1e-10 for s_ in systems]
    order = torch.from_numpy(Sch.order_by_cost(sid.cpu().numpy(), Sch.system_cost(systems, speeds))).cuda()
    samplers = [Bd.make_sampler(Bd.IA_SAMPLE_HEAD_ON, descs[c], 4004, E=float(energies[c])) for c in range(n_cells)]
    with Bd.System(descs) as S:
        out = Bd.alloc_obs(n)
        st = Bd.alloc_stats(n_cells)
        Bd.ia_reserve(S.handle, n, kernel=Bd.IA_KERNEL_PERSISTENT)
        Bd.ia_reserve_stats(S.handle, n, n_cells)
        for _ in range(args.warmup):  # one cell's first 256 trajectories, highest energy of the first species
            c = n_cells // len(I.C2_SPECIES) - 1
            Bd.ia_sample_ics(samplers[c], c * n_per, y[:, :256], ph[:256])
            Bd.ia_launch(S.handle, y[:, :256], ph[:256], torch.full((256,), c, dtype=torch.int32, device="cuda"),
                         Bd.alloc_obs(256))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        for c in range(n_cells):
            a = c * n_per
            Bd.ia_sample_ics(samplers[c], a, y[:, a:a + n_per], ph[a:a + n_per])
        Bd.ia_launch(S.handle, y, ph, sid, out, order=order)
        Bd.ia_reduce_stats(S.handle, out, n, sid, n_cells, st)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        waits = Bd.ia_launch_phases(S.handle)[2]
        stats = Bd.stats_to_numpy(st)
        att = int((out["n_steps"].to(torch.int64) + out["n_rej"].to(torch.int64)).sum().item())
        mx = int((out["n_steps"] + out["n_rej"]).max().item())
        # complexes that outlive one secular period of the ion (2 pi / omega, omega = q_x Omega / 2^(3/2)):
        # a second pericentre within it is the trap swinging the ion back onto the receding atom
        tau = (out["t_last_bounce"] - out["t_first_bounce"]).cpu().numpy()
        nbh = out["n_bounce"].cpu().numpy()
    t_sec = 2.0 * math.pi / (abs(systems[0].q[0]) * systems[0].Omega / (2.0 * math.sqrt(2.0)))
    long_lived = ((nbh >= 2) & (tau >= t_sec)).reshape(n_cells, n_per).sum(axis=1)
    per_species = {}
    uK = 1e6 / I.K_TO_HARTREE
    for sp in dict.fromkeys(names):
        cells = [c for c in range(n_cells) if names[c] == sp]
        E = energies[cells]
        k = stats["n_complex"][cells]
        m = stats["n"][cells]
        fit = St.fit_threshold(E, k, m)
        d0 = systems[cells[0]]
        w0 = St.w0_3d(d0.m_atom, d0.m_ion, d0.Omega, d0.a[0], d0.q[0], 0.5 * d0.alpha)
        kl = long_lived[cells]
        fit_l = St.fit_threshold(E, kl, m)
        per_species[sp] = {"E_threshold_uK": fit["E_th"] * uK, "E_end_uK": fit["E_end"] * uK, "W0_3D_uK": w0 * uK,
                           "threshold_over_W0": fit["E_th"] / w0, "end_over_W0": fit["E_end"] / w0,
                           "P0": fit["P0"], "P_inf": fit["P_inf"], "width_ln_E": fit["width_ln"],
                           "chi2_per_dof": fit["chi2"] / max(fit["dof"], 1),
                           "P_complex_lowest_E": float(k[0] / m[0]), "P_complex_highest_E": float(k[-1] / m[-1]),
                           "beyond_one_secular_period": {
                               "E_threshold_uK": fit_l["E_th"] * uK, "E_end_uK": fit_l["E_end"] * uK,
                               "end_over_W0": fit_l["E_end"] / w0, "P0": fit_l["P0"], "P_inf": fit_l["P_inf"],
                               "chi2_per_dof": fit_l["chi2"] / max(fit_l["dof"], 1),
                               "P_lowest_E": float(kl[0] / m[0]), "P_highest_E": float(kl[-1] / m[-1])}}
    desc = (f"collision-energy scan: Yb+ head-on with {', '.join(dict.fromkeys(names))}, "
            f"{n_cells // len(per_species)} energies 30 nK..1 mK, {n_per} trajectories per energy, r0 = 20,000 a0, "
            f"D_e = 1 K, q = 0.1, t_max = 3 ms, random rf phase; initial conditions drawn on the device")
    print(json.dumps({"metric": METRIC, "workload": "energy-scan", "value": n / (ms / 1e3), "unit": UNIT, "ms": ms,
                      "trajectories": n, "attempted_steps_per_trajectory": att / n, "max_attempted_steps": mx,
                      "wait_errors": waits, "gpu_launches": n_cells + 4, "dtype": "f64", "data": "synthetic",
                      "secular_period_us": t_sec * I.AU_TIME_S * 1e6,
                      "config": {"workload": desc, "rtol": 1e-10}, "per_species": per_species}), flush=True)


def thermal_sweep(args):
    """Fig. 3 workload: the paper's thermal runs (atom uniform on the r0 sphere, Gaussian velocity flipped
    inward, ion Gaussian at 10 uK, random rf phase) drawn on the device for every (species, T, D_e)
    cell, one persistent launch over all cells, per-cell statistics; then the complex probability per
    cell with its 3-sigma Wilson interval and the trends the text states (fewer complexes when hotter,
    more when heavier, no change between D_e = 1 K and 100 K). The paper runs 10^7 per cell; --scale
    is that fraction (default 1e-3)."""
    import torch
    from paper_2509_15117_gb300 import binding as Bd
    from paper_2509_15117_gb300 import schedule as Sch
    from paper_2509_15117_gb300 import statistics as St
    scale = args.scale if args.scale > 0 else 1e-3
    n_per = max(1, int(round(scale * 1e7)))
    systems, cells = I.thermal_sweep_systems()
    descs = [s_.as_dict() for s_ in systems]
    n_cells = len(descs)
    n = n_per * n_cells
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    y = torch.empty((12, n), dtype=torch.float64, device="cuda")
    ph = torch.empty((n,), dtype=torch.float64, device="cuda")
    sid = torch.arange(n_cells, dtype=torch.int32, device="cuda").repeat_interleave(n_per)
    speeds = [s_.atol_vel / 1e-10 for s_ in systems]
    order = torch.from_numpy(Sch.order_by_cost(sid.cpu().numpy(), Sch.system_cost(systems, speeds))).cuda()
    samplers = [Bd.make_sampler(Bd.IA_SAMPLE_SPHERE, descs[c], 3100, kT=I.kelvin(cells[c][1]),
                                kT_ion=I.kelvin(10e-6)) for c in range(n_cells)]
    with Bd.System(descs) as S:
        out = Bd.alloc_obs(n)
        st = Bd.alloc_stats(n_cells)
        Bd.ia_reserve(S.handle, n, kernel=Bd.IA_KERNEL_PERSISTENT)
        Bd.ia_reserve_stats(S.handle, n, n_cells)
        hot = max(range(n_cells), key=lambda c: cells[c][1])  # warm-up on a 1 mK cell: short trajectories
        for _ in range(args.warmup):
            m = min(256, n_per)
            Bd.ia_sample_ics(samplers[hot], hot * n_per, y[:, :m], ph[:m])
            Bd.ia_launch(S.handle, y[:, :m], ph[:m], torch.full((m,), hot, dtype=torch.int32, device="cuda"),
                         Bd.alloc_obs(m))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        for c in range(n_cells):
            a = c * n_per
            Bd.ia_sample_ics(samplers[c], a, y[:, a:a + n_per], ph[a:a + n_per])
        Bd.ia_launch(S.handle, y, ph, sid, out, order=order)
        Bd.ia_reduce_stats(S.handle, out, n, sid, n_cells, st)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        waits = Bd.ia_launch_phases(S.handle)[2]
        stats = Bd.stats_to_numpy(st)
        att = int((out["n_steps"].to(torch.int64) + out["n_rej"].to(torch.int64)).sum().item())
        mx = int((out["n_steps"] + out["n_rej"]).max().item())
    table = {}
    for c, (sp, T, De) in enumerate(cells):
        sm = St.summarize(stats[c])
        table[f"{sp} T={T * 1e6:g}uK De={De:g}K"] = {
            "P_complex": sm["P_complex"], "P_complex_3sigma": list(sm["P_complex_3sigma"]),
            "mean_dE_ion_uK": sm["mean_dE_ion"] / I.K_TO_HARTREE * 1e6}
    P = {cells[c]: St.summarize(stats[c])["P_complex"] for c in range(n_cells)}
    lo_hi = {cells[c]: St.summarize(stats[c])["P_complex_3sigma"] for c in range(n_cells)}
    sp_list = list(dict.fromkeys(cl[0] for cl in cells))
    temps = sorted(set(cl[1] for cl in cells))
    depths = sorted(set(cl[2] for cl in cells))
    trends = {
        "falls_with_T": all(P[(sp, temps[i], De)] >= P[(sp, temps[i + 1], De)]
                            for sp in sp_list for De in depths for i in range(len(temps) - 1)),
        "rises_with_mass": all(P[(sp_list[i], T, De)] <= P[(sp_list[i + 1], T, De)]
                               for T in temps for De in depths for i in range(len(sp_list) - 1)),
        "De_1K_vs_100K_overlap_3sigma": all(
            lo_hi[(sp, T, depths[0])][0] <= lo_hi[(sp, T, depths[1])][1] and
            lo_hi[(sp, T, depths[1])][0] <= lo_hi[(sp, T, depths[0])][1] for sp in sp_list for T in temps),
    }
    desc = (f"thermal runs (Fig. 3): Yb+ with {', '.join(sp_list)} x T = {', '.join(f'{t * 1e6:g} uK' for t in temps)} "
            f"x D_e = {', '.join(f'{d:g} K' for d in depths)}, {n_per} trajectories per cell; atom uniform on the "
            f"5000 a0 sphere, Gaussian velocity flipped inward, ion Gaussian at 10 uK, random rf phase; "
            f"drawn on the device (sphere sampler, seed 3100)")
    print(json.dumps({"metric": METRIC, "workload": "thermal-sweep", "value": n / (ms / 1e3), "unit": UNIT,
                      "ms": ms, "trajectories": n, "attempted_steps_per_trajectory": att / n,
                      "max_attempted_steps": mx, "wait_errors": waits, "gpu_launches": n_cells + 4,
                      "dtype": "f64", "data": "synthetic", "config": {"workload": desc, "rtol": 1e-10},
                      "trends": trends, "cells": table}), flush=True)


def lifetimes(args):
    """Fig. 2 workload: head-on collisions of each species with Yb+ at E = 1.5 uK, D_e = 1 K, r0 = 5000 a0,
    rf phase 0, (theta, phi) uniform on the octant and drawn on the device; one persistent launch over
    all species, per-species statistics; then the survival of complex lifetimes (t_last_bounce -
    t_first_bounce) and the maximum-likelihood fit of its tail beyond 20 us. A complex still alive at
    t_max is censored at its observed lifetime. --scale sets the trajectories per species in units of
    10^5 (default 0.2)."""
    import torch
    from paper_2509_15117_gb300 import binding as Bd
    from paper_2509_15117_gb300 import schedule as Sch
    from paper_2509_15117_gb300 import statistics as St
    scale = args.scale if args.scale > 0 else 0.2
    n_per = max(1, int(round(scale * 1e5)))
    E_K = 1.5e-6
    species = I.C2_SPECIES
    systems = [I.make_system(sp, De_K=1.0, q=0.1, a=0.0, r0=5000.0, t_max_s=1e-3, E_K=E_K) for sp in species]
    descs = [s_.as_dict() for s_ in systems]
    n_cells = len(descs)
    n = n_per * n_cells
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    y = torch.empty((12, n), dtype=torch.float64, device="cuda")
    ph = torch.empty((n,), dtype=torch.float64, device="cuda")
    sid = torch.arange(n_cells, dtype=torch.int32, device="cuda").repeat_interleave(n_per)
    speeds = [s_.atol_vel / 1e-10 for s_ in systems]
    order = torch.from_numpy(Sch.order_by_cost(sid.cpu().numpy(), Sch.system_cost(systems, speeds))).cuda()
    samplers = [Bd.make_sampler(Bd.IA_SAMPLE_HEAD_ON, descs[c], 2002, E=I.kelvin(E_K), random_phase=False,
                                phase=0.0) for c in range(n_cells)]
    with Bd.System(descs) as S:
        out = Bd.alloc_obs(n)
        st = Bd.alloc_stats(n_cells)
        Bd.ia_reserve(S.handle, n, kernel=Bd.IA_KERNEL_PERSISTENT)
        Bd.ia_reserve_stats(S.handle, n, n_cells)
        for _ in range(args.warmup):  # 256 Li trajectories
            Bd.ia_sample_ics(samplers[0], 0, y[:, :256], ph[:256])
            Bd.ia_launch(S.handle, y[:, :256], ph[:256], sid[:256].contiguous(), Bd.alloc_obs(256))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        for c in range(n_cells):
            a = c * n_per
            Bd.ia_sample_ics(samplers[c], a, y[:, a:a + n_per], ph[a:a + n_per])
        Bd.ia_launch(S.handle, y, ph, sid, out, order=order)
        Bd.ia_reduce_stats(S.handle, out, n, sid, n_cells, st)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        waits = Bd.ia_launch_phases(S.handle)[2]
        stats = Bd.stats_to_numpy(st)
        g = Bd.to_numpy(out)
    us = I.AU_TIME_S * 1e6
    t_min_us = 20.0
    k_min = int(math.floor(2.0 * (math.log2(t_min_us / us) - 20.0)))  # first lifetime bin at or after 20 us
    per_species = {}
    for c, sp in enumerate(species):
        sl = slice(c * n_per, (c + 1) * n_per)
        cx = g["n_bounce"][sl] >= 2
        tau = (g["t_last_bounce"][sl] - g["t_first_bounce"][sl])[cx] * us
        cens = ((g["status"][sl] & Bd.ST_TMAX) != 0)[cx]
        fit = St.lifetime_tail_fit(tau, t_min_us, censored=cens)
        binned = St.lifetime_tail_fit_binned(stats["lifetime_hist"][c], k_min + 1)
        alive = {f"{t:g}us": float((tau >= t).mean()) if tau.size else 0.0 for t in (1, 20, 100, 300, 600)}
        per_species[sp] = {"complexes": int(cx.sum()), "P_complex": float(cx.mean()), "alive_after": alive,
                           "beyond_20us": fit["n"], "censored_at_t_max": int(cens.sum()),
                           "gamma": fit["gamma"], "gamma_se": fit["gamma_se"],
                           "loglik_power_minus_exp": fit["loglik_power"] - fit["loglik_exp"],
                           "gamma_from_bins": binned["gamma"], "gamma_from_bins_se": binned["gamma_se"]}
    desc = (f"complex lifetimes (Fig. 2): Yb+ head-on with {', '.join(species)} at E = 1.5 uK, D_e = 1 K, "
            f"r0 = 5000 a0, q = 0.1, rf phase 0, t_max = 1 ms, {n_per} trajectories per species with (theta, phi) "
            f"uniform on the octant drawn on the device (seed 2002)")
    att = int((g["n_steps"].astype(np.int64) + g["n_rej"]).sum())
    print(json.dumps({"metric": METRIC, "workload": "lifetimes", "value": n / (ms / 1e3), "unit": UNIT, "ms": ms,
                      "trajectories": n, "attempted_steps_per_trajectory": att / n,
                      "max_attempted_steps": int((g["n_steps"].astype(np.int64) + g["n_rej"]).max()),
                      "wait_errors": waits, "gpu_launches": n_cells + 4, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": desc, "rtol": 1e-10, "tail_fit_from_us": t_min_us},
                      "per_species": per_species}), flush=True)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def step_offset(step: int, stride: int, rank: int = 0, world: int = 1) -> int:
    """Grid offset of a (step, rank) pair: consecutive pairs take consecutive offsets, so ranks of one
    step integrate disjoint sub-grids whenever stride >= world (with stride 1 every rank integrates
    the whole sweep: replicas)."""
    return (step * world + rank) % stride


def batch(step: int, stride: int, rank: int = 0, world: int = 1):
    """Batch of a step (see step_offset)."""
    off = step_offset(step, stride, rank, world)
    systems, y0, phi0, sid = I.c2_workload(n_grid=GRID, stride=stride, offset=off)
    return systems, y0, phi0, sid


def reduce_over_ranks(dist, device, maxima, sums):
    """Whole-job figures of a multi-rank run: the maximum over ranks of each entry of `maxima` (step
    times) and the sum of each entry of `sums` (trajectories, RHS evaluations, attempts)."""
    import torch
    t = torch.tensor(maxima, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor(sums, dtype=torch.float64, device=device)
    dist.all_reduce(c)
    return [float(x) for x in t.tolist()], [float(x) for x in c.tolist()]


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, max clock, throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def _oracle_sample(seconds: float, steps: int = 1, warmup: int = 0):
    """The oracle, as it stands, on all host cores, over bounded samples of the same workload:
    trajectories drawn uniformly at random (seed 12345) from the step-0 batch at grid stride 4, in
    chunks, until each of `steps` timed steps has used about seconds/steps of wall time; `warmup`
    small untimed chunks first."""
    from oracle import oracle as O
    systems, y0, phi0, sid = batch(0, 4)
    descs = [s.as_dict() for s in systems]
    n_all = len(y0)
    cores = O.max_threads()
    order = np.random.default_rng(12345).permutation(n_all)
    pos = 0
    for _ in range(warmup):
        idx = np.sort(order[pos:pos + 2 * cores])
        pos += len(idx)
        O.run_batch(descs, y0[idx], phi0[idx], sid[idx], nthreads=cores)
    per_step = seconds / max(steps, 1)
    done = attempts = 0
    step_s = []
    for _ in range(steps):
        t_step = 0.0
        chunk = max(cores * 4, 64)
        while t_step < per_step and pos < n_all:
            idx = np.sort(order[pos:pos + chunk])
            pos += len(idx)
            t0 = time.perf_counter()
            r = O.run_batch(descs, y0[idx], phi0[idx], sid[idx], nthreads=cores)
            t_step += time.perf_counter() - t0
            attempts += int(np.sum(r["n_steps"] + r["n_rej"]))
            done += len(idx)
            chunk = min(chunk * 2, 4096)
        step_s.append(t_step)
    t_used = float(sum(step_s))
    return {"value": done / t_used, "unit": UNIT, "cores": cores, "kind": "oracle",
            "rhs_evals_per_s": (6 * attempts + done) / t_used, "ms_per_step": 1e3 * t_used / max(steps, 1),
            "sample": f"{done} trajectories drawn uniformly at random (seed 12345) from the step-0 batch "
                      f"(species x energy sweep, grid stride 4), {t_used:.1f} s on {cores} threads"}


def cpu_baseline(seconds: float, single_seconds: float = 3.0):
    """The oracle on all host cores, plus a single-thread figure on the next trajectories of the same
    random order (about single_seconds of one core)."""
    from oracle import oracle as O
    cb = _oracle_sample(seconds)
    if single_seconds > 0:
        systems, y0, phi0, sid = batch(0, 4)
        descs = [s.as_dict() for s in systems]
        order = np.random.default_rng(12345).permutation(len(y0))[::-1]  # not the multi-thread sample
        done, t_used, pos = 0, 0.0, 0
        while t_used < single_seconds and pos < len(order):
            idx = np.sort(order[pos:pos + 8])
            pos += len(idx)
            t0 = time.perf_counter()
            O.run_batch(descs, y0[idx], phi0[idx], sid[idx], nthreads=1)
            t_used += time.perf_counter() - t0
            done += len(idx)
        cb["single_thread"] = {"value": done / t_used, "unit": UNIT, "trajectories": done, "seconds": t_used}
    return cb


def run_reference(args, rank, world):
    """The reference arm: the oracle timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    cb = _oracle_sample(max(args.cpu_seconds, 5.0), steps=args.steps, warmup=args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": cb["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "Yb+ head-on species x energy sweep (5 species x 8 energies, 1024^2 "
                               "octant grid, D_e = 1 K, q = 0.1, t_max = 1 ms), bounded sample",
                   "rtol": 1e-10},
        "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
        "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "rhs_evals_per_s": cb["rhs_evals_per_s"],
    }
    print(json.dumps(line), flush=True)


def sweep_in_queue_order(stride: int, offset: int, rule: str = "cost"):
    """The species x energy sweep (every stride-th grid point from offset) laid out in queue order
    (systems by expected cost, costliest first; see schedule.py), so that each part of the queue is a
    contiguous range of the arrays. Returns the systems, the pinned host arrays (SoA state (12, n),
    phases, system ids) and the permutation from queue position to grid order."""
    import torch
    from paper_2509_15117_gb300 import schedule as Sch
    systems, y0, phi0, sid = I.c2_workload(n_grid=GRID, stride=stride, offset=offset)
    if rule == "threshold":
        from paper_2509_15117_gb300 import statistics as St
        w0 = [St.w0_3d(s.m_atom, s.m_ion, s.Omega, s.a[0], s.q[0], 0.5 * s.alpha) for s in systems]
        energies = [I.kelvin(E) for (sp, E, s) in I.c2_systems()]
        cost = Sch.system_cost_threshold(energies, w0)
    else:
        speeds = [I.speed_for_energy(I.kelvin(E), s.m_atom) for (sp, E, s) in I.c2_systems()]
        cost = Sch.system_cost(systems, speeds)
    order = Sch.order_by_cost(sid, cost)
    n = len(phi0)
    hy = torch.empty((12, n), dtype=torch.float64).pin_memory()
    hyn = hy.numpy()
    for c in range(12):
        np.take(y0[:, c], order, out=hyn[c])
    del y0
    hp = torch.from_numpy(phi0[order]).pin_memory()
    hs = torch.from_numpy(sid[order]).pin_memory()
    return systems, hy, hp, hs, order


def part_bounds(n: int, parts: int, last_frac: float = 0.0) -> np.ndarray:
    """Queue positions where each of `parts` parts of an n-trajectory batch starts (and n): equal parts,
    or, with last_frac > 0, the last part holding that fraction of the queue (its cheapest trajectories:
    bulk work that overlaps the tail's last complexes instead of leaving the GPU waiting for them) and
    the others equal."""
    if parts < 2 or last_frac <= 0.0:
        return np.linspace(0, n, parts + 1).round().astype(np.int64)
    head = int(round(n * (1.0 - last_frac)))
    return np.concatenate([np.linspace(0, head, parts).round(), [n]]).astype(np.int64)


def lane_options(args, handle, y, p, d, n_sample: int, attempt_cap: int):
    """Launch options of the queue: the autotuner's pick of block, register variant and refill on a
    random sample of the batch (unless --no-autotune or an explicit --block); the reserved tail SMs
    (a reserved SM keeps up to 4 tail warps, one per sub-partition) sized so that the tail has 128
    warps whatever the block size."""
    import torch
    from paper_2509_15117_gb300 import binding as Bd
    kw = {"block": args.block, "refill": args.refill, "blocks_per_sm": args.blocks_per_sm,
          "regs_variant": args.regs_variant, "slice_budget": args.slice_budget, "tail_group": args.tail_group,
          "tail_blocks_per_sm": args.tail_blocks_per_sm, "tail_sms": args.tail_sms, "tail_warps": args.tail_warps}
    tune = None
    if not args.no_autotune and args.block == 0:
        n = int(p.shape[0])
        idx = torch.from_numpy(np.sort(np.random.default_rng(99).choice(n, min(n_sample, n), replace=False))).cuda()
        t0 = time.perf_counter()
        pick, ms = Bd.ia_autotune(handle, y[:, idx].contiguous(), p[idx].contiguous(), d[idx].contiguous(),
                                  attempt_cap=attempt_cap)
        tune = {"pick": pick, "best_ms": ms, "seconds": time.perf_counter() - t0,
                "sample": f"{int(idx.numel())} trajectories drawn at random (seed 99) from the batch, every "
                          f"one stopped after {attempt_cap} attempted steps (lane phase only); 9 candidates "
                          f"(block 64/128/256, register cap 1 or 3 blocks/SM, refill 1/4/16), each timed twice"}
        kw.update(pick)
    block = kw["block"] or 128
    if args.tail_sms == 0:
        kw["tail_sms"] = 128 // min(kw["tail_warps"] or 4, block // 32)
    return kw, tune


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.profile_case:
        profile_case(args.profile_grid)
        return
    if args.workload != "sweep" and args.impl == "ours":
        secondary(args)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    from paper_2509_15117_gb300 import binding as Bd

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    K = args.steps
    # The batch: the whole sweep (or with --stride S every S-th grid point, a different offset per rank)
    # in queue order, pinned on the host; the device holds the whole batch, and the K timed steps are
    # the K parts of one queue over it, so together they integrate every trajectory once.
    systems, hy, hp, hs, order = sweep_in_queue_order(args.stride, step_offset(0, args.stride, rank, world),
                                                      args.order)
    n = int(hp.shape[0])
    descs = [s.as_dict() for s in systems]
    sysh = Bd.System(descs)
    dy = torch.empty_like(hy, device="cuda")
    dp_ = torch.empty_like(hp, device="cuda")
    ds = torch.empty_like(hs, device="cuda")
    out = Bd.alloc_obs(n)
    hout = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in out.items()}
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB > L2

    # lane-phase options from the autotuner (inputs copied once for it, overwritten by the timed steps)
    dy.copy_(hy)
    dp_.copy_(hp)
    ds.copy_(hs)
    kw, tune = lane_options(args, sysh.handle, dy, dp_, ds, 65536, 8192)

    # warm-up: W parts of a queue over the short trajectories of the workload (the 1 mK systems of
    # every 4th grid point), the same kernel and part logic as the timed steps
    e_last = len(I.C2_ENERGIES_K) - 1
    sw, wy, wp, ws, _ = sweep_in_queue_order(4, 0)
    keep = torch.from_numpy(np.nonzero(ws.numpy() % len(I.C2_ENERGIES_K) == e_last)[0])
    wy, wp, ws = wy[:, keep].cuda(), wp[keep].cuda(), ws[keep].cuda()
    nw = int(wp.shape[0])
    wout = Bd.alloc_obs(nw)
    with Bd.Queue(sysh.handle, nw, **kw) as QW:
        wb = part_bounds(nw, max(args.warmup, 1))
        for k in range(max(args.warmup, 1)):
            QW.launch(wy, wp, ws, wout, int(wb[k + 1] - wb[k]))
        torch.cuda.synchronize()
    del wy, wp, ws, wout

    peak_flops = Bd.ia_fp64_peak(4, 20000)

    Q = Bd.Queue(sysh.handle, n, **kw)
    bounds = part_bounds(n, K, args.last_part)
    fields = list(out.keys())
    # timed steps: host -> device copy of the part's inputs, L2 flush, the part's launch (device-timed
    # for `value`), device -> host copy of the part's observables (the last step copies every
    # observable, since trajectories carried between parts end in later parts); the whole is `e2e`
    clocks = ClockSampler(local)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    phases = []
    barrier()
    clocks.start()
    t0 = time.perf_counter()
    h2d = d2h = 0
    for k in range(K):
        a, b = int(bounds[k]), int(bounds[k + 1])
        ev[k][0].record(stream)
        for c in range(12):
            dy[c, a:b].copy_(hy[c, a:b], non_blocking=True)
        dp_[a:b].copy_(hp[a:b], non_blocking=True)
        ds[a:b].copy_(hs[a:b], non_blocking=True)
        h2d += (b - a) * (12 * 8 + 8 + 4)
        flush.zero_()
        ev[k][1].record(stream)
        Q.launch(dy, dp_, ds, out, b - a)
        ev[k][2].record(stream)
        lo, hi = (a, b) if k < K - 1 else (0, n)
        for f in fields:
            hout[f][lo:hi].copy_(out[f][lo:hi], non_blocking=True)
            d2h += (hi - lo) * out[f].element_size()
        ev[k][3].record(stream)
    barrier()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    lane_ms, dev_ms, wait_errors = Q.phases()  # the last part
    kern_ms = [e[1].elapsed_time(e[2]) for e in ev]
    step_ms = [e[0].elapsed_time(e[3]) for e in ev]
    total_ms = float(sum(kern_ms))
    g_steps = hout["n_steps"].numpy().astype(np.int64)
    g_rej = hout["n_rej"].numpy().astype(np.int64)
    per = g_steps + g_rej
    attempts = int(per.sum())
    status = hout["status"].numpy().view(np.uint32)
    status_counts = {nm: int(np.count_nonzero(status & b)) for nm, b in
                     (("tmax", Bd.ST_TMAX), ("max_steps", Bd.ST_MAX_STEPS), ("h_underflow", Bd.ST_H_UNDERFLOW),
                      ("nonfinite", Bd.ST_NONFINITE), ("bad_ic", Bd.ST_BAD_IC), ("exit_outside", Bd.ST_EXIT_OUTSIDE))}
    status_counts["complex"] = int(np.count_nonzero(status & Bd.ST_COMPLEX))
    max_attempts = int(per.max())
    budget_used = kw["slice_budget"] if kw["slice_budget"] > 0 else 131072
    long_counts = {f"over_{b}": int((per > b).sum()) for b in (budget_used, 262144, 1048576)}
    top = np.sort(per)[::-1]
    long_counts["top10_attempts"] = [int(v) for v in top[:10]]
    long_counts["attempts_beyond_budget"] = int(np.maximum(per - budget_used, 0).sum())
    # what other slice budgets would leave to the group-mode tail (attempts beyond each)
    long_counts["attempts_beyond"] = {str(b): int(np.maximum(per - b, 0).sum())
                                      for b in (1 << 16, 1 << 17, 1 << 18, 1 << 19, 1 << 20)}
    long_counts["longest_queue_position"] = int(np.argmax(per)) / n
    if args.dump_long and rank == 0:
        q = np.nonzero(per > (1 << 17))[0]
        sys_attempts = np.bincount(hs.numpy(), weights=per.astype(np.float64), minlength=len(systems))
        np.savez(args.dump_long, position=q, sys_id=hs.numpy()[q], attempts=per[q], bounds=bounds,
                 kernel_ms=np.asarray(kern_ms), n=n, sys_attempts=sys_attempts,
                 sys_count=np.bincount(hs.numpy(), minlength=len(systems)), lane_ms=lane_ms)
    rhs = 6 * attempts + n
    tmax_ms, emax_ms = total_ms, float(sum(step_ms))
    if dist is not None:
        (tmax_ms, emax_ms), (n_all, rhs_all, att_all) = reduce_over_ranks(
            dist, "cuda", [total_ms, emax_ms], [float(n), float(rhs), float(attempts)])
    else:
        n_all, rhs_all, att_all = float(n), float(rhs), float(attempts)
    value = n_all / (tmax_ms / 1e3)
    achieved = FLOPS_PER_ATTEMPT * attempts / (total_ms / 1e3)
    e2e = {"value": n_all / (emax_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d // K),
           "d2h_bytes_per_step": int(d2h // K), "ms_per_step": emax_ms / K,
           "path": "ia_queue_launch per step with the part's inputs copied from pinned host memory before it "
                   "and its observables copied back after it (the last step copies all n), inside the timed "
                   "region"}
    Q.close()
    del dy, dp_, ds

    # plain kernel against the persistent one on a subsample of the batch (every 256th trajectory in
    # queue order): the plain kernel's warps each wait for their longest lane
    plain = None
    if not args.no_plain:
        sub = np.arange(0, n, 256)
        ys = hy[:, torch.from_numpy(sub)].cuda()
        ps, ss = hp[torch.from_numpy(sub)].cuda(), hs[torch.from_numpy(sub)].cuda()
        m = len(sub)
        res = {}
        with Bd.System(descs) as SC:
            for name, kk in (("plain", {"kernel": Bd.IA_KERNEL_PLAIN}), ("persistent", dict(kw))):
                ob = Bd.alloc_obs(m)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                flush.zero_()
                e0.record(stream)
                Bd.ia_launch(SC.handle, ys, ps, ss, ob, **kk)
                e1.record(stream)
                torch.cuda.synchronize()
                res[name] = e0.elapsed_time(e1)
        plain = {"value": m / (res["plain"] / 1e3), "unit": UNIT, "trajectories": m, "ms": res["plain"],
                 "persistent_ms_same_batch": res["persistent"],
                 "persistent_speedup": res["plain"] / res["persistent"],
                 "batch": "every 256th trajectory of the batch in queue order, same inputs for both kernels (both "
                          "end with the latency of the sample's longest trajectory)"}

    diff = None
    if rank == 0 and args.diff_sample > 0:
        diff = diff_bench(args.diff_sample, flush, args.diff_cap)

    sampler = None
    if rank == 0 and args.sampler_sample > 0:
        sampler = sampler_bench(args.sampler_sample, flush)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(args.cpu_seconds)

    sysh.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": tmax_ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {
                "workload": "Yb+ head-on species x energy sweep: Li, Na, K, Rb, Cs x 8 energies 1 uK..1 mK, "
                            "D_e = 1 K, q = 0.1, a = 0, Omega = 2 pi 2 MHz, t_max = 1 ms, rtol 1e-10; "
                            + ("the whole 1024^2 octant grid" if args.stride == 1 else
                               f"1024^2 octant grid, every {args.stride}th point per direction")
                            + f" ({int(n_all / world)} trajectories), integrated once over the {K} steps: step k is "
                              f"part k of one work queue over the batch in queue order",
                "trajectories_per_step": int(n_all / K), "rtol": 1e-10, "kernel": "persistent (ia_queue)",
                "parts": ("equal" if args.last_part <= 0 else
                          f"the last holds {args.last_part:g} of the queue (its cheapest), the others equal"),
                "queue_order": "systems by sqrt(m_atom)/speed, descending",
                "l2": "256 MiB buffer written before each step (each part's inputs also exceed L2)",
                "launch_options": {k_: v for k_, v in kw.items() if v},
                "autotune": tune,
            },
            "rhs_evals_per_s": rhs_all / (tmax_ms / 1e3),
            "attempted_steps_per_trajectory": att_all / n_all,
            "max_attempted_steps": max_attempts,
            "status_counts": status_counts,
            "long_trajectories": long_counts,
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_flops / 1e12,
                         "unit": "TFLOP/s", "frac": achieved / peak_flops,
                         "traffic": DRAM_BYTES_PER_TRAJECTORY * n / K,
                         "traffic_note": "bytes per launch, ncu DRAM bytes of the 512x512 profile case scaled by "
                                         "trajectories (traffic grows with them: ICs in, observables out)",
                         "peak_source": "FP64 FMA microbenchmark (ia_fp64_peak) measured in this run",
                         "flops_per_attempted_step": FLOPS_PER_ATTEMPT},
            "plain": plain,
            "e2e": e2e,
            "gpu_launches": K + (1 if (kw["slice_budget"] or 0) >= 0 else 0),
            "step_kernel_ms": [round(x, 3) for x in kern_ms],
            "phases_last_step": {"lane_phase_ms": lane_ms, "kernel_ms": dev_ms, "wait_errors": wait_errors,
                                 "note": "device clock: until the last warp left the lane phase / until the "
                                         "last warp finished (the last part drains every carried trajectory)"},
            "clocks": clk,
            "wall_s": wall,
        }
        if diff is not None:
            line["tangent"], line["adjoint"] = diff
        if sampler is not None:
            line["ic_sampler"] = sampler
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
