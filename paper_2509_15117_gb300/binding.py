"""Thin Python binding of the C ABI in ``include/ionatom.h`` (argument marshalling only).

Every step of the trajectory computation runs in the CUDA library; this module only builds the C
structs, moves arrays to structure-of-arrays device tensors (PyTorch is used for device memory and
streams), and turns return codes into exceptions. There is no CPU fallback: if the compiled library
or a CUDA device is missing, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

IA_OK = 0
IA_KERNEL_PLAIN = 0
IA_KERNEL_PERSISTENT = 1

ST_EXIT = 0
ST_TMAX = 1 << 0
ST_MAX_STEPS = 1 << 1
ST_H_UNDERFLOW = 1 << 2
ST_NONFINITE = 1 << 3
ST_BAD_IC = 1 << 4
ST_EXIT_OUTSIDE = 1 << 5
ST_COMPLEX = 1 << 8

EXPORTED = ("ia_system_create", "ia_system_destroy", "ia_system_count", "ia_scratch_bytes", "ia_reserve",
            "ia_launch", "ia_launch_static", "ia_reduce_stats", "ia_reserve_stats", "ia_graph_create",
            "ia_graph_launch", "ia_graph_destroy", "ia_autotune", "ia_launch_phases", "ia_launch_tangent",
            "ia_adjoint_scratch_bytes", "ia_launch_adjoint", "ia_philox4x64", "ia_sample_ics", "ia_fp64_peak",
            "ia_rcp_check", "ia_error_string", "ia_version", "ia_queue_create", "ia_queue_launch",
            "ia_queue_reset", "ia_queue_state", "ia_queue_phases", "ia_queue_destroy", "ia_static_phases")

IA_SAMPLE_HEAD_ON = 0
IA_SAMPLE_SPHERE = 1
IA_SAMPLE_DISK = 2

STATS_BOUNCE_BINS = 32
STATS_LIFETIME_BINS = 64
STATS_EXIT_SLOT = 6
STATS_DTYPE = np.dtype([
    ("n", "<i8"), ("n_complex", "<i8"), ("attempts", "<i8"), ("n_status", "<i8", (8,)),
    ("bounce_hist", "<i8", (STATS_BOUNCE_BINS,)), ("lifetime_hist", "<i8", (STATS_LIFETIME_BINS,)),
    ("sum_dE", "<f8"), ("sum_dE2", "<f8"),
])

IA_STATIC_SCRATCH_BYTES = 4 << 20
IA_STATIC_MAX_RECORDS = 16128  # suspend records that fit beside the counters and ready flags


class IaError(RuntimeError):
    pass


class IaArgumentError(IaError, ValueError):
    """A tensor handed to the binding lacks the dtype, shape, layout or device the C ABI expects. The
    C side receives bare pointers and sizes, so these are checked here before any pointer crosses."""


def _on_device(t) -> bool:
    return bool(t.is_cuda)


def _tensor(t, name: str, dtype, shape, contiguous: bool = True):
    """Check one tensor: dtype, rank, sizes (None = any), a dense layout (or, with contiguous=False, a
    structure-of-arrays layout: unit stride along the last axis, rows at least a row's length apart),
    and last the device."""
    import torch
    if t is None:
        raise IaArgumentError(f"{name}: missing")
    if not isinstance(t, torch.Tensor):
        raise IaArgumentError(f"{name}: expected a torch tensor, got {type(t).__name__}")
    if t.dtype != dtype:
        raise IaArgumentError(f"{name}: dtype {t.dtype}, expected {dtype}")
    if t.dim() != len(shape) or any(w is not None and t.shape[a] != w for a, w in enumerate(shape)):
        raise IaArgumentError(f"{name}: shape {tuple(t.shape)}, expected {tuple(shape)}")
    if t.numel() > 0:
        if contiguous and not t.is_contiguous():
            raise IaArgumentError(f"{name}: must be contiguous")
        if not contiguous and (t.stride(-1) != 1 and t.shape[-1] > 1
                               or any(t.stride(a) < t.shape[-1] for a in range(t.dim() - 1))):
            raise IaArgumentError(f"{name}: rows must have unit stride and not overlap, strides {t.stride()}")
    if not _on_device(t):
        raise IaArgumentError(f"{name}: must be on a CUDA device")
    return t


def _ic_tensors(y0_soa, phi0, sys_id, order) -> int:
    import torch
    _tensor(phi0, "phi0", torch.float64, (None,))
    n = int(phi0.shape[0])
    _tensor(y0_soa, "y0_soa", torch.float64, (12, n), contiguous=False)
    if sys_id is not None:
        _tensor(sys_id, "sys_id", torch.int32, (n,))
    if order is not None:
        _tensor(order, "order", torch.int64, (n,))
    return n


def _obs_tensors(out: dict, n: int) -> None:
    import torch
    for f in OBS_FIELDS:
        dt = torch.float64 if f in ("theta_s", "dp", "dE_ion", "t_final", "t_first_bounce", "t_last_bounce") \
            else torch.int32
        if f not in out:
            raise IaArgumentError(f"out[{f!r}]: missing")
        _tensor(out[f], f"out[{f!r}]", dt, (None,))
        if out[f].shape[0] < n:
            raise IaArgumentError(f"out[{f!r}]: {out[f].shape[0]} elements for {n} trajectories")
    if out.get("y_final") is not None:
        _tensor(out["y_final"], "out['y_final']", torch.float64, (12, n))


class ia_system_desc(ctypes.Structure):
    _fields_ = [
        ("m_ion", ctypes.c_double), ("m_atom", ctypes.c_double),
        ("alpha", ctypes.c_double), ("De", ctypes.c_double), ("Omega", ctypes.c_double),
        ("a", ctypes.c_double * 3), ("q", ctypes.c_double * 3),
        ("r0", ctypes.c_double), ("t_max", ctypes.c_double), ("rtol", ctypes.c_double),
        ("atol_pos", ctypes.c_double), ("atol_vel", ctypes.c_double), ("h_max", ctypes.c_double),
        ("rf_sign", ctypes.c_int32), ("reserved", ctypes.c_int32), ("max_attempts", ctypes.c_int64),
    ]


class ia_ic_soa(ctypes.Structure):
    _fields_ = [("y0", ctypes.c_void_p), ("phi0", ctypes.c_void_p), ("sys_id", ctypes.c_void_p),
                ("order", ctypes.c_void_p), ("ld", ctypes.c_int64)]


class ia_obs_soa(ctypes.Structure):
    _fields_ = [("theta_s", ctypes.c_void_p), ("dp", ctypes.c_void_p), ("dE_ion", ctypes.c_void_p),
                ("t_final", ctypes.c_void_p), ("t_first_bounce", ctypes.c_void_p),
                ("t_last_bounce", ctypes.c_void_p), ("n_bounce", ctypes.c_void_p),
                ("status", ctypes.c_void_p), ("n_steps", ctypes.c_void_p), ("n_rej", ctypes.c_void_p),
                ("y_final", ctypes.c_void_p), ("ld", ctypes.c_int64)]


class ia_launch_opts(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("block", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("refill", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("regs_variant", ctypes.c_int32), ("slice_budget", ctypes.c_int32),
                ("tail_group", ctypes.c_int32), ("tail_blocks_per_sm", ctypes.c_int32),
                ("tail_sms", ctypes.c_int32), ("tail_pair", ctypes.c_int32), ("tail_warps", ctypes.c_int32),
                ("suspend_capacity", ctypes.c_int64), ("scratch", ctypes.c_void_p), ("scratch_bytes", ctypes.c_int64)]


class ia_tangent_in(ctypes.Structure):
    _fields_ = [("dy0", ctypes.c_void_p), ("dq", (ctypes.c_double * 3) * 4), ("ndir", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("ld", ctypes.c_int64)]


class ia_adjoint_opts(ctypes.Structure):
    _fields_ = [("seg", ctypes.c_int32), ("max_ckpt", ctypes.c_int32), ("warps", ctypes.c_int64),
                ("scratch", ctypes.c_void_p), ("scratch_bytes", ctypes.c_int64)]


class ia_adjoint_out(ctypes.Structure):
    _fields_ = [("grad_y0", ctypes.c_void_p), ("grad_q", ctypes.c_void_p), ("d_theta_s", ctypes.c_void_p),
                ("d_dp", ctypes.c_void_p), ("d_dE_ion", ctypes.c_void_p), ("d_t_final", ctypes.c_void_p),
                ("ld", ctypes.c_int64)]


class ia_tangent_out(ctypes.Structure):
    _fields_ = [("d_theta_s", ctypes.c_void_p), ("d_dp", ctypes.c_void_p), ("d_dE_ion", ctypes.c_void_p),
                ("d_t_final", ctypes.c_void_p), ("dy_final", ctypes.c_void_p), ("ftle", ctypes.c_void_p),
                ("ld", ctypes.c_int64)]


class ia_sampler(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("random_phase", ctypes.c_int32), ("micromotion", ctypes.c_int32),
                ("rf_sign", ctypes.c_int32), ("m_ion", ctypes.c_double), ("m_atom", ctypes.c_double),
                ("Omega", ctypes.c_double), ("q", ctypes.c_double * 3), ("r0", ctypes.c_double),
                ("E", ctypes.c_double), ("kT", ctypes.c_double), ("kT_ion", ctypes.c_double),
                ("b_max", ctypes.c_double), ("phase", ctypes.c_double), ("seed", ctypes.c_uint64)]


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the compiled library (building it in-tree first if allowed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise IaError(f"CUDA library not built: {path}")
        _build.build()
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    L.ia_system_create.argtypes = [P(ia_system_desc), ctypes.c_int32, P(ctypes.c_void_p)]
    L.ia_system_create.restype = ctypes.c_int
    L.ia_system_destroy.argtypes = [ctypes.c_void_p]
    L.ia_system_destroy.restype = ctypes.c_int
    L.ia_system_count.argtypes = [ctypes.c_void_p]
    L.ia_system_count.restype = ctypes.c_int
    L.ia_launch.argtypes = [ctypes.c_void_p, P(ia_ic_soa), ctypes.c_int64, P(ia_obs_soa),
                            P(ia_launch_opts), ctypes.c_void_p]
    L.ia_launch.restype = ctypes.c_int
    L.ia_launch_static.argtypes = [ctypes.c_void_p, P(ia_ic_soa), ctypes.c_int64, P(ia_obs_soa),
                                   P(ia_launch_opts), ctypes.c_void_p]
    L.ia_launch_static.restype = ctypes.c_int
    L.ia_reduce_stats.argtypes = [ctypes.c_void_p, P(ia_obs_soa), ctypes.c_int64, ctypes.c_void_p, ctypes.c_int32,
                                  ctypes.c_void_p, ctypes.c_void_p]
    L.ia_reduce_stats.restype = ctypes.c_int
    L.ia_reserve_stats.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32]
    L.ia_reserve_stats.restype = ctypes.c_int
    L.ia_graph_create.argtypes = [ctypes.c_void_p, P(ia_ic_soa), ctypes.c_int64, P(ia_obs_soa), P(ia_launch_opts),
                                  ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                  P(ctypes.c_void_p)]
    L.ia_graph_create.restype = ctypes.c_int
    L.ia_graph_launch.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    L.ia_graph_launch.restype = ctypes.c_int
    L.ia_graph_destroy.argtypes = [ctypes.c_void_p]
    L.ia_graph_destroy.restype = ctypes.c_int
    L.ia_autotune.argtypes = [ctypes.c_void_p, P(ia_ic_soa), ctypes.c_int64, ctypes.c_int32, P(ia_launch_opts),
                              P(ia_launch_opts), P(ctypes.c_double), ctypes.c_void_p]
    L.ia_autotune.restype = ctypes.c_int
    L.ia_launch_tangent.argtypes = [ctypes.c_void_p, P(ia_ic_soa), ctypes.c_int64, P(ia_obs_soa),
                                    P(ia_tangent_in), P(ia_tangent_out), ctypes.c_void_p]
    L.ia_launch_tangent.restype = ctypes.c_int
    L.ia_launch_phases.argtypes = [ctypes.c_void_p, ctypes.c_void_p, P(ctypes.c_double), P(ctypes.c_double),
                                   P(ctypes.c_int64)]
    L.ia_launch_phases.restype = ctypes.c_int
    L.ia_adjoint_scratch_bytes.argtypes = [ctypes.c_void_p, ctypes.c_int64, P(ia_adjoint_opts)]
    L.ia_adjoint_scratch_bytes.restype = ctypes.c_int64
    L.ia_launch_adjoint.argtypes = [ctypes.c_void_p, P(ia_ic_soa), ctypes.c_int64, P(ia_obs_soa),
                                    P(ia_tangent_in), P(ia_adjoint_out), P(ia_adjoint_opts), ctypes.c_void_p]
    L.ia_launch_adjoint.restype = ctypes.c_int
    L.ia_scratch_bytes.argtypes = [ctypes.c_int64, P(ia_launch_opts)]
    L.ia_scratch_bytes.restype = ctypes.c_int64
    L.ia_reserve.argtypes = [ctypes.c_void_p, ctypes.c_int64, P(ia_launch_opts)]
    L.ia_reserve.restype = ctypes.c_int
    L.ia_rcp_check.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    L.ia_rcp_check.restype = ctypes.c_int
    L.ia_philox4x64.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                ctypes.c_void_p, ctypes.c_void_p]
    L.ia_philox4x64.restype = ctypes.c_int
    L.ia_sample_ics.argtypes = [P(ia_sampler), ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_int64, ctypes.c_void_p]
    L.ia_sample_ics.restype = ctypes.c_int
    L.ia_fp64_peak.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, P(ctypes.c_double)]
    L.ia_fp64_peak.restype = ctypes.c_int
    L.ia_static_phases.argtypes = [ctypes.c_void_p, P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_int64)]
    L.ia_static_phases.restype = ctypes.c_int
    L.ia_queue_create.argtypes = [ctypes.c_void_p, ctypes.c_int64, P(ia_launch_opts), P(ctypes.c_void_p)]
    L.ia_queue_create.restype = ctypes.c_int
    L.ia_queue_launch.argtypes = [ctypes.c_void_p, P(ia_ic_soa), P(ia_obs_soa), ctypes.c_int64, ctypes.c_void_p]
    L.ia_queue_launch.restype = ctypes.c_int
    L.ia_queue_reset.argtypes = [ctypes.c_void_p]
    L.ia_queue_reset.restype = ctypes.c_int
    L.ia_queue_state.argtypes = [ctypes.c_void_p, P(ctypes.c_int64), P(ctypes.c_int64), P(ctypes.c_int64)]
    L.ia_queue_state.restype = ctypes.c_int
    L.ia_queue_phases.argtypes = [ctypes.c_void_p, P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_int64)]
    L.ia_queue_phases.restype = ctypes.c_int
    L.ia_queue_destroy.argtypes = [ctypes.c_void_p]
    L.ia_queue_destroy.restype = ctypes.c_int
    L.ia_error_string.argtypes = [ctypes.c_int]
    L.ia_error_string.restype = ctypes.c_char_p
    L.ia_version.restype = ctypes.c_int
    _lib = L
    return L


def _check(code: int):
    if code != IA_OK:
        raise IaError(f"{load().ia_error_string(code).decode()} ({code})")


def make_desc(d: dict) -> ia_system_desc:
    s = ia_system_desc()
    for k in ("m_ion", "m_atom", "alpha", "De", "Omega", "r0", "t_max", "rtol", "atol_pos", "atol_vel",
              "h_max"):
        setattr(s, k, float(d[k]))
    for j in range(3):
        s.a[j] = float(d["a"][j])
        s.q[j] = float(d["q"][j])
    s.rf_sign = int(d.get("rf_sign", 1))
    s.reserved = 0
    s.max_attempts = int(d.get("max_attempts", 50_000_000))
    return s


def ia_system_create(systems) -> int:
    """Create a device table from a list of descriptor dicts; returns the opaque handle."""
    L = load()
    arr = (ia_system_desc * len(systems))(*[make_desc(d) for d in systems])
    h = ctypes.c_void_p()
    _check(L.ia_system_create(arr, len(systems), ctypes.byref(h)))
    return h.value


def ia_system_destroy(handle: int) -> None:
    _check(load().ia_system_destroy(handle))


def ia_system_count(handle: int) -> int:
    n = load().ia_system_count(handle)
    if n < 0:
        _check(n)
    return n


def ia_fp64_peak(blocks_per_sm: int = 4, iters: int = 20000, stream=None) -> float:
    out = ctypes.c_double()
    _check(load().ia_fp64_peak(blocks_per_sm, iters, _stream_ptr(stream), ctypes.byref(out)))
    return out.value


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


OBS_FIELDS = ("theta_s", "dp", "dE_ion", "t_final", "t_first_bounce", "t_last_bounce", "n_bounce",
              "status", "n_steps", "n_rej")


def alloc_obs(n: int, device="cuda", y_final: bool = False) -> dict:
    """Device output tensors for n trajectories (torch owns them)."""
    import torch
    out = {}
    for f in ("theta_s", "dp", "dE_ion", "t_final", "t_first_bounce", "t_last_bounce"):
        out[f] = torch.empty(n, dtype=torch.float64, device=device)
    out["n_bounce"] = torch.empty(n, dtype=torch.int32, device=device)
    out["status"] = torch.empty(n, dtype=torch.int32, device=device)  # bit pattern of uint32
    out["n_steps"] = torch.empty(n, dtype=torch.int32, device=device)
    out["n_rej"] = torch.empty(n, dtype=torch.int32, device=device)
    if y_final:
        out["y_final"] = torch.empty((12, n), dtype=torch.float64, device=device)
    return out


def _obs_struct(out: dict, n: int) -> ia_obs_soa:
    _obs_tensors(out, n)
    o = ia_obs_soa()
    for f in OBS_FIELDS:
        setattr(o, f, out[f].data_ptr())
    yf = out.get("y_final")
    o.y_final = yf.data_ptr() if yf is not None else None
    o.ld = n if yf is not None else 0
    return o


def to_device_soa(y0, phi0, sys_id=None, device="cuda"):
    """(n, 12) state and (n,) phases (numpy or torch) -> SoA device tensors."""
    import torch
    y0 = torch.as_tensor(np.ascontiguousarray(y0) if isinstance(y0, np.ndarray) else y0, dtype=torch.float64)
    y0_soa = y0.to(device).t().contiguous()
    ph = torch.as_tensor(phi0, dtype=torch.float64).to(device).contiguous()
    sid = None
    if sys_id is not None:
        sid = torch.as_tensor(sys_id, dtype=torch.int32).to(device).contiguous()
    return y0_soa, ph, sid


def make_opts(kernel: int = IA_KERNEL_PERSISTENT, block: int = 0, grid: int = 0, refill: int = 0,
              blocks_per_sm: int = 0, regs_variant: int = 0, slice_budget: int = 0, tail_group: int = 0,
              tail_blocks_per_sm: int = 0, suspend_capacity: int = 0, scratch=None,
              tail_sms: int = 0, tail_pair: int = 0, tail_warps: int = 0) -> ia_launch_opts:
    opts = ia_launch_opts()
    opts.kernel = kernel
    opts.block = block
    opts.grid = grid
    opts.refill = refill
    opts.blocks_per_sm = blocks_per_sm
    opts.regs_variant = regs_variant
    opts.slice_budget = slice_budget
    opts.tail_group = tail_group
    opts.tail_blocks_per_sm = tail_blocks_per_sm
    opts.suspend_capacity = suspend_capacity
    opts.tail_sms = tail_sms
    opts.tail_pair = tail_pair
    opts.tail_warps = tail_warps
    if scratch is not None:
        _tensor(scratch, "scratch", scratch.dtype, (None,) * scratch.dim())
        opts.scratch = scratch.data_ptr()
        opts.scratch_bytes = scratch.numel() * scratch.element_size()
    return opts


def ia_scratch_bytes(n: int, **kw) -> int:
    v = load().ia_scratch_bytes(n, ctypes.byref(make_opts(**kw)))
    if v < 0:
        _check(int(v))
    return int(v)


def ia_reserve(handle: int, n: int, **kw) -> None:
    _check(load().ia_reserve(handle, n, ctypes.byref(make_opts(**kw))))


def ia_rcp_check(x, y, stream=None) -> None:
    import torch
    _tensor(x, "x", torch.float64, (None,))
    _tensor(y, "y", torch.float64, (x.shape[0],))
    _check(load().ia_rcp_check(x.data_ptr(), y.data_ptr(), int(x.numel()), _stream_ptr(stream)))


def make_sampler(kind: int, desc: dict, seed: int, E: float = 0.0, kT: float = 0.0, kT_ion: float = 0.0,
                 b_max: float = 0.0, random_phase: bool = True, phase: float = 0.0,
                 micromotion: bool = False) -> ia_sampler:
    """ia_sampler for the system of a descriptor dict (masses, Omega, q, r0 and rf sign taken from it)."""
    s = ia_sampler()
    s.kind = int(kind)
    s.random_phase = int(bool(random_phase))
    s.micromotion = int(bool(micromotion))
    s.rf_sign = int(desc.get("rf_sign", 1))
    s.m_ion = float(desc["m_ion"])
    s.m_atom = float(desc["m_atom"])
    s.Omega = float(desc["Omega"])
    for j in range(3):
        s.q[j] = float(desc["q"][j])
    s.r0 = float(desc["r0"])
    s.E, s.kT, s.kT_ion, s.b_max, s.phase = float(E), float(kT), float(kT_ion), float(b_max), float(phase)
    s.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return s


def ia_sample_ics(sampler: ia_sampler, first: int, y0_soa, phi0, stream=None) -> None:
    """Fill device tensors y0_soa (12, n) float64 (row stride = ld) and phi0 (n,) with the initial
    conditions of trajectories first .. first + n - 1."""
    import torch
    _tensor(phi0, "phi0", torch.float64, (None,))
    n = int(phi0.shape[0])
    _tensor(y0_soa, "y0_soa", torch.float64, (12, n), contiguous=False)
    ld = int(y0_soa.stride(0)) if n > 0 else 0
    _check(load().ia_sample_ics(ctypes.byref(sampler), int(first), n, y0_soa.data_ptr(), phi0.data_ptr(), ld,
                                _stream_ptr(stream)))


def ia_philox4x64(key0: int, key1: int, ctr1: int, first: int, out, stream=None) -> None:
    """Raw Philox4x64-10 blocks into a device tensor out (n_blocks, 4) of int64 (the words' bits)."""
    import torch
    _tensor(out, "out", torch.int64, (None, 4))
    m = 0xFFFFFFFFFFFFFFFF
    _check(load().ia_philox4x64(int(key0) & m, int(key1) & m, int(ctr1) & m, int(first), int(out.shape[0]),
                                out.data_ptr(), _stream_ptr(stream)))


def _ic_struct(y0_soa, phi0, sys_id, order) -> ia_ic_soa:
    n = _ic_tensors(y0_soa, phi0, sys_id, order)
    ic = ia_ic_soa()
    ic.y0 = y0_soa.data_ptr()
    ic.phi0 = phi0.data_ptr()
    ic.sys_id = sys_id.data_ptr() if sys_id is not None else None
    ic.order = order.data_ptr() if order is not None else None
    ic.ld = int(y0_soa.stride(0)) if n > 0 else 0
    return ic


def ia_launch(handle: int, y0_soa, phi0, sys_id, out: dict, kernel: int = IA_KERNEL_PERSISTENT,
              stream=None, order=None, **kw) -> None:
    """Launch on device tensors: y0_soa (12, n) float64, phi0 (n,), sys_id (n,) int32 or None,
    order (n,) int64 permutation or None. Keyword options are the fields of ia_launch_opts."""
    n = int(phi0.shape[0])
    ic = _ic_struct(y0_soa, phi0, sys_id, order)
    o = _obs_struct(out, n)
    opts = make_opts(kernel=kernel, **kw)
    _check(load().ia_launch(handle, ctypes.byref(ic), n, ctypes.byref(o), ctypes.byref(opts),
                            _stream_ptr(stream)))


def ia_launch_static(handle: int, y0_soa, phi0, sys_id, out: dict, stream=None, order=None, **kw) -> None:
    """Persistent launch whose scratch is the library's fixed device array (allocates nothing).
    Same tensors as ia_launch; keyword options as make_opts (kernel is always persistent)."""
    n = int(phi0.shape[0])
    ic = _ic_struct(y0_soa, phi0, sys_id, order)
    o = _obs_struct(out, n)
    opts = make_opts(kernel=IA_KERNEL_PERSISTENT, **kw)
    _check(load().ia_launch_static(handle, ctypes.byref(ic), n, ctypes.byref(o), ctypes.byref(opts),
                                   _stream_ptr(stream)))


def ia_static_phases(handle: int) -> tuple:
    """(lane-phase ms, total ms, bounded waits that ran out) of the last ia_launch_static on the current
    device, read from the library's fixed array; synchronous."""
    a, b, e = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    _check(load().ia_static_phases(handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(e)))
    return a.value, b.value, e.value


def alloc_stats(n_cells: int, device="cuda"):
    """Device buffer for n_cells ia_stats records (raw bytes)."""
    import torch
    return torch.empty(n_cells * STATS_DTYPE.itemsize, dtype=torch.uint8, device=device)


def ia_reduce_stats(handle: int, out: dict, n: int, cell_id, n_cells: int, stats, stream=None) -> None:
    """Reduce device observables into the device stats buffer (see alloc_stats)."""
    import torch
    o = _obs_struct(out, n)
    if cell_id is not None:
        _tensor(cell_id, "cell_id", torch.int32, (None,))
        if cell_id.shape[0] < n:
            raise IaArgumentError(f"cell_id: {cell_id.shape[0]} elements for {n} trajectories")
    _stats_tensor(stats, n_cells)
    _check(load().ia_reduce_stats(handle, ctypes.byref(o), n, cell_id.data_ptr() if cell_id is not None else None,
                                  n_cells, stats.data_ptr(), _stream_ptr(stream)))


def _stats_tensor(stats, n_cells: int) -> None:
    import torch
    _tensor(stats, "stats", torch.uint8, (None,))
    if stats.numel() < max(int(n_cells), 0) * STATS_DTYPE.itemsize:
        raise IaArgumentError(f"stats: {stats.numel()} bytes for {n_cells} records")


def ia_reserve_stats(handle: int, n: int, n_cells: int) -> None:
    _check(load().ia_reserve_stats(handle, n, n_cells))


def stats_to_numpy(stats) -> np.ndarray:
    return np.frombuffer(stats.cpu().numpy().tobytes(), dtype=STATS_DTYPE).copy()


class Graph:
    """A captured batch (persistent launch + optional statistics) replayed with ia_graph_launch."""

    def __init__(self, handle: int, y0_soa, phi0, sys_id, out: dict, stream, order=None, cell_id=None,
                 n_cells: int = 0, stats=None, **kw):
        import torch
        n = int(phi0.shape[0])
        self.ptr = None
        self._keep = (y0_soa, phi0, sys_id, out, order, cell_id, stats)
        ic = _ic_struct(y0_soa, phi0, sys_id, order)
        o = _obs_struct(out, n)
        if cell_id is not None:
            _tensor(cell_id, "cell_id", torch.int32, (n,))
        if stats is not None:
            _stats_tensor(stats, n_cells)
        opts = make_opts(kernel=IA_KERNEL_PERSISTENT, **kw)
        g = ctypes.c_void_p()
        _check(load().ia_graph_create(handle, ctypes.byref(ic), n, ctypes.byref(o), ctypes.byref(opts),
                                      cell_id.data_ptr() if cell_id is not None else None, n_cells,
                                      stats.data_ptr() if stats is not None else None,
                                      ctypes.c_void_p(stream.cuda_stream), ctypes.byref(g)))
        self.ptr = g.value

    def launch(self, stream) -> None:
        _check(load().ia_graph_launch(self.ptr, ctypes.c_void_p(stream.cuda_stream)))

    def close(self) -> None:
        if self.ptr:
            _check(load().ia_graph_destroy(self.ptr))
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ia_autotune(handle: int, y0_soa, phi0, sys_id, attempt_cap: int = 1024, order=None, stream=None, **base):
    """Lane-phase autotuner on a sample (device tensors); returns (options dict, best ms)."""
    n = int(phi0.shape[0])
    ic = _ic_struct(y0_soa, phi0, sys_id, order)
    b = make_opts(kernel=IA_KERNEL_PERSISTENT, **base)
    best = ia_launch_opts()
    ms = ctypes.c_double()
    _check(load().ia_autotune(handle, ctypes.byref(ic), n, attempt_cap, ctypes.byref(b), ctypes.byref(best),
                              ctypes.byref(ms), _stream_ptr(stream)))
    return {"block": best.block, "regs_variant": best.regs_variant, "refill": best.refill}, ms.value


def alloc_tangent(n: int, ndir: int, dy_final: bool = False, ftle: bool = True, device="cuda") -> dict:
    import torch
    t = {k: torch.empty((ndir, n), dtype=torch.float64, device=device)
         for k in ("d_theta_s", "d_dp", "d_dE_ion", "d_t_final")}
    if dy_final:
        t["dy_final"] = torch.empty((ndir, 12, n), dtype=torch.float64, device=device)
    if ftle:
        t["ftle"] = torch.empty(n, dtype=torch.float64, device=device)
    return t


def ia_launch_tangent(handle: int, y0_soa, phi0, sys_id, out: dict, dy0, dq, tan: dict, stream=None) -> None:
    """Tangent launch: dy0 (ndir, 12, n) device float64 (d y0 / d p_k), dq (ndir, 3) host (d q / d p_k)."""
    import torch
    n = int(phi0.shape[0])
    ic = _ic_struct(y0_soa, phi0, sys_id, None)
    o = _obs_struct(out, n)
    _tensor(dy0, "dy0", torch.float64, (None, 12, n))
    ndir = int(dy0.shape[0])
    if not 1 <= ndir <= 4:
        raise IaArgumentError(f"dy0: {ndir} directions, expected 1..4")
    for k in ("d_theta_s", "d_dp", "d_dE_ion", "d_t_final"):
        _tensor(tan.get(k), f"tan[{k!r}]", torch.float64, (ndir, n))
    if "dy_final" in tan:
        _tensor(tan["dy_final"], "tan['dy_final']", torch.float64, (ndir, 12, n))
    if "ftle" in tan:
        _tensor(tan["ftle"], "tan['ftle']", torch.float64, (n,))
    dq = np.asarray(dq, dtype=np.float64)
    if dq.ndim != 2 or dq.shape[0] < ndir or dq.shape[1] != 3:
        raise IaArgumentError(f"dq: shape {dq.shape}, expected ({ndir}, 3)")
    ti = ia_tangent_in()
    ti.dy0 = dy0.data_ptr()
    for k in range(ndir):
        for j in range(3):
            ti.dq[k][j] = float(dq[k, j])
    ti.ndir = ndir
    ti.reserved = 0
    ti.ld = n
    to = ia_tangent_out()
    to.d_theta_s = tan["d_theta_s"].data_ptr()
    to.d_dp = tan["d_dp"].data_ptr()
    to.d_dE_ion = tan["d_dE_ion"].data_ptr()
    to.d_t_final = tan["d_t_final"].data_ptr()
    to.dy_final = tan["dy_final"].data_ptr() if "dy_final" in tan else None
    to.ftle = tan["ftle"].data_ptr() if "ftle" in tan else None
    to.ld = n
    _check(load().ia_launch_tangent(handle, ctypes.byref(ic), n, ctypes.byref(o), ctypes.byref(ti), ctypes.byref(to),
                                    _stream_ptr(stream)))


def ia_launch_phases(handle: int, scratch=None) -> tuple:
    """(lane-phase ms, total ms, bounded waits that ran out) of the last persistent launch on
    `scratch` (a device tensor) or on the system's own scratch; synchronous."""
    a, b, e = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    _check(load().ia_launch_phases(handle, scratch.data_ptr() if scratch is not None else None,
                                   ctypes.byref(a), ctypes.byref(b), ctypes.byref(e)))
    return a.value, b.value, e.value


OBJECTIVES = ("theta_s", "dp", "dE_ion", "t_final")


def make_adjoint_opts(seg: int = 0, max_ckpt: int = 0, warps: int = 0, scratch=None) -> ia_adjoint_opts:
    o = ia_adjoint_opts()
    o.seg = int(seg)
    o.max_ckpt = int(max_ckpt)
    o.warps = int(warps)
    if scratch is not None:
        _tensor(scratch, "scratch", scratch.dtype, (None,) * scratch.dim())
        o.scratch = scratch.data_ptr()
        o.scratch_bytes = scratch.numel() * scratch.element_size()
    return o


def ia_adjoint_scratch_bytes(handle, n: int, **opts) -> int:
    """Scratch bytes of an adjoint launch (handle may be None when warps > 0)."""
    o = make_adjoint_opts(**opts)
    r = load().ia_adjoint_scratch_bytes(handle, int(n), ctypes.byref(o))
    if r < 0:
        _check(int(r))
    return int(r)


def alloc_adjoint(n: int, ndir: int = 0, grad_y0: bool = True, grad_q: bool = True, device="cuda") -> dict:
    import torch
    a = {}
    if grad_y0:
        a["grad_y0"] = torch.empty((4, 12, n), dtype=torch.float64, device=device)
    if grad_q:
        a["grad_q"] = torch.empty((4, 3, n), dtype=torch.float64, device=device)
    for k in ("d_theta_s", "d_dp", "d_dE_ion", "d_t_final"):
        if ndir > 0:
            a[k] = torch.empty((ndir, n), dtype=torch.float64, device=device)
    return a


def ia_launch_adjoint(handle: int, y0_soa, phi0, sys_id, out: dict, adj: dict, dy0=None, dq=None, stream=None,
                      **opts) -> None:
    """Adjoint launch: gradients of (theta_s, dp, dE_ion, t_final) w.r.t. y0 and q into adj["grad_y0"]
    (4, 12, n) and adj["grad_q"] (4, 3, n); with seeds dy0 (ndir, 12, n) device and dq (ndir, 3) host,
    their projections into adj["d_theta_s"] .. adj["d_t_final"] (ndir, n). opts: seg, max_ckpt, warps,
    scratch (a device tensor)."""
    import torch
    n = int(phi0.shape[0])
    ic = _ic_struct(y0_soa, phi0, sys_id, None)
    o = _obs_struct(out, n)
    if "grad_y0" in adj:
        _tensor(adj["grad_y0"], "adj['grad_y0']", torch.float64, (4, 12, n))
    if "grad_q" in adj:
        _tensor(adj["grad_q"], "adj['grad_q']", torch.float64, (4, 3, n))
    ti = None
    if dy0 is not None:
        _tensor(dy0, "dy0", torch.float64, (None, 12, n))
        ti = ia_tangent_in()
        ndir = int(dy0.shape[0])
        if not 1 <= ndir <= 4:
            raise IaArgumentError(f"dy0: {ndir} directions, expected 1..4")
        for k in ("d_theta_s", "d_dp", "d_dE_ion", "d_t_final"):
            _tensor(adj.get(k), f"adj[{k!r}]", torch.float64, (ndir, n))
        ti.dy0 = dy0.data_ptr()
        dqa = np.zeros((4, 3)) if dq is None else np.asarray(dq, dtype=np.float64)
        if dqa.ndim != 2 or dqa.shape[0] < ndir or dqa.shape[1] != 3:
            raise IaArgumentError(f"dq: shape {dqa.shape}, expected ({ndir}, 3)")
        for k in range(ndir):
            for j in range(3):
                ti.dq[k][j] = float(dqa[k, j])
        ti.ndir = ndir
        ti.reserved = 0
        ti.ld = n
    ao = ia_adjoint_out()
    for k in ("grad_y0", "grad_q", "d_theta_s", "d_dp", "d_dE_ion", "d_t_final"):
        setattr(ao, k, adj[k].data_ptr() if k in adj else None)
    ao.ld = n
    op = make_adjoint_opts(**opts)
    _check(load().ia_launch_adjoint(handle, ctypes.byref(ic), n, ctypes.byref(o),
                                    ctypes.byref(ti) if ti is not None else None, ctypes.byref(ao),
                                    ctypes.byref(op), _stream_ptr(stream)))


class Queue:
    """Work queue of one batch of n trajectories integrated over several launches (ia_queue_*).

    Each launch() starts the next `count` queue positions and continues what earlier parts left
    running; the part whose count reaches n finishes the batch. The tensors (the whole batch) must be
    the same in every part of a batch."""

    def __init__(self, handle: int, n: int, **kw):
        self.ptr = None
        self.n = int(n)
        opts = make_opts(kernel=IA_KERNEL_PERSISTENT, **kw)
        q = ctypes.c_void_p()
        _check(load().ia_queue_create(handle, self.n, ctypes.byref(opts), ctypes.byref(q)))
        self.ptr = q.value

    def launch(self, y0_soa, phi0, sys_id, out: dict, count: int, order=None, stream=None) -> None:
        n = int(phi0.shape[0])
        if n != self.n:
            raise IaArgumentError(f"phi0: {n} trajectories, the queue holds {self.n}")
        ic = _ic_struct(y0_soa, phi0, sys_id, order)
        o = _obs_struct(out, n)
        _check(load().ia_queue_launch(self.ptr, ctypes.byref(ic), ctypes.byref(o), int(count), _stream_ptr(stream)))

    def reset(self) -> None:
        _check(load().ia_queue_reset(self.ptr))

    def state(self) -> tuple:
        """(positions started, parts launched, n)."""
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().ia_queue_state(self.ptr, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def phases(self) -> tuple:
        """(lane-phase ms, total ms, bounded waits that ran out) of the latest part; synchronous."""
        a, b, e = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
        _check(load().ia_queue_phases(self.ptr, ctypes.byref(a), ctypes.byref(b), ctypes.byref(e)))
        return a.value, b.value, e.value

    def close(self) -> None:
        if self.ptr:
            _check(load().ia_queue_destroy(self.ptr))
            self.ptr = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class System:
    """Owns an ia_system handle (device parameter table)."""

    def __init__(self, systems):
        self.systems = [dict(s) for s in systems]
        self.handle = ia_system_create(self.systems)

    def close(self):
        if self.handle:
            ia_system_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, y0, phi0, sys_id=None, kernel: int = IA_KERNEL_PERSISTENT, y_final: bool = False,
            **launch_kw) -> dict:
        """Integrate a batch given on the host or device; returns device tensors (synchronised)."""
        import torch
        y0_soa, ph, sid = to_device_soa(y0, phi0, sys_id)
        n = int(ph.shape[0])
        out = alloc_obs(n, y_final=y_final)
        ia_launch(self.handle, y0_soa, ph, sid, out, kernel=kernel, **launch_kw)
        torch.cuda.synchronize()
        return out


def to_numpy(out: dict) -> dict:
    r = {}
    for k, v in out.items():
        a = v.cpu().numpy()
        if k == "status":
            a = a.view(np.uint32)
        if k == "y_final":
            a = a.T.copy()
        r[k] = a
    return r
