"""ctypes front end of the CPU FP64 oracle (``ia_oracle.c`` and ``ia_sample_oracle.c``).

TEST INFRASTRUCTURE, NOT PRODUCT CODE: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this module. It shares no
code with the CUDA library; both receive the same seeded initial conditions from
``paper_2509_15117_gb300.inputs``.

The C source restates the method of arXiv 2509.15117: Eq. 1's equations of motion, V(r) = C8/r^8 -
C4/r^4 with C4 = alpha/2 and C8 = C4^2/(4 D_e), the Dormand-Prince 5(4) integrator of Dormand & Prince
(1980) / Shampine & Reichelt (1997) with ode45's step control, the outward crossing of r0 as the end
of a head-on or thermal trajectory, and the Fig. 1 observables. The second source restates the
Philox4x64-10 generator (Salmon et al., SC'11) and the samplers of the paper's head-on and thermal
runs, against which the library's device-drawn initial conditions are checked.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ia_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "ia_sample_oracle.c")]
_LIB = os.path.join(_HERE, "libia_oracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=c11"]

# status bits of the oracle (its own numbering; the CUDA library defines its own)
EXIT = 0
TMAX = 1 << 0
MAX_STEPS = 1 << 1
H_UNDERFLOW = 1 << 2
NONFINITE = 1 << 3
BAD_IC = 1 << 4
EXIT_OUTSIDE = 1 << 5
COMPLEX = 1 << 8


class OrcSystem(ctypes.Structure):
    _fields_ = [
        ("m_ion", ctypes.c_double), ("m_atom", ctypes.c_double),
        ("alpha", ctypes.c_double), ("De", ctypes.c_double),
        ("Omega", ctypes.c_double),
        ("a", ctypes.c_double * 3), ("q", ctypes.c_double * 3),
        ("r0", ctypes.c_double), ("t_max", ctypes.c_double),
        ("rtol", ctypes.c_double), ("atol_pos", ctypes.c_double), ("atol_vel", ctypes.c_double),
        ("h_max", ctypes.c_double),
        ("rf_sign", ctypes.c_int32), ("pad_", ctypes.c_int32),
        ("max_attempts", ctypes.c_int64),
    ]


class OrcResult(ctypes.Structure):
    _fields_ = [
        ("theta_s", ctypes.c_double), ("dp", ctypes.c_double), ("dE_ion", ctypes.c_double),
        ("t_final", ctypes.c_double), ("t_first_bounce", ctypes.c_double),
        ("t_last_bounce", ctypes.c_double), ("y_final", ctypes.c_double * 12),
        ("n_steps", ctypes.c_int64), ("n_rej", ctypes.c_int64),
        ("n_bounce", ctypes.c_int32), ("status", ctypes.c_uint32),
    ]


class OrcSampler(ctypes.Structure):
    """Counter-based initial-condition sampler (``ia_sample_oracle.c``)."""
    _fields_ = [
        ("kind", ctypes.c_int32), ("random_phase", ctypes.c_int32),
        ("micromotion", ctypes.c_int32), ("rf_sign", ctypes.c_int32),
        ("m_ion", ctypes.c_double), ("m_atom", ctypes.c_double), ("Omega", ctypes.c_double),
        ("q", ctypes.c_double * 3), ("r0", ctypes.c_double), ("E", ctypes.c_double),
        ("kT", ctypes.c_double), ("kT_ion", ctypes.c_double), ("b_max", ctypes.c_double),
        ("phase", ctypes.c_double), ("seed", ctypes.c_uint64),
    ]


SAMPLE_HEAD_ON, SAMPLE_SPHERE, SAMPLE_DISK = 0, 1, 2

RESULT_DTYPE = np.dtype([
    ("theta_s", "<f8"), ("dp", "<f8"), ("dE_ion", "<f8"), ("t_final", "<f8"),
    ("t_first_bounce", "<f8"), ("t_last_bounce", "<f8"), ("y_final", "<f8", (12,)),
    ("n_steps", "<i8"), ("n_rej", "<i8"), ("n_bounce", "<i4"), ("status", "<u4"),
])
assert RESULT_DTYPE.itemsize == ctypes.sizeof(OrcResult)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/libia_oracle.so`` (in-tree, git-ignored)."""
    with _lock:
        if not force and os.path.exists(_LIB) and all(os.path.getmtime(_LIB) >= os.path.getmtime(p) for p in _SRCS):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", *CFLAGS, "-o", tmp, *_SRCS, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        d = ctypes.c_double
        dp = P(ctypes.c_double)
        L.orc_run_batch.argtypes = [P(OrcSystem), ctypes.c_int32, P(ctypes.c_int32), dp, dp,
                                    ctypes.c_int64, P(OrcResult), ctypes.c_int32]
        L.orc_run_batch.restype = None
        L.orc_run_batch_noise.argtypes = [P(OrcSystem), ctypes.c_int32, P(ctypes.c_int32), dp, dp,
                                          ctypes.c_int64, P(OrcResult), ctypes.c_int32, ctypes.c_uint64,
                                          ctypes.c_int32]
        L.orc_run_batch_noise.restype = None
        L.orc_potential.argtypes = [P(OrcSystem), d, dp, dp]
        L.orc_ionatom_rhs.argtypes = [P(OrcSystem), d, d, dp, dp]
        L.orc_ion_energy.argtypes = [P(OrcSystem), d, d, dp]
        L.orc_ion_energy.restype = d
        L.orc_test_solve.argtypes = [ctypes.c_int32, d, d, d, d, d, dp, P(ctypes.c_int64), P(ctypes.c_int64)]
        L.orc_test_fixed.argtypes = [ctypes.c_int32, d, d, ctypes.c_int64, dp, dp]
        L.orc_test_dense.argtypes = [ctypes.c_int32, d, d, d, dp, dp]
        _trace_types(L)
        L.orc_ionatom_fixed.argtypes = [P(OrcSystem), d, d, d, ctypes.c_int64, dp]
        L.orc_ionatom_segment.argtypes = [P(OrcSystem), d, d, d, dp, P(ctypes.c_int64), P(ctypes.c_int64)]
        L.orc_max_threads.restype = ctypes.c_int32
        u64 = ctypes.c_uint64
        L.orc_philox4x64.argtypes = [P(u64), P(u64), P(u64)]
        L.orc_philox4x64_stream.argtypes = [u64, u64, u64, ctypes.c_int64, ctypes.c_int64, P(u64)]
        L.orc_sample_ics.argtypes = [P(OrcSampler), ctypes.c_int64, ctypes.c_int64, dp, dp]
        L.orc_sample_ics.restype = ctypes.c_int
        _lib = L
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_system(desc: dict) -> OrcSystem:
    """Oracle system struct from a descriptor dict (keys of ``inputs.SystemDesc``)."""
    s = OrcSystem()
    s.m_ion = desc["m_ion"]
    s.m_atom = desc["m_atom"]
    s.alpha = desc["alpha"]
    s.De = desc["De"]
    s.Omega = desc["Omega"]
    for j in range(3):
        s.a[j] = desc["a"][j]
        s.q[j] = desc["q"][j]
    s.r0 = desc["r0"]
    s.t_max = desc["t_max"]
    s.rtol = desc["rtol"]
    s.atol_pos = desc["atol_pos"]
    s.atol_vel = desc["atol_vel"]
    s.h_max = desc["h_max"]
    s.rf_sign = int(desc.get("rf_sign", 1))
    s.max_attempts = int(desc.get("max_attempts", 50_000_000))
    return s


def max_threads() -> int:
    return int(lib().orc_max_threads())


def run_batch(systems, y0, phi0, sys_id=None, nthreads: int = 0, noise_seed: int = 0,
              noise_ulps: int = 0) -> np.ndarray:
    """Integrate every trajectory; returns a structured array with ``RESULT_DTYPE``.

    systems: list of descriptor dicts; y0: (n, 12) float64; phi0: (n,) float64; sys_id: (n,) int32.
    noise_ulps > 0: under the rounding-noise model (every component moved by up to noise_ulps ulps after
    each accepted step, drawn from noise_seed and the trajectory's position in the batch).
    """
    L = lib()
    y0 = np.ascontiguousarray(y0, dtype=np.float64)
    phi0 = np.ascontiguousarray(phi0, dtype=np.float64)
    n = y0.shape[0]
    assert y0.shape == (n, 12) and phi0.shape == (n,)
    arr = (OrcSystem * len(systems))(*[make_system(d) for d in systems])
    sid_ptr = None
    if sys_id is not None:
        sys_id = np.ascontiguousarray(sys_id, dtype=np.int32)
        assert sys_id.shape == (n,)
        sid_ptr = sys_id.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    out = np.zeros(n, dtype=RESULT_DTYPE)
    if noise_ulps > 0:
        L.orc_run_batch_noise(arr, len(systems), sid_ptr, _dptr(y0), _dptr(phi0), n,
                              out.ctypes.data_as(ctypes.POINTER(OrcResult)), int(nthreads),
                              int(noise_seed) & 0xFFFFFFFFFFFFFFFF, int(noise_ulps))
    else:
        L.orc_run_batch(arr, len(systems), sid_ptr, _dptr(y0), _dptr(phi0), n,
                        out.ctypes.data_as(ctypes.POINTER(OrcResult)), int(nthreads))
    return out


def potential(desc: dict, r: float):
    s = make_system(desc)
    V = ctypes.c_double()
    dV = ctypes.c_double()
    lib().orc_potential(ctypes.byref(s), r, ctypes.byref(V), ctypes.byref(dV))
    return V.value, dV.value


def rhs(desc: dict, phi0: float, t: float, y) -> np.ndarray:
    s = make_system(desc)
    y = np.ascontiguousarray(y, dtype=np.float64)
    f = np.zeros(12)
    lib().orc_ionatom_rhs(ctypes.byref(s), phi0, t, _dptr(y), _dptr(f))
    return f


def ion_energy(desc: dict, phi0: float, t: float, y) -> float:
    s = make_system(desc)
    y = np.ascontiguousarray(y, dtype=np.float64)
    return float(lib().orc_ion_energy(ctypes.byref(s), phi0, t, _dptr(y)))


def test_solve(kind: int, p: float, t_end: float, y0, rtol: float, atol: float, hmax: float):
    y = np.array(y0, dtype=np.float64)
    ns = ctypes.c_int64()
    nr = ctypes.c_int64()
    lib().orc_test_solve(kind, p, t_end, rtol, atol, hmax, _dptr(y), ctypes.byref(ns), ctypes.byref(nr))
    return y, ns.value, nr.value


def test_fixed(kind: int, p: float, h: float, nsteps: int, y0):
    y = np.array(y0, dtype=np.float64)
    err = np.zeros_like(y)
    lib().orc_test_fixed(kind, p, h, nsteps, _dptr(y), _dptr(err))
    return y, err


def _trace_types(L):
    d = ctypes.c_double
    dp = ctypes.POINTER(ctypes.c_double)
    L.orc_test_trace.argtypes = [ctypes.c_int32, d, d, d, d, d, d, dp, ctypes.c_int64, dp, dp, dp,
                                 ctypes.POINTER(ctypes.c_int32)]
    L.orc_test_trace.restype = ctypes.c_int64


def build_variant(defines: dict, workdir: str):
    """A copy of the oracle compiled with some of its macros redefined (``{"ORC_CTRL_SAFETY": 0.9}``),
    loaded from `workdir`: the tests plant a mistake in the oracle this way and check that its pins
    catch it. Only the test-problem hooks are typed."""
    tag = "_".join(f"{k}{v}" for k, v in sorted(defines.items())).replace(".", "p").replace("-", "m")
    path = os.path.join(workdir, f"libia_oracle_{tag}.so")
    flags = [f"-D{k}={v!r}" if not isinstance(v, str) else f"-D{k}={v}" for k, v in defines.items()]
    subprocess.run(["gcc", *CFLAGS, *flags, "-o", path, *_SRCS, "-lm"], check=True)
    L = ctypes.CDLL(path)
    _trace_types(L)
    return L


def test_trace(kind: int, p: float, t_end: float, y0, rtol: float, atol: float, hmax: float, h0: float = 0.0,
               cap: int = 100000, L=None):
    """Every attempted step of an adaptive solve of a test problem: arrays t, h, err (the error measure)
    and accepted, plus the final y. L: a variant library from build_variant (default: the oracle)."""
    L = lib() if L is None else L
    y = np.array(y0, dtype=np.float64)
    t = np.zeros(cap)
    h = np.zeros(cap)
    e = np.zeros(cap)
    acc = np.zeros(cap, dtype=np.int32)
    m = L.orc_test_trace(kind, p, t_end, rtol, atol, hmax, h0, _dptr(y), cap, _dptr(t), _dptr(h), _dptr(e),
                         acc.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return {"t": t[:m], "h": h[:m], "err": e[:m], "acc": acc[:m].astype(bool), "y": y}


def test_dense(kind: int, p: float, h: float, s: float, y0):
    y = np.array(y0, dtype=np.float64)
    out = np.zeros_like(y)
    lib().orc_test_dense(kind, p, h, s, _dptr(y), _dptr(out))
    return out


def ionatom_fixed(desc: dict, phi0: float, t0: float, h: float, nsteps: int, y0) -> np.ndarray:
    s = make_system(desc)
    y = np.array(y0, dtype=np.float64)
    lib().orc_ionatom_fixed(ctypes.byref(s), phi0, t0, h, nsteps, _dptr(y))
    return y


def ionatom_segment(desc: dict, phi0: float, t0: float, t1: float, y0):
    s = make_system(desc)
    y = np.array(y0, dtype=np.float64)
    ns = ctypes.c_int64()
    nr = ctypes.c_int64()
    lib().orc_ionatom_segment(ctypes.byref(s), phi0, t0, t1, _dptr(y), ctypes.byref(ns), ctypes.byref(nr))
    return y, ns.value, nr.value


def trajectory_steps(desc: dict, y0, phi0: float, cap: int = 5_000_000):
    """Run one trajectory and return (result record, accepted step sizes, end mode)."""
    L = lib()
    s = make_system(desc)
    y = np.ascontiguousarray(y0, dtype=np.float64)
    hs = np.zeros(cap)
    res = np.zeros(1, dtype=RESULT_DTYPE)
    mode = ctypes.c_int32()
    L.orc_trajectory_steps.restype = ctypes.c_int64
    L.orc_trajectory_steps.argtypes = [ctypes.POINTER(OrcSystem), ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                                       ctypes.POINTER(OrcResult), ctypes.POINTER(ctypes.c_double), ctypes.c_int64,
                                       ctypes.POINTER(ctypes.c_int32)]
    n = L.orc_trajectory_steps(ctypes.byref(s), _dptr(y), phi0, res.ctypes.data_as(ctypes.POINTER(OrcResult)),
                               _dptr(hs), cap, ctypes.byref(mode))
    assert n <= cap
    return res[0], hs[:n].copy(), int(mode.value)


def replay(desc: dict, y0, phi0: float, hs, mode: int):
    """Fixed-step replay of an accepted step sequence; returns (observables[4], y_final[12])."""
    L = lib()
    s = make_system(desc)
    y = np.ascontiguousarray(y0, dtype=np.float64)
    hs = np.ascontiguousarray(hs, dtype=np.float64)
    obs = np.zeros(4)
    yf = np.zeros(12)
    L.orc_replay.argtypes = [ctypes.POINTER(OrcSystem), ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                             ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.c_int32,
                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.orc_replay(ctypes.byref(s), _dptr(y), phi0, _dptr(hs), len(hs), mode, _dptr(obs), _dptr(yf))
    return obs, yf


def tangent(desc: dict, y0, phi0: float, hs, mode: int, dy0, dq):
    """Discrete tangent along the frozen step sequence; dy0 (ndir, 12), dq (ndir, 3).
    Returns (out (ndir, 4): d theta_s, d dp, d dE_ion, d t_final; dy_final (ndir, 12))."""
    L = lib()
    s = make_system(desc)
    y = np.ascontiguousarray(y0, dtype=np.float64)
    hs = np.ascontiguousarray(hs, dtype=np.float64)
    dy0 = np.ascontiguousarray(dy0, dtype=np.float64)
    dq = np.ascontiguousarray(dq, dtype=np.float64)
    nd = dy0.shape[0]
    out = np.zeros((nd, 4))
    dyf = np.zeros((nd, 12))
    L.orc_tangent.argtypes = [ctypes.POINTER(OrcSystem), ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                              ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.c_int32,
                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), ctypes.c_int32,
                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.orc_tangent(ctypes.byref(s), _dptr(y), phi0, _dptr(hs), len(hs), mode, _dptr(dy0), _dptr(dq), nd,
                  _dptr(out), _dptr(dyf))
    return out, dyf


def fd_extended(desc: dict, y0, phi0: float, hs, mode: int, dy0, dq, delta: float):
    """Richardson-combined central differences of the extended-precision frozen-step replay along
    one direction (dy0 (12,), dq (3,)); returns d(theta_s, dp, dE_ion, t_final)."""
    L = lib()
    s = make_system(desc)
    y = np.ascontiguousarray(y0, dtype=np.float64)
    hs = np.ascontiguousarray(hs, dtype=np.float64)
    d1 = np.ascontiguousarray(dy0, dtype=np.float64)
    d2 = np.ascontiguousarray(dq, dtype=np.float64)
    out = np.zeros(4)
    L.orc_fd_ld.argtypes = [ctypes.POINTER(OrcSystem), ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                            ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.c_int32,
                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                            ctypes.POINTER(ctypes.c_double)]
    L.orc_fd_ld(ctypes.byref(s), _dptr(y), phi0, _dptr(hs), len(hs), mode, _dptr(d1), _dptr(d2), delta,
                _dptr(out))
    return out


def gradient(desc: dict, y0, phi0: float, hs, mode: int):
    """Gradient of (theta_s, dp, dE_ion, t_final) with respect to the initial state and the q vector,
    along the frozen step sequence: the transpose of the Jacobian, assembled column by column from the
    discrete tangent along the fifteen unit directions (twelve state components, three q components).
    Returns (g_y0 (4, 12), g_q (4, 3))."""
    dirs_y = np.vstack([np.eye(12), np.zeros((3, 12))])
    dirs_q = np.vstack([np.zeros((12, 3)), np.eye(3)])
    cols = []
    for k in range(0, 15, 4):
        out, _ = tangent(desc, y0, phi0, hs, mode, dirs_y[k:k + 4], dirs_q[k:k + 4])
        cols.append(out)
    J = np.vstack(cols)  # (15, 4): row = direction, column = objective
    return np.ascontiguousarray(J[:12].T), np.ascontiguousarray(J[12:].T)


def philox4x64(ctr, key) -> np.ndarray:
    """One Philox4x64-10 block of counter ctr (4 words) under key (2 words)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    P = ctypes.POINTER(ctypes.c_uint64)
    lib().orc_philox4x64(c.ctypes.data_as(P), k.ctypes.data_as(P), out.ctypes.data_as(P))
    return out


def philox4x64_stream(key0: int, key1: int, ctr1: int, first: int, n: int) -> np.ndarray:
    """n blocks, block j of counter (first + j, ctr1, 0, 0); returns (n, 4) uint64."""
    out = np.zeros((n, 4), dtype=np.uint64)
    lib().orc_philox4x64_stream(key0, key1, ctr1, first, n, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    return out


def make_sampler(kind: int, desc: dict, seed: int, E: float = 0.0, kT: float = 0.0, kT_ion: float = 0.0,
                 b_max: float = 0.0, random_phase: bool = True, phase: float = 0.0,
                 micromotion: bool = False) -> OrcSampler:
    """Sampler struct; the masses, Omega, q, r0 and rf sign come from a descriptor dict."""
    s = OrcSampler()
    s.kind = kind
    s.random_phase = int(bool(random_phase))
    s.micromotion = int(bool(micromotion))
    s.rf_sign = int(desc.get("rf_sign", 1))
    s.m_ion = desc["m_ion"]
    s.m_atom = desc["m_atom"]
    s.Omega = desc["Omega"]
    for j in range(3):
        s.q[j] = desc["q"][j]
    s.r0 = desc["r0"]
    s.E, s.kT, s.kT_ion, s.b_max, s.phase = E, kT, kT_ion, b_max, phase
    s.seed = seed
    return s


def sample_ics(sampler: OrcSampler, first: int, n: int):
    """Initial states of trajectories first .. first + n - 1: (y0 (n, 12), phi0 (n,))."""
    y = np.zeros((n, 12))
    ph = np.zeros(n)
    rc = lib().orc_sample_ics(ctypes.byref(sampler), first, n, _dptr(y), _dptr(ph))
    if rc != 0:
        raise ValueError("sampler parameters out of range")
    return y, ph
