"""The C-ABI library builds for sm_103a, loads, and exports every function include/ionatom.h declares.
No compute call is made here (no GPU on the build machine)."""
import ctypes

import numpy as np
import os
import re

import pytest

from paper_2509_15117_gb300 import binding as Bd
from paper_2509_15117_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**\s*(ia_[a-z0-9_]+)\s*\(",
                            text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ia_system_create", "ia_system_destroy", "ia_launch", "ia_error_string"):
        assert required in names


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    for name in Bd.EXPORTED:
        assert hasattr(lib, name), name


def test_error_strings_and_version_without_gpu():
    L = Bd.load()
    assert L.ia_version() >= 100
    for code in (0, -1, -2, -3, -4, -5, -6, -99):
        assert L.ia_error_string(code)


def test_struct_layouts_match_header():
    # sizes of the C structs as the header defines them (x86-64 / aarch64 LP64)
    assert ctypes.sizeof(Bd.ia_system_desc) == 8 * 17 + 4 * 2 + 8
    assert ctypes.sizeof(Bd.ia_ic_soa) == 8 * 5
    assert ctypes.sizeof(Bd.ia_obs_soa) == 8 * 12
    assert ctypes.sizeof(Bd.ia_launch_opts) == 4 * 12 + 8 * 3


def test_invalid_arguments_rejected_without_touching_gpu():
    L = Bd.load()
    # NULL handle / arguments are rejected before any CUDA call
    assert L.ia_launch(None, None, 0, None, None, None) == -1
    assert L.ia_system_create(None, 1, None) == -1
    assert L.ia_system_count(None) == -1
    assert L.ia_system_destroy(None) == 0
    assert L.ia_queue_create(None, 10, None, None) == -1
    assert L.ia_queue_launch(None, None, None, 0, None) == -1
    assert L.ia_queue_reset(None) == -1
    assert L.ia_queue_state(None, None, None, None) == -1
    assert L.ia_queue_phases(None, None, None, None) == -1
    assert L.ia_queue_destroy(None) == 0
    assert L.ia_static_phases(None, None, None, None) == -1
    # scratch sizing is pure host arithmetic
    head = 1024
    assert Bd.ia_scratch_bytes(0) == head
    assert Bd.ia_scratch_bytes(100000, kernel=Bd.IA_KERNEL_PERSISTENT) == head + 4 * 4096 + 256 * 4096
    assert Bd.ia_scratch_bytes(1 << 20, kernel=Bd.IA_KERNEL_PERSISTENT) == head + 4 * (1 << 15) + 256 * (1 << 15)
    assert Bd.ia_scratch_bytes(1000, kernel=Bd.IA_KERNEL_PERSISTENT, slice_budget=-1) == head
    assert Bd.ia_scratch_bytes(1000, kernel=Bd.IA_KERNEL_PERSISTENT, suspend_capacity=5) == head + 256 + 5 * 256
    with pytest.raises(Bd.IaError):
        Bd.ia_scratch_bytes(10, kernel=Bd.IA_KERNEL_PERSISTENT, tail_group=5)


def test_stats_layout_and_host_statistics():
    from paper_2509_15117_gb300 import statistics as St
    assert Bd.STATS_DTYPE.itemsize == 8 * (3 + 8 + 32 + 64) + 16
    rec = np.zeros(1, dtype=Bd.STATS_DTYPE)[0]
    rec["n"] = 1000
    rec["n_complex"] = 430
    rec["sum_dE"] = 2.0
    rec["sum_dE2"] = 0.01
    rec["lifetime_hist"][10] = 300
    rec["lifetime_hist"][20] = 130
    s = St.summarize(rec)
    p, lo, hi = s["P_complex"], *s["P_complex_3sigma"]
    assert p == 0.43 and lo < p < hi
    # Wilson interval against its closed form at z = 3
    z, n = 3.0, 1000
    half = z * np.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / (1 + z * z / n)
    assert hi - lo == pytest.approx(2 * half, rel=1e-12)
    assert s["mean_dE_ion"] == pytest.approx(0.002)
    assert s["survival"][0] == 1.0 and s["survival"][11] == pytest.approx(130 / 430)
    assert s["survival"][21] == 0.0


def test_adjoint_structs_and_scratch_arithmetic_without_gpu():
    assert ctypes.sizeof(Bd.ia_adjoint_opts) == 4 * 2 + 8 * 3
    assert ctypes.sizeof(Bd.ia_adjoint_out) == 8 * 7
    # 256 B of counters + per warp: max_ckpt checkpoints of 256 B and seg step records of 128 B
    assert Bd.ia_adjoint_scratch_bytes(None, 1000, warps=10) == 256 + 10 * (64 * 256 + 10000 * 128)
    assert Bd.ia_adjoint_scratch_bytes(None, 3, warps=10, seg=16, max_ckpt=4) == 256 + 3 * (4 * 256 + 16 * 128)
    for bad in (dict(warps=4, max_ckpt=3), dict(warps=4, seg=8), dict(warps=4, max_ckpt=-2), dict(warps=-1)):
        with pytest.raises(Bd.IaError):
            Bd.ia_adjoint_scratch_bytes(None, 10, **bad)
    # default warps need the device's occupancy, hence a system
    with pytest.raises(Bd.IaError):
        Bd.ia_adjoint_scratch_bytes(None, 10)


def test_sampler_struct_and_argument_checks_without_gpu():
    assert ctypes.sizeof(Bd.ia_sampler) == 4 * 4 + 8 * 12 + 8
    L = Bd.load()
    from paper_2509_15117_gb300 import inputs as I
    d = I.make_system("Rb").as_dict()
    good = Bd.make_sampler(Bd.IA_SAMPLE_DISK, d, seed=1, kT=1e-9, kT_ion=1e-11, b_max=2000.0)
    buf = (ctypes.c_double * 16)()
    y, ph = ctypes.addressof(buf), ctypes.addressof(buf) + 8 * 12
    # n = 0 is a no-op; every rejection below happens before any CUDA call
    assert L.ia_sample_ics(ctypes.byref(good), 0, 0, None, None, 0, None) == 0
    assert L.ia_sample_ics(None, 0, 1, y, ph, 1, None) == -1
    assert L.ia_sample_ics(ctypes.byref(good), 0, -1, y, ph, 1, None) == -1
    assert L.ia_sample_ics(ctypes.byref(good), -5, 1, y, ph, 1, None) == -1
    assert L.ia_sample_ics(ctypes.byref(good), 2 ** 63 - 1, 2, y, ph, 2, None) == -1
    assert L.ia_sample_ics(ctypes.byref(good), 0, 2, y, ph, 1, None) == -1          # ld < n
    assert L.ia_sample_ics(ctypes.byref(good), 0, 1, y + 4, ph, 1, None) == -4      # unaligned
    bad = [
        Bd.make_sampler(7, d, seed=1, kT=1e-9),
        Bd.make_sampler(Bd.IA_SAMPLE_HEAD_ON, d, seed=1, E=0.0),
        Bd.make_sampler(Bd.IA_SAMPLE_SPHERE, d, seed=1, kT=-1.0),
        Bd.make_sampler(Bd.IA_SAMPLE_SPHERE, d, seed=1, kT=1e-9, kT_ion=-1e-12),
        Bd.make_sampler(Bd.IA_SAMPLE_DISK, d, seed=1, kT=1e-9, b_max=d["r0"]),
        Bd.make_sampler(Bd.IA_SAMPLE_HEAD_ON, d, seed=1, E=1e-9, random_phase=False, phase=float("nan")),
        Bd.make_sampler(Bd.IA_SAMPLE_SPHERE, dict(d, q=(0.0, 0.0, 0.0)), seed=1, kT=1e-9, kT_ion=1e-12),
    ]
    for s in bad:
        assert L.ia_sample_ics(ctypes.byref(s), 0, 1, y, ph, 1, None) == -1
    s = Bd.make_sampler(Bd.IA_SAMPLE_SPHERE, d, seed=1, kT=1e-9)
    s.rf_sign = 0
    assert L.ia_sample_ics(ctypes.byref(s), 0, 1, y, ph, 1, None) == -1
    # raw generator
    assert L.ia_philox4x64(1, 2, 3, 0, 0, None, None) == 0
    assert L.ia_philox4x64(1, 2, 3, 0, 1, None, None) == -1
    assert L.ia_philox4x64(1, 2, 3, -1, 1, y, None) == -1
    assert L.ia_philox4x64(1, 2, 3, 0, 1, y + 4, None) == -4


def test_tangent_entry_checks_alignment_and_reserved_without_gpu():
    """ia_launch_tangent refuses misaligned pointers and a non-zero reserved field before touching the
    system (a stand-in address that is never dereferenced on these paths)."""
    L = Bd.load()
    fake_sys = ctypes.c_void_p(0x2000)
    n = 4
    ic = Bd.ia_ic_soa(y0=0x10000, phi0=0x20000, sys_id=None, order=None, ld=n)
    out = Bd.ia_obs_soa(*([0x30000 + 0x1000 * k for k in range(10)] + [None, 0]))
    tin = Bd.ia_tangent_in(dy0=0x40000, ndir=1, reserved=0, ld=n)
    tout = Bd.ia_tangent_out(d_theta_s=0x50000, d_dp=0x51000, d_dE_ion=0x52000, d_t_final=0x53000,
                             dy_final=None, ftle=None, ld=n)
    call = lambda: L.ia_launch_tangent(fake_sys, ctypes.byref(ic), n, ctypes.byref(out), ctypes.byref(tin),
                                       ctypes.byref(tout), None)
    ic.y0 = 0x10004
    assert call() == -4
    ic.y0 = 0x10000
    out.dp = 0x31004
    assert call() == -4
    out.dp = 0x31000
    tin.reserved = 1
    assert call() == -1
    tin.reserved, tin.ndir = 0, 5
    assert call() == -1


def test_autotune_and_rcp_hook_check_alignment_without_gpu():
    L = Bd.load()
    fake_sys = ctypes.c_void_p(0x2000)
    ic = Bd.ia_ic_soa(y0=0x10004, phi0=0x20000, sys_id=None, order=None, ld=8)
    best = Bd.ia_launch_opts()
    ms = ctypes.c_double()
    assert L.ia_autotune(fake_sys, ctypes.byref(ic), 8, 1024, None, ctypes.byref(best), ctypes.byref(ms), None) == -4
    ic.y0, ic.order = 0x10000, 0x30004
    assert L.ia_autotune(fake_sys, ctypes.byref(ic), 8, 1024, None, ctypes.byref(best), ctypes.byref(ms), None) == -4
    assert L.ia_autotune(fake_sys, ctypes.byref(ic), 8, 32, None, ctypes.byref(best), ctypes.byref(ms), None) == -1
    assert L.ia_rcp_check(ctypes.c_void_p(0x10004), ctypes.c_void_p(0x20000), 4, None) == -4
