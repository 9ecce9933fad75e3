"""Seeded, synthetic inputs: system descriptors and initial conditions.

This module serves both the CUDA path and the CPU oracle. It holds no arithmetic of the method itself
(no equations of motion, integrator, events or observables). It only builds the workloads: species
constants, trap and tolerance settings, and initial conditions drawn as the paper describes them.

Units are atomic units: lengths in a0, energies in hartree, masses in m_e, times in a.u. of time.

Initial-condition families (arXiv 2509.15117):
  - head-on runs: the ion at rest at the trap centre, the atom on the sphere of radius r0 with speed
    v0 = sqrt(2E/m_a) pointing at the centre; r0 satisfies 10|V(r0)| < E (head-on paragraph, Fig. 1
    caption: the octant of the sphere);
  - thermal runs: the ion Gaussian at T_ion = 10 uK in an isotropic harmonic trap of frequency
    omega = q_x Omega / 2^(3/2); atom velocity components Gaussian at T; atom position uniform on the
    r0 sphere; the velocity negated if it points outward (thermal paragraph, Fig. 3 caption);
  - the disk variant of the thermal runs: the impact parameter uniform over a disk of radius b_max
    perpendicular to the atom velocity, with the ion's lowest-order micromotion added;
  - random rf phase Omega t0 mod 2 pi uniform on [0, 2 pi) (Fig. 4 caption).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# CODATA-based conversions
K_TO_HARTREE = 3.166811563e-6      # k_B * 1 K in E_h
AMU_TO_ME = 1822.888486            # 1 u in m_e
AU_TIME_S = 2.4188843265857e-17    # 1 a.u. of time in s

# Masses (integer mass numbers) and static dipole polarisabilities (a.u.). The paper names the atoms
# and gives alpha = 319 a.u. only for Rb (through C4 = alpha/2). The other polarisabilities are the
# commonly tabulated ground-state values (Schwerdtfeger & Nagle, Mol. Phys. 117, 1200 (2019)).
SPECIES = {
    "Li": {"mass_amu": 6.0, "alpha": 164.1},
    "Na": {"mass_amu": 23.0, "alpha": 162.7},
    "K": {"mass_amu": 39.0, "alpha": 290.6},
    "Rb": {"mass_amu": 87.0, "alpha": 319.0},
    "Cs": {"mass_amu": 133.0, "alpha": 401.0},
}
ION_MASS_AMU = 174.0  # 174Yb+

RF_HZ = 2.0e6


def omega_rf(freq_hz: float = RF_HZ) -> float:
    """rf angular frequency in rad per a.u. of time."""
    return 2.0 * math.pi * freq_hz * AU_TIME_S


def kelvin(x: float) -> float:
    return x * K_TO_HARTREE


def speed_for_energy(E: float, m: float) -> float:
    """v0 with E = m v0^2 / 2."""
    return math.sqrt(2.0 * E / m)


def r0_rule(alpha: float, E: float, r_min: float = 5000.0) -> float:
    """Smallest round r0 >= r_min with 10 |C4 / r0^4| < E (head-on paragraph of the paper).

    The attractive tail C4/r^4 dominates |V| at r0, so the rule is r0 > (10 C4 / E)^(1/4); a 1% margin
    is added and the result rounded up to a whole a0."""
    C4 = 0.5 * alpha
    need = (10.0 * C4 / E) ** 0.25
    return float(max(r_min, math.ceil(1.01 * need)))


@dataclasses.dataclass
class SystemDesc:
    """One physical system plus its integration settings (the fields of both C structs)."""
    m_ion: float
    m_atom: float
    alpha: float
    De: float
    Omega: float
    a: tuple
    q: tuple
    r0: float
    t_max: float
    rtol: float = 1e-10
    atol_pos: float = 1e-10
    atol_vel: float = 1e-19
    h_max: float = 0.0
    rf_sign: int = 1
    max_attempts: int = 50_000_000

    def as_dict(self) -> dict:
        d = dataclasses.asdict(self)
        d["a"] = tuple(float(x) for x in self.a)
        d["q"] = tuple(float(x) for x in self.q)
        return d


def linear_trap(q: float, a: float = 0.0):
    """Per-axis Mathieu parameters of a linear Paul trap with q_x = -q_y (Fig. 1 discussion):
    q = (q, -q, 0) and a static part a = (a, a, -2a) that satisfies Laplace's equation."""
    return (a, a, -2.0 * a), (q, -q, 0.0)


def make_system(species: str = "Rb", De_K: float = 1.0, q: float = 0.1, a: float = 0.0,
                r0: float = 5000.0, t_max_s: float = 1e-3, v_scale: float | None = None,
                E_K: float | None = None, rtol: float = 1e-10, freq_hz: float = RF_HZ,
                rf_sign: int = 1, alpha: float | None = None, ion_mass_amu: float = ION_MASS_AMU,
                max_attempts: int = 50_000_000) -> SystemDesc:
    """Descriptor of Yb+ + atom in a linear Paul trap.

    The velocity tolerance is atol_vel = 1e-10 * v_scale, where v_scale is the head-on speed for E_K
    (or an explicit thermal speed); positions use atol_pos = 1e-10 a0. h_max is a sixteenth of the
    rf period, so no step can jump over an rf cycle while the ion sits at the trap centre.
    """
    sp = SPECIES[species]
    m_a = sp["mass_amu"] * AMU_TO_ME
    m_i = ion_mass_amu * AMU_TO_ME
    Om = omega_rf(freq_hz)
    a_vec, q_vec = linear_trap(q, a)
    if v_scale is None:
        if E_K is None:
            E_K = 1.5e-6
        v_scale = speed_for_energy(kelvin(E_K), m_a)
    return SystemDesc(
        m_ion=m_i, m_atom=m_a, alpha=sp["alpha"] if alpha is None else alpha, De=kelvin(De_K),
        Omega=Om, a=a_vec, q=q_vec, r0=float(r0), t_max=t_max_s / AU_TIME_S, rtol=rtol,
        atol_pos=1e-10, atol_vel=1e-10 * v_scale, h_max=(2.0 * math.pi / Om) / 16.0,
        rf_sign=rf_sign, max_attempts=max_attempts)


# --------------------------------------------------------------------------------------------
# Initial conditions. y0 rows are [x_ion(3), v_ion(3), x_atom(3), v_atom(3)].

def octant_grid(n_theta: int, n_phi: int | None = None):
    """Cell-centred (theta, phi) grid over the octant: theta_k = (k + 1/2)(pi/2)/N, same for phi.
    Returned flattened with phi fastest."""
    n_phi = n_theta if n_phi is None else n_phi
    th = (np.arange(n_theta) + 0.5) * (0.5 * math.pi / n_theta)
    ph = (np.arange(n_phi) + 0.5) * (0.5 * math.pi / n_phi)
    T, P = np.meshgrid(th, ph, indexing="ij")
    return T.ravel(), P.ravel()


def octant_random(n: int, seed: int):
    """(theta, phi) uniform on the octant's surface: cos(theta) ~ U[0,1], phi ~ U[0, pi/2)."""
    rng = np.random.default_rng(seed)
    cth = rng.random(n)
    ph = rng.random(n) * (0.5 * math.pi)
    return np.arccos(cth), ph


def head_on(theta, phi, r0: float, v0: float) -> np.ndarray:
    """Head-on initial state: ion at rest at the centre; atom at r0 (sin t cos p, sin t sin p, cos t)
    moving at speed v0 toward the centre."""
    theta = np.asarray(theta, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    n = theta.shape[0]
    u = np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)], axis=1)
    y = np.zeros((n, 12))
    y[:, 6:9] = r0 * u
    y[:, 9:12] = -v0 * u
    return y


def head_on_seeds(theta, phi, r0: float, v0: float, E: float) -> np.ndarray:
    """Derivatives of the head-on initial state with respect to (theta, phi, E): shape (n, 3, 12).
    x_a = r0 u(theta, phi), v_a = -v0 u with v0 = sqrt(2E/m), so dv0/dE = v0/(2E); E in hartree."""
    theta = np.asarray(theta, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    n = theta.shape[0]
    u = np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)], axis=1)
    ut = np.stack([np.cos(theta) * np.cos(phi), np.cos(theta) * np.sin(phi), -np.sin(theta)], axis=1)
    up = np.stack([-np.sin(theta) * np.sin(phi), np.sin(theta) * np.cos(phi), np.zeros(n)], axis=1)
    d = np.zeros((n, 3, 12))
    d[:, 0, 6:9] = r0 * ut
    d[:, 0, 9:12] = -v0 * ut
    d[:, 1, 6:9] = r0 * up
    d[:, 1, 9:12] = -v0 * up
    d[:, 2, 9:12] = -(v0 / (2.0 * E)) * u
    return d


def q_direction():
    """d q_vector / d q of the linear trap q = (q, -q, 0)."""
    return np.array([1.0, -1.0, 0.0])


def random_phase(n: int, seed: int) -> np.ndarray:
    """rf phase Omega t0 mod 2 pi, uniform on [0, 2 pi)."""
    return np.random.default_rng(seed).random(n) * (2.0 * math.pi)


def secular_omega(q: float, Omega: float) -> float:
    """Isotropic secular frequency used for the thermal ion: omega = q_x Omega / 2^(3/2)."""
    return q * Omega / 2.0 ** 1.5


def thermal_ion(n: int, rng, m_ion: float, T_ion_K: float, q_vec, Omega: float, phi0,
                rf_sign: int = 1, micromotion: bool = True) -> np.ndarray:
    """Ion position and velocity: secular X ~ N(0, kT/(m omega^2)), V ~ N(0, kT/m) per axis, with
    omega = q_x Omega / 2^(3/2); optionally the lowest-order micromotion of the Mathieu solution
    x = X (1 + s (q_j/2) cos(phi0)), v = V (1 + s (q_j/2) cos(phi0)) - X s (q_j Omega / 2) sin(phi0)."""
    kT = kelvin(T_ion_K)
    w = secular_omega(abs(q_vec[0]), Omega)
    X = rng.normal(0.0, math.sqrt(kT / (m_ion * w * w)), size=(n, 3))
    V = rng.normal(0.0, math.sqrt(kT / m_ion), size=(n, 3))
    if not micromotion:
        return np.concatenate([X, V], axis=1)
    qv = np.asarray(q_vec, dtype=np.float64)[None, :]
    c = np.cos(phi0)[:, None]
    s = np.sin(phi0)[:, None]
    x = X * (1.0 + rf_sign * 0.5 * qv * c)
    v = V * (1.0 + rf_sign * 0.5 * qv * c) - X * rf_sign * 0.5 * qv * Omega * s
    return np.concatenate([x, v], axis=1)


def thermal_sphere(n: int, seed: int, sysd: SystemDesc, T_K: float, T_ion_K: float = 10e-6):
    """The paper's thermal runs: atom uniform on the r0 sphere, velocity components Gaussian at T,
    negated where v_r >= 0; ion thermal at T_ion; random rf phase. Returns (y0, phi0)."""
    rng = np.random.default_rng(seed)
    phi0 = rng.random(n) * (2.0 * math.pi)
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    v = rng.normal(0.0, math.sqrt(kelvin(T_K) / sysd.m_atom), size=(n, 3))
    outward = np.sum(v * u, axis=1) >= 0.0
    v[outward] *= -1.0
    y = np.zeros((n, 12))
    y[:, 0:6] = thermal_ion(n, rng, sysd.m_ion, T_ion_K, sysd.q, sysd.Omega, phi0, sysd.rf_sign,
                            micromotion=False)
    y[:, 6:9] = sysd.r0 * u
    y[:, 9:12] = v
    return y, phi0


def _perp_basis(vhat):
    """Two unit vectors perpendicular to each row of vhat."""
    ref = np.where(np.abs(vhat[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    e1 = np.cross(vhat, ref)
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(vhat, e1)
    return e1, e2


def thermal_disk(n: int, seed: int, sysd: SystemDesc, T_K: float, b_max: float = 2000.0,
                 T_ion_K: float = 10e-6):
    """Thermal bath with the impact parameter uniform over a disk of radius b_max: v Maxwell-Boltzmann
    at T; b = b_max sqrt(u) at a uniform azimuth in the plane perpendicular to v; the atom starts at
    x_a = b - sqrt(r0^2 - b^2) v_hat; ion thermal at T_ion with micromotion; rf phase uniform.
    Returns (y0, phi0)."""
    rng = np.random.default_rng(seed)
    phi0 = rng.random(n) * (2.0 * math.pi)
    v = rng.normal(0.0, math.sqrt(kelvin(T_K) / sysd.m_atom), size=(n, 3))
    vhat = v / np.linalg.norm(v, axis=1, keepdims=True)
    e1, e2 = _perp_basis(vhat)
    b = b_max * np.sqrt(rng.random(n))
    psi = rng.random(n) * (2.0 * math.pi)
    bvec = b[:, None] * (np.cos(psi)[:, None] * e1 + np.sin(psi)[:, None] * e2)
    xa = bvec - np.sqrt(sysd.r0 ** 2 - b ** 2)[:, None] * vhat
    y = np.zeros((n, 12))
    y[:, 0:6] = thermal_ion(n, rng, sysd.m_ion, T_ion_K, sysd.q, sysd.Omega, phi0, sysd.rf_sign)
    y[:, 6:9] = xa
    y[:, 9:12] = v
    return y, phi0


# --------------------------------------------------------------------------------------------
# Workloads shaped like the paper's runs

C2_SPECIES = ("Li", "Na", "K", "Rb", "Cs")
C2_ENERGIES_K = tuple(1e-6 * 1000.0 ** (k / 7.0) for k in range(8))  # 1 uK .. 1 mK, log-spaced


def c1_workload(n_grid: int = 32):
    """Yb+-Rb head-on, D_e = 1 K, E = 1.5 uK, r0 = 5000 a0, q = 0.1, a = 0, t_max = 1 ms,
    cell-centred n_grid x n_grid octant grid, rf phase 0 (Fig. 1 setup)."""
    sysd = make_system("Rb", De_K=1.0, q=0.1, a=0.0, r0=5000.0, t_max_s=1e-3, E_K=1.5e-6)
    th, ph = octant_grid(n_grid)
    v0 = speed_for_energy(kelvin(1.5e-6), sysd.m_atom)
    y0 = head_on(th, ph, sysd.r0, v0)
    return [sysd], y0, np.zeros(len(th)), np.zeros(len(th), dtype=np.int32)


def c2_systems(t_max_s: float = 1e-3):
    """The 40 (species, energy) systems of the head-on species x energy sweep (D_e = 1 K, q = 0.1)."""
    out = []
    for sp in C2_SPECIES:
        for E_K in C2_ENERGIES_K:
            r0 = r0_rule(SPECIES[sp]["alpha"], kelvin(E_K))
            out.append((sp, E_K, make_system(sp, De_K=1.0, q=0.1, a=0.0, r0=r0, t_max_s=t_max_s, E_K=E_K)))
    return out


def c2_workload(n_grid: int = 1024, stride: int = 1, offset: int = 0, t_max_s: float = 1e-3):
    """Head-on sweep over 5 species x 8 energies on an n_grid^2 octant grid each; every
    `stride`-th grid point in each direction starting at `offset` (stride 1 = the full grid).
    Trajectories are ordered system by system. Returns (systems, y0, phi0, sys_id)."""
    systems = c2_systems(t_max_s)
    th, ph = octant_grid(n_grid)
    idx = np.arange(n_grid * n_grid).reshape(n_grid, n_grid)[offset::stride, offset::stride].ravel()
    th, ph = th[idx], ph[idx]
    ys, sids = [], []
    for k, (sp, E_K, sysd) in enumerate(systems):
        v0 = speed_for_energy(kelvin(E_K), sysd.m_atom)
        ys.append(head_on(th, ph, sysd.r0, v0))
        sids.append(np.full(len(th), k, dtype=np.int32))
    y0 = np.concatenate(ys)
    return [s for (_, _, s) in systems], y0, np.zeros(len(y0)), np.concatenate(sids)


def c3_workload(n_per_T: int, seed_base: int = 3001, temps_K=(10e-6, 100e-6, 1e-3)):
    """Monte Carlo bath (disk sampler), Yb+-Rb, one system per temperature."""
    systems, ys, ps, sids = [], [], [], []
    for k, T in enumerate(temps_K):
        vth = math.sqrt(kelvin(T) / (SPECIES["Rb"]["mass_amu"] * AMU_TO_ME))
        sysd = make_system("Rb", De_K=1.0, q=0.1, a=0.0, r0=5000.0, t_max_s=1e-3, v_scale=vth)
        y, p = thermal_disk(n_per_T, seed_base + k, sysd, T)
        systems.append(sysd)
        ys.append(y)
        ps.append(p)
        sids.append(np.full(n_per_T, k, dtype=np.int32))
    return systems, np.concatenate(ys), np.concatenate(ps), np.concatenate(sids)


def splitmix64(x: int) -> int:
    """splitmix64 finaliser (Steele, Lea & Flood 2014)."""
    x = (x + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
    x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    return x ^ (x >> 31)


def c4_cells():
    """250 cells: D_e x q x a x species, each with N_cell = 4096 * 2^(splitmix64(cell ^ seed) mod 7)."""
    cells = []
    k = 0
    for De in (0.1, 0.3, 1.0, 3.0, 10.0):
        for q in (0.05, 0.1, 0.2, 0.3, 0.4):
            for a in (0.0, -0.001):
                for sp in C2_SPECIES:
                    n_cell = 4096 * 2 ** (splitmix64(k ^ 4) % 7)
                    cells.append({"De_K": De, "q": q, "a": a, "species": sp, "n": n_cell})
                    k += 1
    return cells


def c4_workload(scale: float = 1.0, seed: int = 4, t_max_s: float = 1e-3):
    """Mixed-parameter sweep: each cell is its own system; head-on with (theta, phi) uniform on the
    octant surface, random rf phase, E = 1.5 uK. `scale` shrinks every cell (>= 1 trajectory)."""
    systems, ys, ps, sids = [], [], [], []
    E_K = 1.5e-6
    for k, c in enumerate(c4_cells()):
        sysd = make_system(c["species"], De_K=c["De_K"], q=c["q"], a=c["a"], r0=5000.0,
                           t_max_s=t_max_s, E_K=E_K)
        sysd.r0 = r0_rule(sysd.alpha, kelvin(E_K))
        n = max(1, int(round(c["n"] * scale)))
        th, ph = octant_random(n, seed * 1_000_003 + k)
        v0 = speed_for_energy(kelvin(E_K), sysd.m_atom)
        ys.append(head_on(th, ph, sysd.r0, v0))
        ps.append(random_phase(n, seed * 2_000_003 + k))
        sids.append(np.full(n, k, dtype=np.int32))
        systems.append(sysd)
    return systems, np.concatenate(ys), np.concatenate(ps), np.concatenate(sids)


def c5_workload(n: int = 1_000_000, seed: int = 5, t_max_s: float = 1e-3):
    """Differentiation workload: Yb+-Rb head-on at E = 1.5 uK (D_e = 1 K, q = 0.1, a = 0, r0 = 5000 a0),
    (theta, phi) uniform on the octant surface, rf phase 0. Returns (system, y0, phi0, seeds, dq) with
    seeds (n, 3, 12) = d y0 / d(theta, phi, E) and dq (4, 3): zero for those three, the q direction of
    the linear trap for the fourth seed (whose d y0 is zero)."""
    E_K = 1.5e-6
    sysd = make_system("Rb", De_K=1.0, q=0.1, a=0.0, r0=5000.0, t_max_s=t_max_s, E_K=E_K)
    th, ph = octant_random(n, seed)
    v0 = speed_for_energy(kelvin(E_K), sysd.m_atom)
    y0 = head_on(th, ph, sysd.r0, v0)
    seeds = head_on_seeds(th, ph, sysd.r0, v0, kelvin(E_K))
    dq = np.zeros((4, 3))
    dq[3] = q_direction()
    return sysd, y0, np.zeros(n), seeds, dq


def c5_ftle_grid(n_grid: int = 2048, t_max_s: float = 1e-3):
    """FTLE map of the differentiation workload: cell-centred n_grid x n_grid (theta, phi) octant grid
    with the theta seed as the tangent direction. Returns (system, y0, phi0, dy0 (n, 1, 12))."""
    E_K = 1.5e-6
    sysd = make_system("Rb", De_K=1.0, q=0.1, a=0.0, r0=5000.0, t_max_s=t_max_s, E_K=E_K)
    th, ph = octant_grid(n_grid)
    v0 = speed_for_energy(kelvin(E_K), sysd.m_atom)
    y0 = head_on(th, ph, sysd.r0, v0)
    seeds = head_on_seeds(th, ph, sysd.r0, v0, kelvin(E_K))[:, :1, :]
    return sysd, y0, np.zeros(len(th)), seeds


def energy_scan_systems(species=C2_SPECIES, n_energies: int = 100, E_min_K: float = 3e-8, E_max_K: float = 1e-3,
                        r0: float = 20000.0, t_max_s: float = 3e-3, q: float = 0.1):
    """Cells of the collision-energy scan of Fig. 4: head-on Yb+ collisions, r0 = 20,000 a0, D_e = 1 K,
    a random rf phase per trajectory, n_energies fixed collision energies log-spaced over
    [E_min_K, E_max_K] (k_B units) for each species. One system per (species, energy) cell, with the
    velocity tolerance scaled by that cell's head-on speed. Returns (systems, energies in hartree,
    species per cell). The paper's energy axis and the longest lifetime are not given; 30 nK .. 1 mK
    brackets every species' threshold (a few W0^3D), and t_max = 3 ms lets the slowest atoms (Cs at
    30 nK needs about 0.55 ms to reach the ion from 20,000 a0) collide, form complexes and leave."""
    systems, energies, names = [], [], []
    for sp in species:
        for E_K in np.geomspace(E_min_K, E_max_K, n_energies):
            systems.append(make_system(sp, De_K=1.0, q=q, a=0.0, r0=r0, t_max_s=t_max_s, E_K=float(E_K)))
            energies.append(kelvin(float(E_K)))
            names.append(sp)
    return systems, np.array(energies), names


FIG3_TEMPS_K = (10e-6, 100e-6, 1e-3)
FIG3_DEPTHS_K = (1.0, 100.0)


def thermal_sweep_systems(species=C2_SPECIES, temps_K=FIG3_TEMPS_K, depths_K=FIG3_DEPTHS_K, t_max_s: float = 1e-3):
    """Cells of the thermal runs of Fig. 3: Yb+ with each species, bath temperature T and well depth
    D_e (1 K and 100 K, the caption's two depths), r0 = 5000 a0, q = 0.1. The caption gives no
    temperatures; 10 uK, 100 uK and 1 mK span the range the text discusses. One system per cell, with
    the velocity tolerance scaled by that cell's thermal speed sqrt(k_B T / m_a). Returns (systems,
    cells as (species, T_K, De_K))."""
    systems, cells = [], []
    for sp in species:
        m_a = SPECIES[sp]["mass_amu"] * AMU_TO_ME
        for T in temps_K:
            for De in depths_K:
                vth = math.sqrt(kelvin(T) / m_a)
                systems.append(make_system(sp, De_K=De, q=0.1, a=0.0, r0=5000.0, t_max_s=t_max_s, v_scale=vth))
                cells.append((sp, T, De))
    return systems, cells
