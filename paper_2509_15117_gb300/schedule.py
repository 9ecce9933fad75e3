"""Host-side scheduling helpers for persistent launches (queue order).

The persistent kernel takes trajectories from its work queue in the order given by `ia_ic_soa.order`.
Trajectory lengths are heavy-tailed (long-lived complexes run 10^2-10^3 times longer than single
passes), and a batch ends when its longest trajectory ends; starting the trajectories most likely to
be long first lets them overlap the bulk of the batch. Slow, heavy atoms form complexes most often and
stay longest (the paper's Fig. 3 and Fig. 4 trends: probability of complex formation rises with atom
mass and falls with collision energy), so the expected cost of a system grows with m_a and with
1/speed.
"""
from __future__ import annotations

import numpy as np


def system_cost(systems, speeds) -> np.ndarray:
    """Expected relative cost per system: sqrt(m_atom) / speed (slow and heavy first)."""
    m = np.array([s["m_atom"] if isinstance(s, dict) else s.m_atom for s in systems], dtype=np.float64)
    v = np.asarray(speeds, dtype=np.float64)
    return np.sqrt(m) / v


def system_cost_threshold(energies, w0) -> np.ndarray:
    """Relative cost per system from the complex-formation threshold: W0^3D / E, so that the systems
    whose collision energy lies furthest below the heating energy scale W0^3D (where the complex
    probability is highest, Fig. 4) come first. Energies and W0 in the same units."""
    return np.asarray(w0, dtype=np.float64) / np.asarray(energies, dtype=np.float64)


def order_by_cost(sys_id, cost) -> np.ndarray:
    """Permutation of 0..n-1 that visits trajectories of costlier systems first (stable within a system)."""
    sys_id = np.asarray(sys_id)
    key = -np.asarray(cost, dtype=np.float64)[sys_id]
    return np.argsort(key, kind="stable").astype(np.int64)
