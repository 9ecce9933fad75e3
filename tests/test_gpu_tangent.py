"""Tangent (forward-mode) kernel against the oracle's discrete tangent and against quad-precision
finite differences of the frozen-step replay (needs a GB300)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_15117_gb300 import binding as Bd
from paper_2509_15117_gb300 import inputs as I
from tests import test_oracle_tangent as OT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Bd.load()
    return torch


def gpu_tangent(torch, descs, y0, phi0, sid, dy0, dq, dy_final=False):
    n = len(phi0)
    with Bd.System(descs) as S:
        yd, pd, sd = Bd.to_device_soa(y0, phi0, sid)
        out = Bd.alloc_obs(n, y_final=True)
        tan = Bd.alloc_tangent(n, dy0.shape[1], dy_final=dy_final)
        dyd = torch.from_numpy(np.ascontiguousarray(np.transpose(dy0, (1, 2, 0)))).cuda()
        Bd.ia_launch_tangent(S.handle, yd, pd, sd, out, dyd, dq, tan)
        torch.cuda.synchronize()
        res = {k: v.cpu().numpy() for k, v in tan.items()}
        return Bd.to_numpy(out), res


def test_tangent_primal_is_bitwise_the_launch(cuda):
    torch = cuda
    systems, y0, phi0, sid = I.c1_workload(16)
    descs = [s.as_dict() for s in systems]
    d = descs[0]
    v0 = I.speed_for_energy(I.kelvin(1.5e-6), d["m_atom"])
    th, ph = I.octant_grid(16)
    seeds = I.head_on_seeds(th, ph, d["r0"], v0, I.kelvin(1.5e-6))
    dy0 = np.concatenate([seeds, np.zeros((len(th), 1, 12))], axis=1)
    dq = np.zeros((4, 3))
    dq[3] = I.q_direction()
    g, tan = gpu_tangent(torch, descs, y0, phi0, sid, dy0, dq)
    with Bd.System(descs) as S:
        ref = Bd.to_numpy(S.run(y0, phi0, sid, kernel=Bd.IA_KERNEL_PLAIN, y_final=True))
    for k in ref:
        np.testing.assert_array_equal(g[k], ref[k], err_msg=k)
    single = ref["n_bounce"] == 1
    assert np.all(np.isfinite(tan["d_theta_s"][:, single]))
    assert np.all(np.isfinite(tan["ftle"]))


@pytest.mark.parametrize("species,E_K,q,theta,phi", OT.CASES)
def test_tangent_against_oracle_tangent_and_finite_differences(cuda, species, E_K, q, theta, phi):
    torch = cuda
    d, y0, E, dy0, dq = OT.make_case(species, E_K, q, theta, phi)
    rec, hs, mode = O.trajectory_steps(d, y0, 0.0)
    g, tan = gpu_tangent(torch, [d], y0[None, :], np.zeros(1), None, dy0[None, :, :], dq, dy_final=True)
    # same frozen step sequence on both sides (accept/reject decisions agree)
    assert g["n_steps"][0] == rec["n_steps"] and g["n_rej"][0] == rec["n_rej"]
    gt = np.stack([tan["d_theta_s"][:, 0], tan["d_dp"][:, 0], tan["d_dE_ion"][:, 0], tan["d_t_final"][:, 0]], axis=1)
    ot, odyf = O.tangent(d, y0, 0.0, hs, mode, dy0, dq)
    spread = OT.tangent_spread(d, y0, hs, mode, dy0, dq, ot)
    obs = [rec["theta_s"], rec["dp"], rec["dE_ion"], rec["t_final"]]
    ok = OT.agree(gt, ot, obs, E, q, spread)
    assert ok.all(), (np.argwhere(~ok).tolist(), (gt / ot - 1)[~ok])
    fd = OT.fd_reference(d, y0, hs, mode, dy0, dq, E, q)
    ok = OT.agree(gt, fd, obs, E, q, spread)
    assert ok.all(), (np.argwhere(~ok).tolist(), (gt / fd - 1)[~ok])
    # FTLE along direction 0 from the oracle's tangent of the final state
    inv_len = 1.0 / (0.5 * d["alpha"] / (2.0 * d["De"])) ** 0.25
    mu = d["m_ion"] * d["m_atom"] / (d["m_ion"] + d["m_atom"])
    inv_vel = 1.0 / np.sqrt(2.0 * d["De"] / mu)
    w = np.array([inv_len] * 3 + [inv_vel] * 3 + [inv_len] * 3 + [inv_vel] * 3)
    def ftle_of(dyf):
        return (np.log(np.linalg.norm(dyf * w)) - np.log(np.linalg.norm(dy0[0] * w))) / rec["t_final"]
    ftle = ftle_of(odyf[0])
    # the FTLE's own rounding noise: its change under six ulp perturbations of y0 (as the tangent spread)
    rng = np.random.default_rng(7)
    sp = 0.0
    for _ in range(6):
        yp = np.asarray(y0, dtype=np.float64) * (1.0 + rng.integers(-2, 3, 12) * 2.0 ** -52)
        _, pdyf = O.tangent(d, yp, 0.0, hs, mode, dy0, dq)
        sp = max(sp, abs(ftle_of(pdyf[0]) - ftle))
    assert abs(tan["ftle"][0] - ftle) <= max(1e-6 * abs(ftle), OT.K_SPREAD * sp) + 1e-9 / rec["t_final"], \
        (tan["ftle"][0], ftle, sp)
