"""Adjoint (reverse-mode) kernel: primal bit-identity with ia_launch, agreement with the tangent kernel
(the same frozen-step map differentiated forwards), with the oracle's gradient, with the symmetries of
the trap-off equations, and independence of the checkpoint layout (needs a GB300)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_15117_gb300 import binding as Bd
from paper_2509_15117_gb300 import inputs as I
from tests import test_oracle_adjoint as OA
from tests import test_oracle_tangent as OT

pytestmark = pytest.mark.gpu

KEYS = ("d_theta_s", "d_dp", "d_dE_ion", "d_t_final")


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Bd.load()
    return torch


def gpu_adjoint(torch, descs, y0, phi0, sid, dy0=None, dq=None, **opts):
    n = len(phi0)
    with Bd.System(descs) as S:
        yd, pd, sd = Bd.to_device_soa(y0, phi0, sid)
        out = Bd.alloc_obs(n, y_final=True)
        ndir = 0 if dy0 is None else dy0.shape[1]
        adj = Bd.alloc_adjoint(n, ndir)
        dyd = None
        if dy0 is not None:
            dyd = torch.from_numpy(np.ascontiguousarray(np.transpose(dy0, (1, 2, 0)))).cuda()
        Bd.ia_launch_adjoint(S.handle, yd, pd, sd, out, adj, dyd, dq, **opts)
        torch.cuda.synchronize()
        return Bd.to_numpy(out), {k: v.cpu().numpy() for k, v in adj.items()}


def gpu_tangent(torch, descs, y0, phi0, sid, dy0, dq):
    from tests.test_gpu_tangent import gpu_tangent as gt
    return gt(torch, descs, y0, phi0, sid, dy0, dq)


def c1_batch(n_grid=16):
    systems, y0, phi0, sid = I.c1_workload(n_grid)
    descs = [s.as_dict() for s in systems]
    d = descs[0]
    E = I.kelvin(1.5e-6)
    v0 = I.speed_for_energy(E, d["m_atom"])
    th, ph = I.octant_grid(n_grid)
    seeds = I.head_on_seeds(th, ph, d["r0"], v0, E)
    dy0 = np.concatenate([seeds, np.zeros((len(th), 1, 12))], axis=1)
    dq = np.zeros((4, 3))
    dq[3] = I.q_direction()
    return descs, y0, phi0, sid, dy0, dq


def test_adjoint_primal_is_bitwise_the_launch(cuda):
    descs, y0, phi0, sid, dy0, dq = c1_batch(16)
    g, adj = gpu_adjoint(cuda, descs, y0, phi0, sid, dy0, dq)
    with Bd.System(descs) as S:
        ref = Bd.to_numpy(S.run(y0, phi0, sid, kernel=Bd.IA_KERNEL_PLAIN, y_final=True))
    for k in ref:
        np.testing.assert_array_equal(g[k], ref[k], err_msg=k)
    assert np.all(np.isfinite(adj["grad_y0"])) and np.all(np.isfinite(adj["grad_q"]))
    assert np.any(ref["n_bounce"] >= 2)


def test_adjoint_equals_tangent_along_seeds(cuda):
    """<grad J, v> from the reverse sweep against J'v from the forward sweep, on the same primal.
    Both sum the same products of step Jacobians in different orders; the bar is 4x the rounding
    response of the tangent (its largest change under six perturbations of the initial state by -2..2
    ulps per component) plus 1e-10 of the sum of magnitudes |grad| . |v|."""
    torch = cuda
    descs, y0, phi0, sid, dy0, dq = c1_batch(16)
    _, adj = gpu_adjoint(torch, descs, y0, phi0, sid, dy0, dq)
    _, tan = gpu_tangent(torch, descs, y0, phi0, sid, dy0, dq)
    spread = np.zeros_like(tan["d_theta_s"][None].repeat(4, 0))
    rng = np.random.default_rng(7)
    for _ in range(6):
        yp = np.asarray(y0, dtype=np.float64) * (1.0 + rng.integers(-2, 3, y0.shape) * 2.0 ** -52)
        _, tp = gpu_tangent(torch, descs, yp, phi0, sid, dy0, dq)
        for m, k in enumerate(KEYS):
            spread[m] = np.maximum(spread[m], np.abs(tp[k] - tan[k]))
    n = len(phi0)
    G = np.concatenate([adj["grad_y0"], adj["grad_q"]], axis=1)  # (4, 15, n)
    V = np.concatenate([np.transpose(dy0, (1, 2, 0)), np.broadcast_to(dq[:, :, None], (4, 3, n))], axis=1)
    for m, k in enumerate(KEYS):
        a, t = adj[k], tan[k]
        mag = np.einsum("cn,kcn->kn", np.abs(G[m]), np.abs(V))
        # the projections the kernel wrote are the inner products of its own gradient with the seeds
        assert np.all(np.abs(a - np.einsum("cn,kcn->kn", G[m], V)) <= 1e-13 * mag)
        bar = OT.K_SPREAD * spread[m] + 1e-10 * mag
        bad = np.abs(a - t) > bar
        assert not bad.any(), (k, np.argwhere(bad)[:5].tolist(), (np.abs(a - t) / np.maximum(mag, 1e-300))[bad][:5])


@pytest.mark.parametrize("species,E_K,q,theta,phi", OT.CASES)
def test_adjoint_against_oracle_gradient(cuda, species, E_K, q, theta, phi):
    torch = cuda
    d, y0, E, dy0, dq = OT.make_case(species, E_K, q, theta, phi)
    rec, hs, mode = O.trajectory_steps(d, y0, 0.0)
    g, adj = gpu_adjoint(torch, [d], y0[None, :], np.zeros(1), None, dy0[None, :, :], dq)
    assert g["n_steps"][0] == rec["n_steps"] and g["n_rej"][0] == rec["n_rej"]
    # projections on the (theta, phi, E, q) seeds against quad-precision central differences of the
    # frozen-step replay (the bar of the tangent kernel's test)
    ga = np.stack([adj[k][:, 0] for k in KEYS], axis=1)
    ot, _ = O.tangent(d, y0, 0.0, hs, mode, dy0, dq)
    spread = OT.tangent_spread(d, y0, hs, mode, dy0, dq, ot)
    fd = OT.fd_reference(d, y0, hs, mode, dy0, dq, E, q)
    obs = [rec["theta_s"], rec["dp"], rec["dE_ion"], rec["t_final"]]
    ok = OT.agree(ga, fd, obs, E, q, spread)
    assert ok.all(), (np.argwhere(~ok).tolist(), (ga / fd - 1)[~ok])
    oy, oq = O.gradient(d, y0, 0.0, hs, mode)
    # rounding response of the oracle's gradient (six perturbations of -2..2 ulps per component)
    sp = np.zeros((4, 15))
    rng = np.random.default_rng(7)
    for _ in range(6):
        yp = np.asarray(y0, dtype=np.float64) * (1.0 + rng.integers(-2, 3, 12) * 2.0 ** -52)
        py, pq = O.gradient(d, yp, 0.0, hs, mode)
        sp = np.maximum(sp, np.abs(np.concatenate([py - oy, pq - oq], axis=1)))
    s = OA.scales(d, E, q)
    go = np.concatenate([oy, oq], axis=1) * s
    gg = np.concatenate([adj["grad_y0"][:, :, 0], adj["grad_q"][:, :, 0]], axis=1) * s
    for m in range(4):
        bar = 1e-6 * np.max(np.abs(go[m])) + OT.K_SPREAD * sp[m] * s
        bad = np.abs(gg[m] - go[m]) > bar
        assert not bad.any(), (m, np.argwhere(bad).ravel().tolist(), gg[m][bad], go[m][bad])


def test_adjoint_trap_off_invariances(cuda):
    torch = cuda
    d, y0, E, dy0, dq = OT.make_case("Rb", 1e-3, 0.0, 0.9, 0.5)
    y0 = np.array(y0, copy=True)
    y0[0:3] = [37.0, -21.0, 12.5]
    y0[6:9] += y0[0:3]
    _, adj = gpu_adjoint(torch, [d], y0[None, :], np.zeros(1), None)
    s = OA.scales(d, E, 0.0)[:12]
    gy = adj["grad_y0"][:, :, 0]
    for gen in OA.generators(y0):
        for m in range(4):
            scale = np.linalg.norm(gy[m] * s) * np.linalg.norm(gen / s)
            assert abs(gy[m] @ gen) <= 1e-7 * scale


def test_adjoint_checkpoint_layout_does_not_change_bits(cuda):
    """Block length, checkpoint count (with repeated thinning) and warps in flight change only where
    the primal is recomputed, never the arithmetic: the gradients are bit-identical."""
    torch = cuda
    descs, y0, phi0, sid, dy0, dq = c1_batch(8)
    y0, phi0, sid, dy0 = y0[:16], phi0[:16], sid[:16], dy0[:16]
    _, ref = gpu_adjoint(torch, descs, y0, phi0, sid, dy0, dq)
    for opts in (dict(seg=64, max_ckpt=4), dict(seg=37, max_ckpt=6), dict(seg=1000, max_ckpt=2, warps=3)):
        _, a = gpu_adjoint(torch, descs, y0, phi0, sid, dy0, dq, **opts)
        for k in ref:
            np.testing.assert_array_equal(a[k], ref[k], err_msg=f"{k} {opts}")


def test_adjoint_bad_inputs(cuda):
    torch = cuda
    descs, y0, phi0, sid, dy0, dq = c1_batch(2)
    sid = np.array(sid if sid is not None else np.zeros(len(phi0)), dtype=np.int32)
    sid[1] = 7  # outside the one-row table
    y0 = np.array(y0, copy=True)
    y0[2, 6:9] = y0[2, 0:3]  # zero separation
    g, adj = gpu_adjoint(torch, descs, y0, phi0, sid, dy0, dq)
    assert g["status"][1] & Bd.ST_BAD_IC and g["status"][2] & Bd.ST_BAD_IC
    for k in ("grad_y0", "grad_q"):
        assert np.all(adj[k][..., 1] == 0.0) and np.all(adj[k][..., 2] == 0.0)
    assert np.all(np.isfinite(adj["grad_y0"][..., 0]))
    with Bd.System(descs) as S:
        yd, pd, sd = Bd.to_device_soa(y0, phi0, None)
        out = Bd.alloc_obs(len(phi0))
        a = Bd.alloc_adjoint(len(phi0))
        with pytest.raises(Bd.IaError):
            Bd.ia_launch_adjoint(S.handle, yd, pd, sd, out, a, max_ckpt=5)
        with pytest.raises(Bd.IaError):
            Bd.ia_launch_adjoint(S.handle, yd, pd, sd, out, {})


def test_autograd_function_backward_is_the_adjoint(cuda):
    """observables(...).backward() is the vector-Jacobian product of the adjoint kernel's gradients
    with the incoming cotangents (for y0 per trajectory, for q summed over the batch), and its
    forward values are the launch's observables. (The gradients themselves are checked against the
    tangent kernel, the oracle and finite differences above.)"""
    torch = cuda
    from paper_2509_15117_gb300 import autograd as AG
    descs, y0, phi0, sid, dy0, dq = c1_batch(4)
    d = descs[0]
    n = len(phi0)
    W = np.random.default_rng(3).standard_normal((n, 4))
    w = torch.tensor(W, dtype=torch.float64, device="cuda")
    yt = torch.tensor(y0, dtype=torch.float64, device="cuda", requires_grad=True)
    qt = torch.tensor(d["q"], dtype=torch.float64, requires_grad=True)
    obs = AG.observables(yt, qt, torch.tensor(phi0, dtype=torch.float64, device="cuda"), d)
    (obs * w).sum().backward()
    g, adj = gpu_adjoint(torch, descs, y0, phi0, sid)
    np.testing.assert_array_equal(obs.detach().cpu().numpy(),
                                  np.stack([g[k] for k in ("theta_s", "dp", "dE_ion", "t_final")], axis=1))
    ey = np.einsum("nm,mcn->nc", W, adj["grad_y0"])
    my = np.einsum("nm,mcn->nc", np.abs(W), np.abs(adj["grad_y0"]))
    assert np.all(np.abs(yt.grad.cpu().numpy() - ey) <= 1e-13 * my)
    eq = np.einsum("nm,mjn->j", W, adj["grad_q"])
    mq = np.einsum("nm,mjn->j", np.abs(W), np.abs(adj["grad_q"]))
    assert np.all(np.abs(qt.grad.numpy() - eq) <= 1e-13 * mq)
