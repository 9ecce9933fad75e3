"""torch.autograd front end of the trajectory engine.

``observables(y0, q, phi0, desc)`` integrates a batch of trajectories of one system (Eq. 1 with the
C8-C4 potential, DP5(4), exit at r0) and returns, per trajectory, the observables of the Fig. 1 caption
plus the ion energy change and the exit time: columns (theta_s, |p_f - p_i|, dE_ion, t_final). It is
differentiable with respect to the initial states y0 (n, 12) and the trap's q vector (3,): the backward
pass runs the adjoint kernel (checkpointed reverse sweep of the frozen-step map) and contracts its
per-trajectory gradients with the incoming cotangents. Everything runs through the C ABI; tensors
must be float64 on the CUDA device.
"""
from __future__ import annotations

import torch

from . import binding as Bd

COLUMNS = ("theta_s", "dp", "dE_ion", "t_final")


def _system_desc(desc: dict, q: torch.Tensor) -> dict:
    d = dict(desc)
    d["q"] = [float(v) for v in q.detach().to("cpu", torch.float64)]
    return d


class IonAtomFn(torch.autograd.Function):
    """y0 (n, 12), q (3,), phi0 (n,) -> observables (n, 4); see the module docstring."""

    @staticmethod
    def forward(ctx, y0, q, phi0, desc, adjoint_opts):
        if not (y0.is_cuda and phi0.is_cuda) or y0.dtype != torch.float64 or phi0.dtype != torch.float64:
            raise TypeError("y0 and phi0 must be float64 CUDA tensors")
        if y0.dim() != 2 or y0.shape[1] != 12 or phi0.shape != (y0.shape[0],) or q.shape != (3,):
            raise ValueError("shapes: y0 (n, 12), q (3,), phi0 (n,)")
        d = _system_desc(desc, q)
        n = int(y0.shape[0])
        y0_soa = y0.detach().t().contiguous()
        ph = phi0.detach().contiguous()
        out = Bd.alloc_obs(n, device=y0.device)
        with Bd.System([d]) as S:
            Bd.ia_launch(S.handle, y0_soa, ph, None, out)
            torch.cuda.current_stream().synchronize()  # the table is freed on leaving the block
        ctx.save_for_backward(y0_soa, ph)
        ctx.desc = d
        ctx.q_device = q.device
        ctx.adjoint_opts = dict(adjoint_opts or {})
        obs = torch.stack([out[c] for c in COLUMNS], dim=1)
        return obs

    @staticmethod
    def backward(ctx, g_obs):
        y0_soa, ph = ctx.saved_tensors
        n = int(ph.shape[0])
        out = Bd.alloc_obs(n, device=ph.device)
        adj = Bd.alloc_adjoint(n, 0, device=ph.device)
        with Bd.System([ctx.desc]) as S:
            Bd.ia_launch_adjoint(S.handle, y0_soa, ph, None, out, adj, **ctx.adjoint_opts)
            torch.cuda.current_stream().synchronize()
        g = g_obs.to(torch.float64).contiguous()
        gy0 = gq = None
        if ctx.needs_input_grad[0]:
            gy0 = torch.einsum("nm,mcn->nc", g, adj["grad_y0"])
        if ctx.needs_input_grad[1]:
            gq = torch.einsum("nm,mjn->j", g, adj["grad_q"]).to(ctx.q_device)
        return gy0, gq, None, None, None


def observables(y0: torch.Tensor, q: torch.Tensor, phi0: torch.Tensor, desc: dict,
                adjoint_opts: dict | None = None) -> torch.Tensor:
    """Differentiable observables (n, 4) = (theta_s, dp, dE_ion, t_final) of one system's batch.
    desc: the system descriptor (its "q" entry is replaced by q); adjoint_opts: seg, max_ckpt, warps."""
    return IonAtomFn.apply(y0, q, phi0, desc, adjoint_opts)
