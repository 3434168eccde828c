"""torch.autograd bindings of the differentiable form.

``tild_energy(t, positions, chi, kappa, a)`` returns the model's energy
U = E_bond + E_chi + E_kappa of the configuration as a 0-d tensor; its
backward gives dU/dpositions (the adjoint of the density assignment applied
to the potential fields, plus bonds) and dU/dchi, dU/dkappa, dU/da, all
computed by the CUDA library through ``tild_energy_gradient``.

``tild_trajectory(t, n_steps, positions, velocities, chi, kappa, a)`` runs
n_steps steps of the context's scheme (ik force) and returns r^K, v^K; its
backward gives the derivatives of the loss with respect to the initial
positions and velocities and to chi, kappa, a through
``tild_trajectory_vjp`` (the thermal noise held fixed).
"""
from __future__ import annotations

import torch

from .binding import Tild
from .trajectory import trajectory_vjp


class TildEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, tild: Tild, positions: torch.Tensor, chi: torch.Tensor, kappa: torch.Tensor,
                a: torch.Tensor):
        tild.set_interactions(float(chi), float(kappa), float(a))
        pos = positions.detach().contiguous()
        tild.set_positions(pos)
        dudr = torch.empty(3 * tild.n_beads, dtype=pos.dtype, device=pos.device)
        g, _ = tild.energy_gradient(out=dudr)
        ctx.save_for_backward(dudr.view(-1, 3))
        ctx.dparams = (g["dU_dchi"], g["dU_dkappa"], g["dU_da"])
        ctx.param_meta = [(p.dtype, p.device) for p in (chi, kappa, a)]
        return torch.tensor(g["energy"], dtype=torch.float64, device=pos.device)

    @staticmethod
    def backward(ctx, grad_out):
        (dudr,) = ctx.saved_tensors
        gp = [torch.as_tensor(v, dtype=dt, device=dev) * grad_out.to(dt)
              for v, (dt, dev) in zip(ctx.dparams, ctx.param_meta)]
        return None, dudr * grad_out.to(dudr.dtype), gp[0], gp[1], gp[2]


def tild_energy(tild: Tild, positions: torch.Tensor, chi, kappa, a) -> torch.Tensor:
    """Differentiable energy of `positions` ([n_beads, 3]) for parameters chi, kappa, a."""
    as_t = lambda v: v if isinstance(v, torch.Tensor) else torch.tensor(float(v), dtype=torch.float64)
    return TildEnergy.apply(tild, positions, as_t(chi), as_t(kappa), as_t(a))


class TildTrajectory(torch.autograd.Function):
    """r^K, v^K after n_steps steps from (positions, velocities) with the
    parameters (chi, kappa, a); the step counter starts at 0, so the noise is
    that of Philox counters 1..K. Positions come back wrapped into [0, L);
    derivatives are those of the unwrapped trajectory (wrapping is a
    translation by box vectors). The backward restores the start state,
    runs the reverse sweep and puts the context back where it was: its
    state and the interaction parameters current before the backward."""

    @staticmethod
    def forward(ctx, tild: Tild, n_steps: int, checkpoint_every: int, positions: torch.Tensor,
                velocities: torch.Tensor, chi: torch.Tensor, kappa: torch.Tensor, a: torch.Tensor):
        params = (float(chi), float(kappa), float(a))
        tild.set_interactions(*params)
        pos = positions.detach().contiguous()
        tild.set_positions(pos)
        tild.set_velocities(velocities.detach().to(pos.dtype).contiguous())
        ctx.start = tild.get_state()
        tild.step(int(n_steps))
        r_k = torch.empty(3 * tild.n_beads, dtype=pos.dtype, device=pos.device)
        v_k = torch.empty_like(r_k)
        tild.positions(out=r_k)
        tild.velocities(out=v_k)
        ctx.tild, ctx.params, ctx.n, ctx.every = tild, params, int(n_steps), int(checkpoint_every)
        ctx.pos_meta = (pos.dtype, pos.device)
        ctx.param_meta = [(p.dtype, p.device) for p in (chi, kappa, a)]
        return r_k.view(-1, 3), v_k.view(-1, 3)

    @staticmethod
    def backward(ctx, grad_r, grad_v):
        t = ctx.tild
        here = t.get_state()
        before = t.interactions  # the parameters current before this backward
        t.set_interactions(*ctx.params)
        t.set_state(ctx.start)
        dt, dev = ctx.pos_meta
        if grad_r is None:
            grad_r = torch.zeros(t.n_beads, 3, dtype=torch.float64, device=dev)
        if dev.type == "cuda":
            # adjoint vectors stay on the device (no host round trip)
            gr = grad_r.detach().to(device=dev, dtype=torch.float64)
            gv = None if grad_v is None else grad_v.detach().to(device=dev, dtype=torch.float64)
        else:
            gr = grad_r.detach().double().cpu().numpy()
            gv = None if grad_v is None else grad_v.detach().double().cpu().numpy()
        g = trajectory_vjp(t, ctx.n, gr, gv, ctx.every)
        # the parameters first: the saved state's carried velocity belongs to them
        if before is not None:
            t.set_interactions(*before)
        t.set_state(here)
        d_r0 = torch.as_tensor(g["r0"], device=dev).to(dt)
        d_v0 = torch.as_tensor(g["v0"], device=dev).to(dt)
        gp = [torch.as_tensor(g[k], dtype=d, device=v) for k, (d, v) in zip(("chi", "kappa", "a"), ctx.param_meta)]
        return None, None, None, d_r0, d_v0, gp[0], gp[1], gp[2]


def tild_trajectory(tild: Tild, n_steps: int, positions: torch.Tensor, velocities: torch.Tensor, chi, kappa, a,
                    checkpoint_every: int = 20):
    """Differentiable (r^K, v^K) after `n_steps` steps of context `tild` from
    `positions`, `velocities` ([n_beads, 3]) with parameters chi, kappa, a."""
    as_t = lambda v: v if isinstance(v, torch.Tensor) else torch.tensor(float(v), dtype=torch.float64)
    return TildTrajectory.apply(tild, n_steps, checkpoint_every, positions, velocities, as_t(chi), as_t(kappa),
                                as_t(a))
