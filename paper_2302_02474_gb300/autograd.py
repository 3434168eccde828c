"""torch.autograd binding of the TILD energy (differentiable form).

``tild_energy(t, positions, chi, kappa, a)`` returns the model's energy
U = E_bond + E_chi + E_kappa of the configuration as a 0-d tensor; its
backward gives dU/dpositions (the adjoint of the density assignment applied
to the potential fields, plus bonds) and dU/dchi, dU/dkappa, dU/da, all
computed by the CUDA library through ``tild_energy_gradient``.
"""
from __future__ import annotations

import torch

from .binding import Tild


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
