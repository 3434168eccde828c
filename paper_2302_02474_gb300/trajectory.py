"""Derivatives through trajectories (the differentiable form).

`trajectory_vjp` runs K steps of a context's integrator scheme (GJF, EM or
VV + Langevin, with the ik force) and returns the derivatives of a loss
L(r^K, v^K) with respect to the initial positions and velocities and to chi,
kappa and a, holding the thermal noise fixed (the same Philox counters).
Reverse mode needs the states of every step in reverse order; they are
recomputed segment by segment from checkpoints taken every
`checkpoint_every` steps (bit-identical, since a step depends only on the
state and its counters). The sweep runs in the library: device
checkpoints, one force vector-Jacobian product per state and the adjoint
recursion below on FP64 device vectors, all stream-ordered with one host
synchronisation at the end.

Every scheme advances the state (r, u), u the carried velocity, in one
linear form with F = F(r) and fixed normals xi:
  h = su u + sf F + sg xi,   r' = r + sd h + se xi,   u' = sh h + sk xi,
with the velocity of a state v = vu u + vf F + vg xi and the initial
u^0 = wu v^0 + wf F(r^0) + wg xi. GJF (a = (1 - alpha dt/2m)/(1 + alpha
dt/2m), b = 1/(1 + alpha dt/2m)): u = v - (dt/2m) F, su = 1, sf = dt/m,
sd = b dt, sh = a. EM: su = sh = 0, sf = dt/alpha, sd = 1, no velocity. VV:
u is the half-step velocity v^{n-1/2}; the Langevin force -alpha u + s xi
folds into su = 1 - alpha dt/m and sg. The adjoint of one step is
  hb = sd rb' + sh ub',   ub = su hb,   rb = rb' + J(r)^T (sf hb),
the loss enters through ub^K = vu vb^K and J(r^K)^T (vf vb^K), the start
through J(r^0)^T (wf ub^0) and dL/dv^0 = wu ub^0, and the parameters collect
(dF/dtheta)^T of the same adjoint vectors.
"""
from __future__ import annotations

import ctypes
from typing import Dict

import numpy as np

from .binding import TILD_DEVICE, TILD_DTYPE_F64, TILD_HOST, Tild


def _is_cuda_tensor(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


def trajectory_vjp(t: Tild, n_steps: int, r_bar, v_bar=None, checkpoint_every: int = 20) -> Dict[str, object]:
    """Derivatives of L through `n_steps` steps of context `t` (positions and
    velocities set; any scheme, ik force). r_bar, v_bar: dL/dr^K, dL/dv^K
    (n_beads x 3, by bead id; numpy arrays or CUDA tensors). Returns
    {"r0", "v0"} and {"chi", "kappa", "a"}; `t` is left at step K. The sweep
    runs inside the library (tild_trajectory_vjp). With a CUDA tensor r_bar
    the adjoint vectors stay on the device (FP64 CUDA tensors in and out, no
    host copy); otherwise r0 and v0 are numpy FP64 arrays."""
    if t.force_method != "ik":
        raise ValueError("trajectory_vjp needs the ik force")
    n3 = 3 * t.n_beads
    th = (ctypes.c_double * 3)()
    if _is_cuda_tensor(r_bar):
        import torch

        rb = r_bar.detach().to(torch.float64).contiguous().view(-1)
        vb = None
        if v_bar is not None:
            if not _is_cuda_tensor(v_bar):
                raise ValueError("r_bar and v_bar must both be CUDA tensors or both host arrays")
            vb = v_bar.detach().to(device=rb.device, dtype=torch.float64).contiguous().view(-1)
        if rb.numel() != n3 or (vb is not None and vb.numel() != n3):
            raise ValueError("r_bar and v_bar need n_beads x 3 values")
        r0 = torch.empty(n3, dtype=torch.float64, device=rb.device)
        v0 = torch.empty_like(r0)
        t._chk(t.lib.tild_trajectory_vjp(t.ctx, int(n_steps), int(checkpoint_every), ctypes.c_void_p(rb.data_ptr()),
                                         None if vb is None else ctypes.c_void_p(vb.data_ptr()), TILD_DTYPE_F64,
                                         TILD_DEVICE, ctypes.c_void_p(r0.data_ptr()), ctypes.c_void_p(v0.data_ptr()),
                                         th))
        return {"r0": r0.view(-1, 3), "v0": v0.view(-1, 3), "chi": th[0], "kappa": th[1], "a": th[2]}
    rb = np.ascontiguousarray(np.asarray(r_bar.cpu() if hasattr(r_bar, "cpu") else r_bar, dtype=np.float64)).reshape(-1)
    vb = None
    if v_bar is not None:
        vb = np.ascontiguousarray(np.asarray(v_bar.cpu() if hasattr(v_bar, "cpu") else v_bar, dtype=np.float64)).reshape(-1)
    if rb.size != n3 or (vb is not None and vb.size != n3):
        raise ValueError("r_bar and v_bar need n_beads x 3 values")
    r0 = np.empty(n3, dtype=np.float64)
    v0 = np.empty(n3, dtype=np.float64)
    t._chk(t.lib.tild_trajectory_vjp(t.ctx, int(n_steps), int(checkpoint_every), rb.ctypes.data,
                                     None if vb is None else vb.ctypes.data, TILD_DTYPE_F64, TILD_HOST,
                                     r0.ctypes.data, v0.ctypes.data, th))
    return {"r0": r0.reshape(-1, 3), "v0": v0.reshape(-1, 3), "chi": th[0], "kappa": th[1], "a": th[2]}


def profile_loss_gradient(t: Tild, n_steps: int, target, weight: float = 1.0, axis: int = 2,
                          checkpoint_every: int = 20, energy_weight: float = 1.0) -> Dict[str, object]:
    """The differentiable form's density-profile objective through a
    trajectory: after `n_steps` steps from the current state,
      L = energy_weight * U(r^K) + weight * sum_j (p_A(j) - target(j))^2,
    U the gridded energy (E_bond + E_chi + E_kappa, Eqs. bonds, fh, HelfandP)
    and p_A the species-0 density averaged over the two grid axes other than
    `axis` (a length-n profile; axis 2 = z). Returns L and its derivatives
    with respect to chi, kappa and a (the energy's explicit dependence at
    r^K plus the trajectory's) and to r^0 and v^0.

    dL/dr^K is the energy gradient (tild_energy_gradient) plus the density
    term carried back to the positions by the assignment's vector-Jacobian
    product (tild_density_vjp) of dL/drho_A(g) = 2 weight (p_A - target)/n^2
    along the profile; the reverse sweep is tild_trajectory_vjp. The forward
    is run twice (once to reach r^K, once inside the sweep); the context ends
    at step K. Needs CUDA (the grids stay on the device)."""
    import torch

    n = t.n
    dev = torch.device("cuda", torch.cuda.current_device())
    start = torch.empty(t.state_bytes(), dtype=torch.uint8, device=dev)
    t.get_state(start)
    t.step(int(n_steps))
    t.synchronize()
    e, dU_dr = t.energy_gradient()
    rho = torch.empty(t.n_species * n ** 3, dtype=torch.float64, device=dev)
    t.density(out=rho)
    rhoA = rho.view(t.n_species, n, n, n)[0]  # [z][y][x]
    dims = {0: (0, 1), 1: (0, 2), 2: (1, 2)}[axis]  # axis x, y, z of the [z][y][x] grid
    prof = rhoA.mean(dim=dims)
    tgt = torch.as_tensor(np.asarray(target, dtype=np.float64), device=dev)
    resid = prof - tgt
    loss_prof = float(weight * torch.sum(resid * resid))
    shape = [1, 1, 1]
    shape[2 - axis] = n
    psi = torch.zeros(t.n_species, n, n, n, dtype=torch.float64, device=dev)
    psi[0] = (2.0 * weight / (n * n)) * resid.view(*shape).expand(n, n, n)
    dens_bar = torch.empty(3 * t.n_beads, dtype=torch.float64, device=dev)
    t.density_vjp(psi.view(-1), out=dens_bar)
    ew = float(energy_weight)
    r_bar = dens_bar.view(-1, 3) + ew * torch.as_tensor(dU_dr, device=dev)
    t.set_state(start)
    g = trajectory_vjp(t, int(n_steps), r_bar, None, checkpoint_every)
    return {"loss": ew * e["energy"] + loss_prof, "energy": e["energy"], "profile_loss": loss_prof,
            "profile": prof.cpu().numpy(), "chi": ew * e["dU_dchi"] + g["chi"], "kappa": ew * e["dU_dkappa"] + g["kappa"],
            "a": ew * e["dU_da"] + g["a"], "r0": g["r0"], "v0": g["v0"]}
