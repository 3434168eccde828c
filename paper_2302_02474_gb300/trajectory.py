"""Derivatives through GJF trajectories (the differentiable form).

`gjf_trajectory_vjp` runs K GJF steps on a context and returns the
derivatives of a loss L(r^K, v^K) with respect to the initial positions and
velocities and to chi, kappa and a, holding the thermal noise fixed (the same
Philox counters). Reverse mode needs the states of every step in reverse
order; they are recomputed segment by segment from checkpoints taken every
`checkpoint_every` steps (bit-identical, since a step depends only on the
state and its counters). Checkpoints are device-memory state blobs. Each
reverse step is one call of the force's vector-Jacobian product
(tild_force_vjp); the adjoint recursion itself is a few FP64 vector updates
on device tensors.

One GJF step maps (r, v, F) to (r', v', F') with F' = F(r') and
  r' = r + b dt v + (b dt^2 / 2m) F + (b dt / 2m) beta,
  v' = a v + (dt / 2m)(a F + F'),
a = (1 - alpha dt/2m)/(1 + alpha dt/2m), b = 1/(1 + alpha dt/2m). With
h = dt/2m its adjoint is
  Fb'_tot = Fb' + h vb',   rb'_tot = rb' + J(r')^T Fb'_tot,
  rb = rb'_tot,  vb = b dt rb'_tot + a vb',  Fb = (b dt^2 / 2m) rb'_tot + h a vb',
and the parameters collect (dF/dtheta)(r')^T Fb'_tot at every step and at r^0.
"""
from __future__ import annotations

from typing import Dict, Optional

import numpy as np

from .binding import Tild


def gjf_trajectory_vjp(t: Tild, n_steps: int, r_bar, v_bar=None, checkpoint_every: int = 20) -> Dict[str, object]:
    """Derivatives of L through `n_steps` GJF steps of context `t` (positions
    and velocities set). r_bar, v_bar: dL/dr^K, dL/dv^K (n_beads x 3, by bead
    id; numpy arrays or CUDA tensors). Returns {"r0", "v0"} as numpy arrays
    and {"chi", "kappa", "a"}; `t` is left at step K. Checkpoints and the
    adjoint vectors stay in device memory (FP64)."""
    import torch

    if t.scheme != "gjf" or t.force_method != "ik":
        raise ValueError("gjf_trajectory_vjp needs the GJF scheme and the ik force")
    if n_steps < 0 or checkpoint_every < 1:
        raise ValueError("need n_steps >= 0 and checkpoint_every >= 1")
    dt, alpha, _kT, mass = t.integrator
    h = dt / (2.0 * mass)
    ga = (1.0 - alpha * h) / (1.0 + alpha * h)
    gb = 1.0 / (1.0 + alpha * h)
    c1, c2 = gb * dt, gb * dt * dt / (2.0 * mass)
    nbytes = t.state_bytes()

    def snapshot():
        return t.get_state(out=torch.empty(nbytes, dtype=torch.uint8, device="cuda"))

    def dev(x):
        if x is None:
            return torch.zeros((t.n_beads, 3), dtype=torch.float64, device="cuda")
        return torch.as_tensor(np.asarray(x) if not torch.is_tensor(x) else x, dtype=torch.float64,
                               device="cuda").reshape(-1, 3).clone()

    checkpoints = {0: snapshot()}
    for s in range(n_steps):
        t.step(1)
        if (s + 1) % checkpoint_every == 0:
            checkpoints[s + 1] = snapshot()
    final = snapshot()
    rb, vb, fb = dev(r_bar), dev(v_bar), dev(None)
    jt = torch.empty_like(rb)
    tb = {"chi": 0.0, "kappa": 0.0, "a": 0.0}
    for s0 in reversed(range(0, n_steps, checkpoint_every)):
        s1 = min(s0 + checkpoint_every, n_steps)
        # states s0 + 1 .. s1 of this segment, recomputed from its checkpoint
        t.set_state(checkpoints[s0])
        states = []
        for _ in range(s0, s1):
            t.step(1)
            states.append(snapshot())
        for k in range(s1 - s0 - 1, -1, -1):
            t.set_state(states[k])
            ft = fb + h * vb
            _, th = t.force_vjp(ft, out=jt)
            rt = rb + jt
            for key in tb:
                tb[key] += th[key]
            rb, vb, fb = rt, c1 * rt + ga * vb, c2 * rt + h * ga * vb
    t.set_state(checkpoints[0])
    _, th = t.force_vjp(fb, out=jt)
    for key in tb:
        tb[key] += th[key]
    t.set_state(final)
    return {"r0": (rb + jt).cpu().numpy(), "v0": vb.cpu().numpy(), **tb}
