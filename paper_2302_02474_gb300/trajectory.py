"""Derivatives through GJF trajectories (the differentiable form).

`gjf_trajectory_vjp` runs K GJF steps on a context and returns the
derivatives of a loss L(r^K, v^K) with respect to the initial positions and
velocities and to chi, kappa and a, holding the thermal noise fixed (the same
Philox counters). Reverse mode needs the states of every step in reverse
order; they are recomputed segment by segment from checkpoints taken every
`checkpoint_every` steps (bit-identical, since a step depends only on the
state and its counters). The sweep runs in the library: device
checkpoints, one force vector-Jacobian product per reverse step and the
adjoint recursion below on FP64 device vectors, all stream-ordered with one
host synchronisation at the end.

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

import ctypes

from .binding import TILD_DTYPE_F64, TILD_HOST, Tild


def gjf_trajectory_vjp(t: Tild, n_steps: int, r_bar, v_bar=None, checkpoint_every: int = 20) -> Dict[str, object]:
    """Derivatives of L through `n_steps` GJF steps of context `t` (positions
    and velocities set). r_bar, v_bar: dL/dr^K, dL/dv^K (n_beads x 3, by bead
    id; numpy arrays or CUDA tensors). Returns {"r0", "v0"} (numpy FP64) and
    {"chi", "kappa", "a"}; `t` is left at step K. The sweep runs inside the
    library (tild_gjf_trajectory_vjp)."""
    if t.scheme != "gjf" or t.force_method != "ik":
        raise ValueError("gjf_trajectory_vjp needs the GJF scheme and the ik force")
    n3 = 3 * t.n_beads
    rb = np.ascontiguousarray(np.asarray(r_bar.cpu() if hasattr(r_bar, "cpu") else r_bar, dtype=np.float64)).reshape(-1)
    vb = None
    if v_bar is not None:
        vb = np.ascontiguousarray(np.asarray(v_bar.cpu() if hasattr(v_bar, "cpu") else v_bar, dtype=np.float64)).reshape(-1)
    if rb.size != n3 or (vb is not None and vb.size != n3):
        raise ValueError("r_bar and v_bar need n_beads x 3 values")
    r0 = np.empty(n3, dtype=np.float64)
    v0 = np.empty(n3, dtype=np.float64)
    th = (ctypes.c_double * 3)()
    t._chk(t.lib.tild_gjf_trajectory_vjp(t.ctx, int(n_steps), int(checkpoint_every), rb.ctypes.data,
                                         None if vb is None else vb.ctypes.data, TILD_DTYPE_F64, TILD_HOST,
                                         r0.ctypes.data, v0.ctypes.data, th))
    return {"r0": r0.reshape(-1, 3), "v0": v0.reshape(-1, 3), "chi": th[0], "kappa": th[1], "a": th[2]}
