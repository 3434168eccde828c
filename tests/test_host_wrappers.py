"""Host-side argument checks of the Python wrappers, on CPU: they reject
bad input before any library call."""
import types

import numpy as np
import pytest

from paper_2302_02474_gb300.trajectory import trajectory_vjp


def _fake(force_method="ik", n_beads=4):
    def no_call(*a, **k):
        raise AssertionError("the library must not be called")

    return types.SimpleNamespace(force_method=force_method, n_beads=n_beads, ctx=None, _chk=no_call,
                                 lib=types.SimpleNamespace(tild_trajectory_vjp=no_call))


def test_trajectory_vjp_needs_the_ik_force():
    with pytest.raises(ValueError, match="ik force"):
        trajectory_vjp(_fake("analytic"), 3, np.zeros((4, 3)))


@pytest.mark.parametrize("r_shape,v_shape", [((3, 3), None), ((4, 3), (5, 3)), ((12, 1), (4, 2))])
def test_trajectory_vjp_checks_array_sizes(r_shape, v_shape):
    v = None if v_shape is None else np.zeros(v_shape)
    with pytest.raises(ValueError, match="n_beads x 3"):
        trajectory_vjp(_fake(), 3, np.zeros(r_shape), v)
