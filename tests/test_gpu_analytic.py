"""The analytic-differentiation force (F_i = -sum_g grad W(r_i - g) w_K(g),
one inverse transform of the potentials) on the GPU against the oracle's
variant="analytic", through the C ABI. Tolerances as in test_gpu_parity."""
import numpy as np
import pytest

from oracle import tild_oracle as O
from paper_2302_02474_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_02474_gb300 import _build, binding

    _build.build()
    return binding


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def _analytic(m, p):
    return O.forces(m, p, variant="analytic")


def _setup(B, spec, sort_every=4):
    pos = I.initial_positions(spec)
    if spec.precision == "fp32":
        pos = pos.astype(np.float32).astype(np.float64)
    t = B.Tild.from_spec(spec, sort_every=sort_every)
    t.set_force_method("analytic")
    t.set_positions(pos)
    m = O.model_from_spec(spec, I.species_of_beads(spec.moltypes), I.bond_pairs(spec.moltypes))
    return t, m, pos


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_analytic_forces_and_energies(B, prec, order):
    spec = I.small_system(n_chains=83, N=10, n_a=4, L=8.0, n=16, pmeorder=order, precision=prec, chi=1.3, kappa=7.0)
    t, m, pos = _setup(B, spec)
    t.init_velocities()
    f, e = t.compute()
    assert _rel(f, _analytic(m, pos)) < (1e-12 if prec == "fp64" else 1e-5)
    eref = O.energies(m, pos)
    for k in ("bond", "chi", "kappa"):
        assert abs(e[k] - eref[k]) <= (1e-10 if prec == "fp64" else 1e-6) * abs(eref[k])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_analytic_ten_step_trajectory(B, prec):
    spec = I.small_system(n_chains=97, N=10, n_a=4, L=9.0, n=16, precision=prec, chi=1.2, kappa=8.0)
    t, m, pos = _setup(B, spec)
    t.init_velocities()
    t.step(10)
    t.synchronize()
    st = O.run(m, O.initial_state(m, pos, force_fn=_analytic), 10, force_fn=_analytic)
    d = np.abs(O.minimum_image(t.positions() - st.pos, m.L)).max()
    if prec == "fp64":
        assert d < 1e-10
        assert _rel(t.velocities(), st.vel) < 1e-10
    else:
        assert d < 1e-4 * m.L
        assert _rel(t.velocities(), st.vel) < 1e-4


def test_analytic_force_is_minus_position_gradient(B):
    """The step's force and tild_energy_gradient's dU/dr are two GPU paths
    to the same quantity."""
    spec = I.small_system(n_chains=60, N=10, n_a=4, L=8.0, n=16, pmeorder=2, precision="fp64", chi=0.9, kappa=6.0)
    t, m, pos = _setup(B, spec)
    f, _ = t.compute()
    _, dudr = t.energy_gradient()
    assert _rel(f, -dudr) < 1e-12


def test_analytic_force_conserves_energy_under_velocity_verlet(B):
    """The analytic force is the exact gradient of the gridded energy, so
    frictionless velocity-Verlet keeps E = U + kinetic within the O(dt^2)
    shadow-energy band."""
    spec = I.small_system(n_chains=40, N=10, n_a=4, L=7.0, n=16, precision="fp64", chi=1.0, kappa=6.0,
                          friction=0.0, dt=0.004)
    t, m, pos = _setup(B, spec, sort_every=10)
    t.set_scheme("vv")
    t.init_velocities()

    def total():
        _, e = t.compute()
        return e["bond"] + e["chi"] + e["kappa"] + e["kinetic"], e["kinetic"]

    e0, k0 = total()
    es = []
    for _ in range(20):
        t.step(10)
        es.append(total()[0])
    assert np.abs(np.array(es) - e0).max() < 2e-3 * k0


def test_field_gradient_and_batches_under_the_analytic_method(B):
    spec = I.small_system(n_chains=50, N=10, n_a=4, L=8.0, n=16, precision="fp32", chi=1.0, kappa=6.0)
    t, m, pos = _setup(B, spec)
    g_an = t.field_gradient()
    t.set_force_method("ik")
    assert np.array_equal(g_an, t.field_gradient())
    t.set_force_method("analytic")
    t.init_velocities()
    with pytest.raises(B.TildError, match="EUNSUPPORTED"):
        B.TildBatch([t])
