"""Euler-Maruyama and velocity-Verlet + Langevin force (the other two
integrators of Sec. "Integrator Class") on the GPU against the oracle's
em_step / vv_step, through the C ABI. Tolerances as in test_gpu_parity:
1e-10 in FP64, 1e-4 L (positions) and 1e-4 relative (velocities) in FP32
after 10 steps."""
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


def _setup(B, spec, scheme, sort_every=4):
    pos = I.initial_positions(spec)
    if spec.precision == "fp32":
        pos = pos.astype(np.float32).astype(np.float64)
    t = B.Tild.from_spec(spec, sort_every=sort_every)
    t.set_scheme(scheme)
    t.set_positions(pos)
    m = O.model_from_spec(spec, I.species_of_beads(spec.moltypes), I.bond_pairs(spec.moltypes))
    return t, m, pos


def _spec(prec, **kw):
    return I.small_system(n_chains=97, N=10, n_a=4, L=9.0, n=16, precision=prec, chi=1.2, kappa=8.0, **kw)


def _close(prec, m, r, r_ref, v=None, v_ref=None):
    d = np.abs(O.minimum_image(r - r_ref, m.L)).max()
    if prec == "fp64":
        assert d < 1e-10
    else:
        assert d < 1e-4 * m.L
    if v is not None:
        rel = np.linalg.norm(v - v_ref) / np.linalg.norm(v_ref)
        assert rel < (1e-10 if prec == "fp64" else 1e-4)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_euler_maruyama_trajectory(B, prec):
    spec = _spec(prec, friction=2.0)
    t, m, pos = _setup(B, spec, "em")
    t.init_velocities()
    t.step(10)
    t.synchronize()
    st = O.run_with(O.em_step, m, O.em_initial_state(m, pos), 10)
    _close(prec, m, t.positions(), st.pos)
    assert not np.any(t.velocities())
    _, e = t.compute()
    assert e["kinetic"] == 0.0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("friction", [0.0, 1.5])
def test_velocity_verlet_trajectory_and_velocities(B, prec, friction):
    spec = _spec(prec, friction=friction)
    t, m, pos = _setup(B, spec, "vv")
    t.init_velocities()
    v0 = O.initial_state(m, pos).vel  # Maxwell-Boltzmann draw shared by all schemes
    _close(prec, m, t.positions(), O.wrap(pos, m.L), t.velocities(), v0)
    t.step(10)
    t.synchronize()
    st = O.run_with(O.vv_step, m, O.vv_initial_state(m, pos, v0), 10)
    _close(prec, m, t.positions(), st.pos, t.velocities(), st.vel)
    # kinetic energy of the reported velocities
    _, e = t.compute()
    assert e["kinetic"] == pytest.approx(O.kinetic_energy(m, st.vel), rel=1e-9 if prec == "fp64" else 1e-4)


def test_scheme_switch_keeps_velocities(B):
    spec = _spec("fp64", friction=1.0)
    t, m, pos = _setup(B, spec, "gjf")
    t.init_velocities()
    t.step(6)
    t.synchronize()
    r6, v6 = t.positions(), t.velocities()
    t.set_scheme("vv")
    np.testing.assert_allclose(t.velocities(), v6, rtol=0, atol=1e-12)
    t.step(6)
    t.synchronize()
    st = O.run_with(O.vv_step, m, O.vv_initial_state(m, r6, v6, step=6), 6)
    _close("fp64", m, t.positions(), st.pos, t.velocities(), st.vel)
    t.set_scheme("em")
    assert not np.any(t.velocities())
    t.set_scheme("gjf")  # starts from v = 0 (carried state u = -(dt/2m) F, so v = 0 up to rounding)
    assert np.abs(t.velocities()).max() < 1e-12


def test_scheme_limits_are_rejected(B):
    spec = _spec("fp64", friction=0.0)
    t, m, pos = _setup(B, spec, "gjf")
    with pytest.raises(B.TildError, match="EINVAL"):
        t.set_scheme("em")  # needs friction > 0
    t.set_scheme("vv")
    with pytest.raises(B.TildError, match="EINVAL"):
        t.set_integrator(0.01, 400.0, 1.0, 1.0)  # friction dt / 2m >= 1
    with pytest.raises(B.TildError, match="EINVAL"):
        t._chk(t.lib.tild_set_integrator_scheme(t.ctx, 7))


def test_batch_with_mixed_schemes_matches_individual_bitwise(B):
    specs = [_spec("fp32", friction=f, seed=s) for f, s in ((1.0, 31), (2.0, 32), (0.5, 33))]
    schemes = ["gjf", "em", "vv"]

    def make():
        out = []
        for s, sc in zip(specs, schemes):
            t, _, _ = _setup(B, s, sc, sort_every=5)
            t.init_velocities()
            out.append(t)
        return out

    batch, alone = make(), make()
    with B.TildBatch(batch) as bt:
        bt.step(23)
        bt.synchronize()
    for t in alone:
        t.step(23)
        t.synchronize()
    for tb, ta in zip(batch, alone):
        assert np.array_equal(tb.positions(), ta.positions())
        assert np.array_equal(tb.velocities(), ta.velocities())
