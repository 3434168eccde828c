"""Smeared-charge electrostatics (per-species charges, Bjerrum length,
charge spreading length) on the GPU against the oracle, through the C ABI.
Tolerances as in test_gpu_parity."""
import numpy as np
import pytest

from oracle import tild_oracle as O
from paper_2302_02474_gb300 import inputs as I

pytestmark = pytest.mark.gpu

Q = (1.0, -1.0)  # polycation / polyanion, as in the paper's coacervate example
LB, AE = 2.0, 0.6


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


def _setup(B, spec, q=Q, lb=LB, ae=AE, method="ik", sort_every=4):
    pos = I.initial_positions(spec)
    if spec.precision == "fp32":
        pos = pos.astype(np.float32).astype(np.float64)
    t = B.Tild.from_spec(spec, sort_every=sort_every)
    t.set_electrostatics(q[0], q[1], lb, ae)
    t.set_force_method(method)
    t.set_positions(pos)
    m = O.model_from_spec(spec, I.species_of_beads(spec.moltypes), I.bond_pairs(spec.moltypes))
    m.charges, m.bjerrum, m.charge_smear = np.array(q), lb, ae
    return t, m, pos


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("order,method", [(1, "ik"), (3, "ik"), (1, "analytic"), (2, "analytic")])
def test_charged_forces_and_energies(B, prec, order, method):
    spec = I.small_system(n_chains=83, N=10, n_a=4, L=8.0, n=16, pmeorder=order, precision=prec, chi=0.6, kappa=7.0)
    t, m, pos = _setup(B, spec, q=(0.8, -1.3), method=method)
    t.init_velocities()
    f, e = t.compute()
    assert _rel(f, O.forces(m, pos, variant=method)) < (1e-12 if prec == "fp64" else 1e-5)
    eref = O.energies(m, pos)
    assert abs(eref["elec"]) > 1e-2
    for k in ("bond", "chi", "kappa", "elec"):
        assert abs(e[k] - eref[k]) <= (1e-10 if prec == "fp64" else 1e-6) * abs(eref[k]), k


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_charged_ten_step_trajectory(B, prec):
    spec = I.small_system(n_chains=97, N=10, n_a=5, L=9.0, n=16, precision=prec, chi=0.5, kappa=8.0)
    t, m, pos = _setup(B, spec)
    t.init_velocities()
    t.step(10)
    t.synchronize()
    st = O.run(m, O.initial_state(m, pos), 10)
    d = np.abs(O.minimum_image(t.positions() - st.pos, m.L)).max()
    if prec == "fp64":
        assert d < 1e-10
        assert _rel(t.velocities(), st.vel) < 1e-10
    else:
        assert d < 1e-4 * m.L
        assert _rel(t.velocities(), st.vel) < 1e-4


def test_charged_energy_gradient(B):
    spec = I.small_system(n_chains=50, N=10, n_a=4, L=8.0, n=16, pmeorder=2, precision="fp64", chi=0.9, kappa=6.0)
    t, m, pos = _setup(B, spec)
    g, dudr = t.energy_gradient()
    eref = O.energies(m, pos)
    assert g["e_elec"] == pytest.approx(eref["elec"], rel=1e-10)
    assert g["energy"] == pytest.approx(sum(eref[k] for k in ("bond", "chi", "kappa", "elec")), rel=1e-10)
    assert _rel(dudr, -O.forces(m, pos, variant="analytic")) < 1e-12


def test_electrostatics_off_and_invalid(B):
    spec = I.small_system(n_chains=40, N=10, n_a=4, L=8.0, n=16, precision="fp64", chi=0.9, kappa=6.0)
    t, m, pos = _setup(B, spec, lb=0.0)
    f, e = t.compute()
    assert e["elec"] == 0.0
    assert _rel(f, O.forces(m, pos)) < 1e-12  # l_B = 0: no electrostatics
    for bad in ((1.0, -1.0, -1.0, 0.5), (1.0, -1.0, 1.0, 0.0), (np.nan, 0.0, 1.0, 0.5)):
        with pytest.raises(B.TildError, match="EINVAL"):
            t.set_electrostatics(*bad)


def test_batch_with_charged_replicas_matches_individual_bitwise(B):
    specs = [I.small_system(n_chains=nc, N=10, n_a=5, L=L, n=n, precision="fp32", chi=0.5, kappa=8.0, seed=sd)
             for nc, L, n, sd in ((60, 8.0, 16, 41), (90, 12.0, 24, 42))]

    def make():
        out = []
        for i, s in enumerate(specs):
            t, _, _ = _setup(B, s, q=(1.0, -1.0 + 0.5 * i), sort_every=5)
            t.init_velocities()
            out.append(t)
        return out

    batch, alone = make(), make()
    with B.TildBatch(batch) as bt:
        bt.step(17)
        bt.synchronize()
    for t in alone:
        t.step(17)
        t.synchronize()
    for tb, ta in zip(batch, alone):
        assert np.array_equal(tb.positions(), ta.positions())
