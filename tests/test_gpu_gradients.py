"""Differentiable form: energy gradients through the C ABI and torch.autograd.

dU/dchi, dU/dkappa and dU/da are checked against central differences of the
oracle energy; dU/dr against the oracle's analytic-differentiation forces
(the exact gradient of the gridded energy) and against central differences
of the GPU energy itself."""
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


def _etot(m, pos):
    e = O.energies(m, pos)
    return e["bond"] + e["chi"] + e["kappa"]


@pytest.mark.parametrize("order", [1, 3])
def test_parameter_gradients_match_oracle_finite_differences(B, order):
    spec = I.small_system(n_chains=60, N=10, n_a=4, L=7.0, n=16, pmeorder=order, precision="fp64", chi=1.4,
                          kappa=6.0, a=0.55)
    pos = I.initial_positions(spec)
    m = O.model_from_spec(spec, I.species_of_beads(spec.moltypes), I.bond_pairs(spec.moltypes))
    with B.Tild.from_spec(spec) as t:
        t.set_positions(pos)
        g, _ = t.energy_gradient(with_positions=False)
    assert g["energy"] == pytest.approx(_etot(m, pos), rel=1e-10)
    h = 1e-5
    for name, attr in (("dU_dchi", "chi"), ("dU_dkappa", "kappa"), ("dU_da", "a")):
        mp, mm = O.Model(**{**m.__dict__}), O.Model(**{**m.__dict__})
        if attr == "chi":
            mp.chi = m.chi * (1 + h / m.chi[0, 1])
            mm.chi = m.chi * (1 - h / m.chi[0, 1])
        else:
            setattr(mp, attr, getattr(m, attr) + h)
            setattr(mm, attr, getattr(m, attr) - h)
        fd = (_etot(mp, pos) - _etot(mm, pos)) / (2 * h)
        assert g[name] == pytest.approx(fd, rel=1e-7), name


@pytest.mark.parametrize("prec,order", [("fp64", 1), ("fp64", 2), ("fp64", 4), ("fp32", 1)])
def test_position_adjoint_matches_oracle_analytic_gradient(B, prec, order):
    spec = I.small_system(n_chains=70, N=10, n_a=4, L=8.0, n=16, pmeorder=order, precision=prec, chi=1.2, kappa=7.0)
    pos = I.initial_positions(spec)
    if prec == "fp32":
        pos = pos.astype(np.float32).astype(np.float64)
    m = O.model_from_spec(spec, I.species_of_beads(spec.moltypes), I.bond_pairs(spec.moltypes))
    with B.Tild.from_spec(spec) as t:
        t.set_positions(pos)
        _, dudr = t.energy_gradient()
    ref = -O.forces(m, pos, variant="analytic")
    assert _rel(dudr, ref) < (1e-12 if prec == "fp64" else 1e-5)


def test_autograd_function_against_energy_differences(B):
    import torch

    from paper_2302_02474_gb300.autograd import tild_energy

    spec = I.small_system(n_chains=30, N=8, n_a=3, L=6.0, n=16, precision="fp64", chi=1.1, kappa=5.0)
    pos0 = torch.tensor(I.initial_positions(spec), dtype=torch.float64, device="cuda")
    with B.Tild.from_spec(spec) as t:
        pos = pos0.clone().requires_grad_(True)
        chi = torch.tensor(1.1, dtype=torch.float64, requires_grad=True)
        kappa = torch.tensor(5.0, dtype=torch.float64, requires_grad=True)
        a = torch.tensor(0.5, dtype=torch.float64, requires_grad=True)
        U = tild_energy(t, pos, chi, kappa, a)
        U.backward()
        h = 1e-5
        for idx in [(0, 0), (17, 2), (101, 1), (239, 0)]:
            pp, pm = pos0.clone(), pos0.clone()
            pp[idx] += h
            pm[idx] -= h
            fd = (tild_energy(t, pp, 1.1, 5.0, 0.5) - tild_energy(t, pm, 1.1, 5.0, 0.5)).item() / (2 * h)
            assert pos.grad[idx].item() == pytest.approx(fd, rel=1e-6, abs=1e-6)
        fd_chi = (tild_energy(t, pos0, 1.1 + h, 5.0, 0.5) - tild_energy(t, pos0, 1.1 - h, 5.0, 0.5)).item() / (2 * h)
        fd_a = (tild_energy(t, pos0, 1.1, 5.0, 0.5 + h) - tild_energy(t, pos0, 1.1, 5.0, 0.5 - h)).item() / (2 * h)
        assert chi.grad.item() == pytest.approx(fd_chi, rel=1e-6)
        assert a.grad.item() == pytest.approx(fd_a, rel=1e-6)
