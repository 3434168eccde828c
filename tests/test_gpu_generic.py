"""Odd grid sizes and two-dimensional boxes through the C ABI, against the
FP64 oracle (Sec. "TILD Branch": 2D or 3D periodic boxes; Listing infile:
"Dim 2", a 65 x 65 grid, pmeorder 1, GJF, dt 0.005, Gaussian pair styles).

Grids outside the tiled kernels' sizes run on the any-size kernels (line
transforms in two factors n = n1 n2 with direct DFTs, one thread per bead).
Tolerances as in the parity tests: forces 1e-5 (FP32) / 1e-12 (FP64)
norm-wise, energies 1e-6 / 1e-10 relative per term, 10-step trajectories
1e-4 L (FP32) / 1e-9 (FP64).
"""
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
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


FTOL = {"fp32": 1e-5, "fp64": 1e-12}
ETOL = {"fp32": 1e-6, "fp64": 1e-10}


def _ctx(B, moltypes, L, n, order, prec, chi, kappa, a, seed, dim, pos, dt=0.005):
    t = B.Tild(L, n, order, prec, seed, dim=dim)
    t.set_chains([(m.n_chains, m.N, m.n_a) for m in moltypes], 1.0)
    t.set_interactions(chi, kappa, a)
    t.set_integrator(dt, 1.0, 1.0, 1.0)
    t.set_positions(pos)
    sp = I.species_of_beads(moltypes).astype(np.int64)
    m = O.Model(L=L, n=n, P=order + 1, species=sp, n_species=2, bonds=I.bond_pairs(moltypes).astype(np.int64), b=1.0,
                chi=np.array([[0.0, chi], [chi, 0.0]]), kappa=kappa, a=a, dt=dt, seed=seed, dim=dim)
    return t, m


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,order", [(15, 1), (21, 2), (25, 3), (45, 4), (65, 1), (20, 1), (36, 2)])
def test_3d_any_grid_size_forces_energies_density(B, prec, n, order):
    mt = (I.MolType(120, 10, 4),)
    L = 0.5 * n
    pos = I.random_walk_positions(mt, L, 1.0, 40 + n)
    if prec == "fp32":
        pos = pos.astype(np.float32).astype(np.float64)
    t, m = _ctx(B, mt, L, n, order, prec, 1.1, 6.0, 0.5, 3, 3, pos)
    f, e = t.compute()
    assert _rel(f, O.forces(m, pos)) < FTOL[prec]
    eref = O.energies(m, pos)
    for k in ("bond", "chi", "kappa"):
        assert abs(e[k] - eref[k]) <= ETOL[prec] * max(1.0, abs(eref[k])), (k, e[k], eref[k])
    rho = t.density()
    ref = O.spread(m, pos).transpose(0, 3, 2, 1)
    assert np.abs(rho - ref).max() <= (1e-12 if prec == "fp64" else 2e-6) * np.abs(ref).max()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_3d_odd_grid_trajectory(B, prec):
    mt = (I.MolType(80, 12, 5),)
    n, L = 27, 13.5
    pos = I.random_walk_positions(mt, L, 1.0, 71)
    if prec == "fp32":
        pos = pos.astype(np.float32).astype(np.float64)
    t, m = _ctx(B, mt, L, n, 1, prec, 0.9, 8.0, 0.5, 5, 3, pos)
    t.init_velocities()
    t.step(10)
    t.synchronize()
    st = O.run(m, O.initial_state(m, pos), 10)
    d = O.minimum_image(t.positions() - st.pos, L)
    assert np.abs(d).max() < (1e-4 * L if prec == "fp32" else 1e-9)


def _listing_2d(prec):
    """Listing infile's setting: D = 2, 65 x 65 grid, pmeorder 1, GJF with
    dt 0.005. Pair amplitudes 1.5625 (like species) and 3.0 (unlike) map to
    eps_KK = kappa / rho_0 and eps_AB = (chi + kappa) / rho_0 (Eqs. fh,
    HelfandP): kappa = 1.5625 rho_0, chi = 1.4375 rho_0; smearing a = 0.5
    (the listing's width parameter is not labelled). The data file is not
    given: 250 A10-B10 chains in a 32.5 x 32.5 box (dx = 0.5), 2D random
    walks from a seed."""
    mt = (I.MolType(250, 20, 10),)
    L, n = 32.5, 65
    rho0 = 250 * 20 / L ** 2
    pos = I.random_walk_positions_2d(mt, L, 1.0, 2302)
    if prec == "fp32":
        pos = pos.astype(np.float32).astype(np.float64)
    return mt, L, n, 1.4375 * rho0, 1.5625 * rho0, pos


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_2d_listing_setting_forces_energies_trajectory(B, prec):
    mt, L, n, chi, kappa, pos = _listing_2d(prec)
    t, m = _ctx(B, mt, L, n, 1, prec, chi, kappa, 0.5, 11, 2, pos)
    p2 = pos[:, :2]
    f, e = t.compute()
    fref = O.forces(m, p2)
    assert np.abs(f[:, 2]).max() == 0.0
    assert _rel(f[:, :2], fref) < FTOL[prec]
    eref = O.energies(m, p2)
    for k in ("bond", "chi", "kappa"):
        assert abs(e[k] - eref[k]) <= ETOL[prec] * max(1.0, abs(eref[k])), (k, e[k], eref[k])
    rho = t.density()
    assert rho.shape == (2, 1, n, n)
    ref = O.spread(m, p2).transpose(0, 2, 1)[:, None]
    assert np.abs(rho - ref).max() <= (1e-12 if prec == "fp64" else 2e-6) * np.abs(ref).max()
    t.init_velocities()
    t.step(10)
    t.synchronize()
    st = O.run(m, O.initial_state(m, p2), 10)
    r = t.positions()
    assert np.abs(r[:, 2]).max() == 0.0
    d = O.minimum_image(r[:, :2] - st.pos, L)
    assert np.abs(d).max() < (1e-4 * L if prec == "fp32" else 1e-9)
    v = t.velocities()
    assert np.abs(v[:, 2]).max() == 0.0
    assert _rel(v[:, :2], st.vel) < (1e-4 if prec == "fp32" else 1e-9)


def test_2d_orders_and_even_grid(B):
    mt = (I.MolType(60, 10, 5),)
    for n, order in ((32, 2), (33, 3), (40, 4)):
        L = 0.45 * n
        pos = I.random_walk_positions_2d(mt, L, 1.0, n)
        t, m = _ctx(B, mt, L, n, order, "fp64", 1.3, 5.0, 0.6, 2, 2, pos)
        f, _ = t.compute()
        assert _rel(f[:, :2], O.forces(m, pos[:, :2])) < 1e-12


def test_2d_three_species_rings(B):
    topo = I.ring_star_system(8, 10, 5, 3, 4, 10, 8, L=12.0, n_species=3, seed=5)
    pos = topo.positions.copy()
    pos[:, 2] = 0.0
    L, n = 12.0, 25
    t = B.Tild(L, n, 1, "fp64", 4, dim=2)
    t.set_chains([(1, len(topo.species), 0)], 1.0)
    t.set_species(3, topo.species)
    t.set_bonds(topo.bonds)
    chi = np.array([[0.0, 1.0, 0.5], [1.0, 0.0, 0.7], [0.5, 0.7, 0.0]])
    t.set_interactions(1.0, 4.0, 0.5)
    t.set_chi_matrix(chi)
    t.set_positions(pos)
    m = O.Model(L=L, n=n, P=2, species=topo.species.astype(np.int64), n_species=3, bonds=topo.bonds.astype(np.int64),
                b=1.0, chi=chi, kappa=4.0, a=0.5, dim=2)
    f, e = t.compute()
    assert _rel(f[:, :2], O.forces(m, pos[:, :2])) < 1e-12
    eref = O.energies(m, pos[:, :2])
    for k in ("bond", "chi", "kappa"):
        assert abs(e[k] - eref[k]) <= 1e-10 * max(1.0, abs(eref[k]))


def test_any_size_grids_reject_what_they_do_not_implement(B):
    t = B.Tild(10.0, 25, 1, "fp64", 1)
    t.set_chains([(10, 10, 5)], 1.0)
    with pytest.raises(B.TildError) as ei:
        t.set_force_method("analytic")
    assert ei.value.status == B.TILD_EUNSUPPORTED
    with pytest.raises(B.TildError) as ei:
        t.set_electrostatics(1.0, -1.0, 1.0, 0.5)
    assert ei.value.status == B.TILD_EUNSUPPORTED
    t.set_positions(I.random_walk_positions((I.MolType(10, 10, 5),), 10.0, 1.0, 1))
    with pytest.raises(B.TildError) as ei:
        t.energy_gradient()
    assert ei.value.status == B.TILD_EUNSUPPORTED
