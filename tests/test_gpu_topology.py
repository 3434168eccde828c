"""General topologies and more species through the C ABI, against the FP64
oracle: explicit bond lists (rings, stars with three bonds at a bead),
per-bead species (three and four species with a Flory matrix, Eq. fh over
every pair), SoA layout of the per-bead arrays, and the caller's device
allocator.

Tolerances as in the parity tests: forces 1e-5 (FP32) / 1e-12 (FP64)
norm-wise; energies 1e-6 / 1e-10 relative per term; 3-step trajectories
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


def _chi_matrix(S):
    chi = np.zeros((S, S))
    vals = [1.1, 0.4, -0.3, 0.8, 0.25, 0.6]
    k = 0
    for i in range(S):
        for j in range(i + 1, S):
            chi[i, j] = chi[j, i] = vals[k]
            k += 1
    return chi


def _system(B, topo, L, n, pmeorder, prec, kappa=6.0, a=0.5, seed=3):
    pos = topo.positions
    if prec == "fp32":
        pos = pos.astype(np.float32).astype(np.float64)
    N = len(topo.species)
    t = B.Tild(L, n, pmeorder, prec, seed)
    t.set_chains([(1, N, N)], 1.0)
    t.set_species(topo.n_species, topo.species)
    t.set_bonds(topo.bonds)
    chi = _chi_matrix(topo.n_species)
    t.set_interactions(chi[0, 1] if topo.n_species > 1 else 0.0, kappa, a)
    if topo.n_species > 2:
        t.set_chi_matrix(chi)
    t.set_positions(pos)
    m = O.Model(L=L, n=n, P=pmeorder + 1, species=topo.species.astype(np.int64), n_species=topo.n_species,
                bonds=topo.bonds.astype(np.int64), b=1.0, chi=chi, kappa=kappa, a=a, seed=seed)
    return t, m, pos


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("S", [2, 3, 4])
@pytest.mark.parametrize("order", [1, 2])
def test_rings_stars_species_forces_energies_density(B, prec, S, order):
    topo = I.ring_star_system(6, 12, 5, 3, 6, 8, 10, L=9.0, n_species=S, seed=10 + S)
    t, m, pos = _system(B, topo, 9.0, 24, order, prec)
    f, e = t.compute()
    ref = O.forces(m, pos)
    assert _rel(f, ref) < FTOL[prec]
    eref = O.energies(m, pos)
    for k in ("bond", "chi", "kappa"):
        assert abs(e[k] - eref[k]) <= ETOL[prec] * max(1.0, abs(eref[k])), (k, e[k], eref[k])
    rho = t.density()
    rref = O.spread(m, pos).transpose(0, 3, 2, 1)
    assert rho.shape == rref.shape
    assert np.abs(rho - rref).max() <= (1e-12 if prec == "fp64" else 2e-6) * np.abs(rref).max()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_three_species_trajectory_matches_oracle(B, prec):
    topo = I.ring_star_system(5, 10, 4, 3, 5, 6, 12, L=8.0, n_species=3, seed=31)
    t, m, pos = _system(B, topo, 8.0, 16, 1, prec)
    t.init_velocities()
    t.step(3)
    t.synchronize()
    st = O.run(m, O.initial_state(m, pos), 3)
    d = O.minimum_image(t.positions() - st.pos, 8.0)
    assert np.abs(d).max() < (1e-4 * 8.0 if prec == "fp32" else 1e-9)
    assert _rel(t.velocities(), st.vel) < (1e-4 if prec == "fp32" else 1e-9)


def test_explicit_linear_bonds_equal_the_chains_bitwise(B):
    """The chains' own bonds given as a list (any order) reproduce the
    implicit chain topology bit for bit: forces, positions and velocities."""
    spec = I.small_system(n_chains=60, N=10, n_a=4, L=7.0, n=16, precision="fp32")
    pos = I.initial_positions(spec).astype(np.float32).astype(np.float64)
    out = []
    for explicit in (False, True):
        t = B.Tild.from_spec(spec, sort_every=3)
        if explicit:
            bonds = I.bond_pairs(spec.moltypes)[::-1][:, ::-1]
            t.set_bonds(bonds)
        t.set_positions(pos)
        t.init_velocities()
        f, e = t.compute()
        t.step(7)
        out.append((f, t.positions(), t.velocities(), e["bond"]))
    for a, b in zip(out[0][:3], out[1][:3]):
        assert np.array_equal(np.asarray(a), np.asarray(b))
    # FP64 energy sums follow the slot order inside a tile, which re-binning
    # does not fix: equal to rounding
    assert out[0][3] == pytest.approx(out[1][3], rel=1e-13)


def test_species_pattern_none_keeps_chain_species_and_one_species(B):
    spec = I.small_system(n_chains=40, N=8, n_a=3, L=6.0, n=16, precision="fp64", chi=0.0)
    pos = I.initial_positions(spec)
    t = B.Tild.from_spec(spec)
    t.set_positions(pos)
    f2, _ = t.compute()
    # one species: every bead species 0; with chi = 0 the field force is the same
    t.set_species(1, np.zeros(spec.n_beads, np.int32))
    f1, e1 = t.compute()
    assert t.density().shape == (1, 16, 16, 16)
    assert _rel(f1, f2) < 1e-12
    assert e1["chi"] == 0.0
    with pytest.raises(B.TildError):
        t.set_species(3, None)
    with pytest.raises(B.TildError):
        t.set_species(2, np.full(spec.n_beads, 2, np.int32))


def test_bond_list_validation(B):
    spec = I.small_system(n_chains=4, N=5, n_a=2, L=6.0, n=16, precision="fp64")
    t = B.Tild.from_spec(spec)
    for bad in ([[0, 0]], [[0, 1], [1, 0]], [[0, 20]], [[-1, 2]]):
        with pytest.raises(B.TildError) as ei:
            t.set_bonds(bad)
        assert ei.value.status == B.TILD_EINVAL
    t.set_bonds(np.zeros((0, 2), np.int32))  # no bonds at all
    t.set_positions(I.initial_positions(spec))
    _, e = t.compute()
    assert e["bond"] == 0.0


def test_more_than_two_species_reject_unsupported_paths(B):
    topo = I.ring_star_system(2, 8, 2, 3, 4, 2, 8, L=6.0, n_species=3, seed=4)
    t, m, pos = _system(B, topo, 6.0, 16, 1, "fp64")
    with pytest.raises(B.TildError) as ei:
        t.energy_gradient()
    assert ei.value.status == B.TILD_EUNSUPPORTED
    with pytest.raises(B.TildError) as ei:
        t.set_electrostatics(1.0, -1.0, 1.0, 0.5)
    assert ei.value.status == B.TILD_EUNSUPPORTED


@pytest.mark.parametrize("where", ["host", "device"])
def test_soa_layout_matches_aos(B, where):
    import torch

    spec = I.small_system(n_chains=50, N=10, n_a=4, L=7.0, n=16, precision="fp64")
    pos = I.initial_positions(spec)
    ref = B.Tild.from_spec(spec)
    ref.set_positions(pos)
    ref.init_velocities()
    f_ref, _ = ref.compute()
    ref.step(4)
    r_ref, v_ref = ref.positions(), ref.velocities()

    t = B.Tild.from_spec(spec)
    t.set_layout("soa")
    soa = np.ascontiguousarray(pos.T)
    t.set_positions(torch.from_numpy(soa).cuda() if where == "device" else soa)
    t.init_velocities()
    if where == "device":
        f = torch.empty(3 * spec.n_beads, dtype=torch.float64, device="cuda")
        t.compute(out=f)
        f = f.cpu().numpy().reshape(3, -1)
    else:
        f, _ = t.compute()
    assert f.shape == (3, spec.n_beads)
    assert np.array_equal(f.T, f_ref)
    t.step(4)
    assert np.array_equal(t.positions().T, r_ref)
    assert np.array_equal(t.velocities().T, v_ref)
    assert t.lib.tild_set_layout(t.ctx, 7) == B.TILD_EINVAL


def test_torch_allocator_routes_every_allocation_and_frees_them(B):
    import torch

    spec = I.small_system(n_chains=50, N=10, n_a=4, L=7.0, n=16, precision="fp32")
    pos = I.initial_positions(spec).astype(np.float32).astype(np.float64)
    plain = B.Tild.from_spec(spec)
    plain.set_positions(pos)
    plain.init_velocities()
    plain.step(5)
    r_plain = plain.positions()
    plain.close()

    alloc = B.TorchAllocator(torch.cuda.current_device())
    t = B.Tild(spec.L, spec.n, spec.pmeorder, spec.precision, spec.dyn_seed, allocator=alloc)
    t.set_chains([(m.n_chains, m.N, m.n_a) for m in spec.moltypes], spec.b)
    t.set_interactions(spec.chi, spec.kappa, spec.a)
    t.set_positions(pos)
    t.init_velocities()
    t.step(5)
    assert np.array_equal(t.positions(), r_plain)
    grids = 2 * spec.n ** 3 * 8  # at least the fixed-point density
    assert alloc.n_alloc > 0 and alloc.live_bytes > grids
    t.close()
    assert alloc.live_bytes == 0


def test_allocator_failure_returns_enomem(B):
    """A refused allocation gives TILD_ENOMEM at create (early or late in its
    allocations) or at set_chains, and every block handed out is returned."""
    import torch

    for k in (0, 3, 14):
        alloc = B.TorchAllocator(torch.cuda.current_device())
        alloc.fail_after = k
        t = None
        with pytest.raises(B.TildError) as ei:
            t = B.Tild(6.0, 16, 1, "fp32", 1, allocator=alloc)
            t.set_chains([(20, 10, 4)], 1.0)
        assert ei.value.status == B.TILD_ENOMEM
        if t is not None:
            t.close()
        assert alloc.live_bytes == 0
