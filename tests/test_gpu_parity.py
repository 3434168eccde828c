"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (norm-wise relative errors ||x_gpu - x_ref|| / ||x_ref||):
forces 1e-5 in FP32 and 1e-12 in FP64; energies 1e-6 relative per term
(1e-10 in FP64); 10-step trajectories within 1e-4 L (FP32). FP32 runs
feed the oracle the same FP32-rounded positions the GPU holds.
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


def _setup(B, spec, sort_every=0, pos=None):
    if pos is None:
        pos = I.initial_positions(spec)
    if spec.precision == "fp32":
        pos = pos.astype(np.float32).astype(np.float64)
    t = B.Tild.from_spec(spec, sort_every=sort_every)
    t.set_positions(pos)
    m = O.model_from_spec(spec, I.species_of_beads(spec.moltypes), I.bond_pairs(spec.moltypes))
    return t, m, pos


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


FTOL = {"fp32": 1e-5, "fp64": 1e-12}


# ----------------------------------------------------------- density


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_density_matches_oracle(B, prec, order):
    spec = I.small_system(n_chains=53, N=9, n_a=4, L=7.0, n=16, pmeorder=order, precision=prec)
    t, m, pos = _setup(B, spec)
    rho = t.density()
    ref = O.spread(m, pos).transpose(0, 3, 2, 1)  # -> [K][z][y][x]
    tol = 1e-12 if prec == "fp64" else 2e-6
    assert np.abs(rho - ref).max() <= tol * np.abs(ref).max()
    dV = (spec.L / spec.n) ** 3
    sp = I.species_of_beads(spec.moltypes)
    mass_tol = 1e-9 if prec == "fp64" else 1e-6  # FP32 weights sum to 1 within ~1e-7 per bead
    for K in range(2):
        assert abs(rho[K].sum() * dV - np.sum(sp == K)) < mass_tol * len(sp)


def test_density_bit_identical_for_any_bead_order(B):
    """Fixed-point accumulation: the grid is the same bits whatever the order
    in which beads are listed or binned."""
    spec = I.small_system(n_chains=200, N=8, n_a=3, L=10.0, n=32, precision="fp32")
    pos = I.initial_positions(spec).astype(np.float32).astype(np.float64)
    t1 = B.Tild.from_spec(spec, sort_every=5)
    t1.set_positions(pos)
    d1 = t1.density(dtype=np.float64)
    perm = np.random.default_rng(0).permutation(200)
    pos2 = pos.reshape(200, 8, 3)[perm].reshape(-1, 3)
    t2 = B.Tild.from_spec(spec, sort_every=1000)
    t2.set_positions(pos2)
    d2 = t2.density(dtype=np.float64)
    assert np.array_equal(d1, d2)
    t1.set_positions(pos)
    assert np.array_equal(d1, t1.density(dtype=np.float64))


# ------------------------------------------------------ spectrum / fields


@pytest.mark.parametrize("prec,n", [("fp64", 8), ("fp64", 32), ("fp32", 16), ("fp32", 64), ("fp64", 128),
                                    ("fp64", 24), ("fp32", 40), ("fp64", 48), ("fp32", 80)])
def test_spectrum_matches_oracle_dft(B, prec, n):
    spec = I.small_system(n_chains=60, N=10, n_a=4, L=n / 2.0, n=n, precision=prec)
    t, m, pos = _setup(B, spec)
    Z = t.spectrum()
    rho = O.spread(m, pos).transpose(0, 3, 2, 1)
    ref = np.fft.fftn(rho[0] + 1j * rho[1])
    assert _rel(Z, ref) < (1e-13 if prec == "fp64" else 2e-6)


@pytest.mark.parametrize("prec,n,order", [("fp64", 16, 1), ("fp64", 32, 3), ("fp32", 32, 1), ("fp32", 64, 2)])
def test_field_gradient_matches_oracle(B, prec, n, order):
    spec = I.small_system(n_chains=80, N=10, n_a=4, L=n / 2.0, n=n, pmeorder=order, precision=prec)
    t, m, pos = _setup(B, spec)
    g = t.field_gradient()  # [d][z][y][x][K]
    ref = O.potential_fields(m, O.spread(m, pos))["grad_w"]  # [K][d][x][y][z]
    ref = ref.transpose(1, 4, 3, 2, 0)
    assert _rel(g, ref) < (1e-12 if prec == "fp64" else 3e-6)


# ----------------------------------------------------------- forces


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_forces_and_energies_match_oracle(B, prec, order):
    spec = I.small_system(n_chains=71, N=11, n_a=5, L=8.0, n=16, pmeorder=order, precision=prec, chi=1.5,
                          kappa=9.0)
    t, m, pos = _setup(B, spec)
    t.init_velocities()
    f, e = t.compute()
    ref = O.forces(m, pos)
    assert _rel(f, ref) < FTOL[prec]
    eref = O.energies(m, pos)
    etol = 1e-10 if prec == "fp64" else 1e-6
    for k in ("bond", "chi", "kappa"):
        assert abs(e[k] - eref[k]) <= etol * abs(eref[k]), (k, e[k], eref[k])
    assert np.abs(e["net_force"]).max() < 1e-6 * np.abs(f).sum()


@pytest.mark.parametrize("prec,n,order", [("fp64", 24, 1), ("fp64", 40, 2), ("fp32", 48, 1), ("fp64", 80, 3)])
def test_mixed_radix_grids_forces_and_trajectory(B, prec, n, order):
    """5-smooth grids (radix-3 and radix-5 FFT passes): forces, energies and
    a 5-step trajectory against the oracle."""
    spec = I.small_system(n_chains=90, N=10, n_a=4, L=n / 2.5, n=n, pmeorder=order, precision=prec, chi=1.3,
                          kappa=8.0)
    t, m, pos = _setup(B, spec, sort_every=3)
    t.init_velocities()
    f, e = t.compute()
    assert _rel(f, O.forces(m, pos)) < FTOL[prec]
    eref = O.energies(m, pos)
    for k in ("chi", "kappa"):
        assert abs(e[k] - eref[k]) <= (1e-10 if prec == "fp64" else 1e-6) * abs(eref[k])
    t.step(5)
    st = O.run(m, O.initial_state(m, pos), 5)
    d = O.minimum_image(t.positions() - st.pos, m.L)
    assert np.abs(d).max() < (1e-10 if prec == "fp64" else 1e-4 * m.L)


def test_homogeneous_melt_zero_field_force(B):
    L, n = 4.0, 8
    g = np.stack(np.meshgrid(*[np.arange(n) * (L / n)] * 3, indexing="ij"), axis=-1).reshape(-1, 3)
    t = B.Tild(L, n, 1, "fp64", 1)
    # A and B monomers (N = 1 chains): one of each on every node
    t.set_chains([(len(g), 1, 1), (len(g), 1, 0)], 1.0)
    t.set_interactions(2.0, 5.0, 0.5)
    t.set_positions(np.concatenate([g, g]))
    f, e = t.compute()
    assert np.abs(f).max() < 1e-11
    assert abs(e["kappa"]) < 1e-9


def test_single_species_and_single_chain(B):
    spec = I.SystemSpec("homo", (I.MolType(1, 37, 37),), 5.0, 16, 2, 0.5, 0.0, 4.0, 0.005, 1.0, 1.0, 1.0, 1.0,
                        10, "fp64", 3, 4)
    t, m, pos = _setup(B, spec)
    t.init_velocities()
    f, e = t.compute()
    assert _rel(f, O.forces(m, pos)) < 1e-12
    spec_b = spec.with_(moltypes=(I.MolType(1, 37, 0),))
    t2, m2, pos2 = _setup(B, spec_b, pos=pos)
    f2, _ = t2.compute()
    assert _rel(f2, O.forces(m2, pos2)) < 1e-12


def test_single_bead_and_wrap_at_box_edge(B):
    t = B.Tild(6.0, 8, 1, "fp64", 9)
    t.set_chains([(2, 1, 1)], 1.0)
    t.set_interactions(0.0, 3.0, 0.5)
    # x exactly at L (wraps to 0); the second bead 1e-14 below 0 in x (wraps to
    # just below L) and 1e-9 below L in y, so it spreads across the x and y
    # faces; its z = 2L + 0.7 wraps to 0.7, 2.3 from the first bead, which
    # gives an O(1) force along z (with z = 0 the reference force is ~1e-10
    # and a relative tolerance is meaningless)
    pos = np.array([[6.0, 0.0, 3.0], [-1e-14, 5.999999999, 12.7]])
    t.set_positions(pos)
    r = t.positions()
    assert np.all(r >= 0) and np.all(r < 6.0)
    m = O.Model(L=6.0, n=8, P=2, species=np.array([0, 0]), n_species=1, bonds=np.zeros((0, 2), np.int64), b=1.0,
                chi=np.zeros((1, 1)), kappa=3.0, a=0.5)
    f, _ = t.compute()
    assert _rel(f, O.forces(m, pos)) < 1e-12


# ------------------------------------------------------- trajectories


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ten_step_trajectory_matches_oracle(B, prec):
    spec = I.small_system(n_chains=97, N=10, n_a=4, L=9.0, n=16, precision=prec, chi=1.2, kappa=8.0)
    t, m, pos = _setup(B, spec, sort_every=4)
    t.init_velocities()
    t.step(10)
    t.synchronize()
    r, v = t.positions(), t.velocities()
    st = O.run(m, O.initial_state(m, pos), 10)
    d = O.minimum_image(r - st.pos, m.L)
    if prec == "fp64":
        assert np.abs(d).max() < 1e-10
        assert _rel(v, st.vel) < 1e-10
    else:
        assert np.abs(d).max() < 1e-4 * m.L
        assert _rel(v, st.vel) < 1e-4
    assert t.step_count() == 10


def test_trajectory_independent_of_binning_and_graphs(B):
    """Same bits whatever the re-binning period or launch grouping."""
    spec = I.small_system(n_chains=150, N=10, n_a=4, L=10.0, n=32, precision="fp32")
    outs = []
    for sort_every, chunks in ((3, [45]), (1000, [45]), (5, [1] * 45), (2, [7, 30, 8])):
        t, m, pos = _setup(B, spec, sort_every=sort_every)
        t.init_velocities()
        for c in chunks:
            t.step(c)
        outs.append(t.positions())
    for o in outs[1:]:
        assert np.array_equal(outs[0], o)


@pytest.mark.parametrize("prec,n_chains", [("fp32", 480), ("fp32", 1000), ("fp64", 480)])
def test_trajectory_independent_of_binning_crowded_tiles(B, prec, n_chains):
    """Crowded tiles (600 or 1250 beads on each of 8 tiles: several staging
    chunks, and above 1023 beads the tile spreads through global memory),
    large steps and rare re-binning, so that more beads leave their tile's
    patch, and more bonded neighbours lie outside the staged chunk, than the
    per-chunk lists of the bead kernel hold: the overflow paths must give the
    same bits as frequent re-binning."""
    spec = I.small_system(n_chains=n_chains, N=10, n_a=4, L=8.0, n=16, precision=prec, chi=1.0, kappa=5.0)
    spec = spec.with_(dt=0.02, kT=2.0)
    outs = []
    for sort_every in (2, 100000):
        t, m, pos = _setup(B, spec, sort_every=sort_every)
        t.init_velocities()
        t.step(30)
        outs.append(t.positions())
    assert np.array_equal(outs[0], outs[1])
    # beads moved by more than a cell (many of those near a tile face left it)
    assert np.abs(O.minimum_image(outs[1] - pos, spec.L)).max() > spec.L / spec.n


def test_beads_escaping_their_tile_patch(B):
    """Large steps and no re-binning: beads leave the shared-memory patch of
    their tile and are spread through the global fallback; results still
    match the oracle."""
    spec = I.small_system(n_chains=60, N=8, n_a=4, L=8.0, n=16, precision="fp64", chi=1.0, kappa=5.0)
    spec = spec.with_(dt=0.05, kT=2.0)
    t, m, pos = _setup(B, spec, sort_every=100000)
    t.init_velocities()
    t.step(40)
    r = t.positions()
    st = O.run(m, O.initial_state(m, pos), 40)
    assert np.abs(O.minimum_image(r - st.pos, m.L)).max() < 1e-9
    # beads did move by more than a tile margin
    assert np.abs(O.minimum_image(r - pos, m.L)).max() > 2 * spec.L / spec.n


def test_checkpoint_resume_bit_identical(B):
    spec = I.small_system(n_chains=80, N=10, n_a=4, L=8.0, n=16, precision="fp32")
    t, m, pos = _setup(B, spec, sort_every=3)
    t.init_velocities()
    t.step(7)
    blob = t.get_state()
    t.step(11)
    a = t.positions()
    t2, _, _ = _setup(B, spec, sort_every=5)
    t2.set_state(blob)
    assert t2.step_count() == 7
    t2.step(11)
    assert np.array_equal(a, t2.positions())


def test_parameter_change_keeps_velocity(B):
    spec = I.small_system(n_chains=40, N=10, n_a=4, L=6.0, n=16, precision="fp64")
    t, m, pos = _setup(B, spec)
    t.init_velocities()
    t.step(3)
    v0 = t.velocities()
    t.set_interactions(2.5, 11.0, 0.6)
    assert _rel(t.velocities(), v0) < 1e-13
    t.set_integrator(0.01, 0.5, 1.3, 1.0)
    assert _rel(t.velocities(), v0) < 1e-13


def test_device_buffers_and_fp32_io(B):
    import torch

    spec = I.small_system(n_chains=50, N=10, n_a=4, L=7.0, n=16, precision="fp32")
    pos = I.initial_positions(spec).astype(np.float32)
    t = B.Tild.from_spec(spec)
    t.set_positions(torch.from_numpy(pos).cuda())
    t.init_velocities()
    out = torch.empty(3 * spec.n_beads, dtype=torch.float32, device="cuda")
    t.positions(out=out)
    assert np.array_equal(out.cpu().numpy().reshape(-1, 3), O.wrap(pos.astype(np.float64), spec.L).astype(np.float32))
    f_dev = torch.empty(3 * spec.n_beads, dtype=torch.float64, device="cuda")
    f_host, _ = t.compute()
    t.compute(out=f_dev)
    assert np.allclose(f_dev.cpu().numpy().reshape(-1, 3), f_host, rtol=0, atol=0)


def test_invalid_calls_return_errors(B):
    t = B.Tild(6.0, 16, 1, "fp32", 0)
    with pytest.raises(B.TildError, match="ESTATE"):
        t.step(1)
    with pytest.raises(B.TildError, match="ESTATE"):
        t.set_positions(np.zeros((0, 3)))
    t.set_chains([(2, 3, 1)], 1.0)
    with pytest.raises(B.TildError, match="ESTATE"):
        t.compute()
    with pytest.raises(B.TildError, match="EINVAL"):
        t.set_interactions(1.0, -1.0, 0.5)
    with pytest.raises(ValueError):
        t.set_positions(np.zeros((5, 3)))
    # a non-finite coordinate is reported; the context stays usable
    bad = 1.0 + 0.5 * np.arange(18, dtype=np.float64).reshape(6, 3)
    bad[2, 1] = np.nan
    bad[4, 0] = np.inf
    with pytest.raises(B.TildError, match="ENAN"):
        t.set_positions(bad)
    good = 1.0 + 0.25 * np.arange(18, dtype=np.float64).reshape(6, 3)
    t.set_positions(good)
    t.init_velocities()
    t.step(2)
    t.synchronize()
    assert np.isfinite(t.positions()).all()


# --------------------------------------------------- named workloads


def test_diblock_20k_fp64_full_config(B):
    """1,000 x A10-B10 on 32^3, FP64: forces 1e-12, energies, 10 steps."""
    spec = I.config("diblock_20k_32")
    t, m, pos = _setup(B, spec)
    t.init_velocities()
    f, e = t.compute()
    assert _rel(f, O.forces(m, pos)) < 1e-12
    eref = O.energies(m, pos)
    for k in ("bond", "chi", "kappa"):
        assert abs(e[k] - eref[k]) <= 1e-10 * abs(eref[k])
    t.step(10)
    st = O.run(m, O.initial_state(m, pos), 10)
    assert np.abs(O.minimum_image(t.positions() - st.pos, m.L)).max() < 1e-10


def _sampled_force_check(B, spec, n_sample=4000):
    t, m, pos = _setup(B, spec)
    t.init_velocities()
    f, e = t.compute()
    rho = O.spread(m, pos)
    fields = O.potential_fields(m, rho)
    which = np.random.default_rng(1).choice(m.n_beads, n_sample, replace=False)
    f_nb = -O.gather(m, pos, fields["grad_w"], which)
    f_b = O.bond_forces(m, pos)[which]
    assert _rel(f[which], f_nb + f_b) < 1e-5
    eref = O.field_energies(m, fields["rho_hat"])
    assert abs(e["chi"] - eref["chi"]) <= 1e-6 * abs(eref["chi"])
    assert abs(e["kappa"] - eref["kappa"]) <= 1e-6 * abs(eref["kappa"])
    assert abs(e["bond"] - O.bond_energy(m, pos)) <= 1e-6 * O.bond_energy(m, pos)
    assert np.abs(e["net_force"]).max() < 1e-5 * np.abs(f).sum()
    dens = t.density()
    dV = (spec.L / spec.n) ** 3
    assert abs(dens.sum() * dV - m.n_beads) < 1e-6 * m.n_beads
    return t, m, pos


def test_diblock_1p6M_128_sampled_forces(B):
    """1.6M-bead A8-B12 melt on 128^3 in FP32 (the benchmarked workload):
    forces of 4,000 sampled beads, energies, mass."""
    t, m, pos = _sampled_force_check(B, I.config("diblock_1p6M_128"))
    # a few steps run and keep the beads in the box
    t.step(25)
    t.synchronize()
    r = t.positions()
    assert np.all(np.isfinite(r)) and r.min() >= 0 and r.max() < m.L


def test_diblock_1p6M_128_steps_match_oracle(B):
    """The benchmarked FP32 step at full size (1.6M beads, 128^3): forces of
    all beads at t = 0, then 4 steps through tild_step with re-binning every
    step (so the captured re-binning cycle graph runs too), positions and
    velocities of all beads against the oracle from the same FP32-rounded
    start."""
    import json

    spec = I.config("diblock_1p6M_128")
    t, m, pos = _setup(B, spec, sort_every=1)
    rho = t.density()
    rref = O.spread(m, pos).transpose(0, 3, 2, 1)
    t.init_velocities()
    f, e = t.compute()
    st = O.initial_state(m, pos)
    eref = O.energies(m, pos)
    assert _rel(f, st.force) < 1e-5
    t.step(4)
    r, v = t.positions(), t.velocities()
    st = O.run(m, st, 4)
    dr = np.abs(O.minimum_image(r - st.pos, m.L)).max()
    assert dr < 1e-4 * m.L
    assert _rel(v, st.vel) < 1e-4
    # the FP32 path's error against the FP64 oracle on this workload
    # (printed for the design notes; run pytest with -s to see it)
    report = {"density_max_rel": float(np.abs(rho - rref).max() / np.abs(rref).max()),
              "force_normwise_rel": float(_rel(f, O.forces(m, pos))),
              "energy_rel": {k: float(abs(e[k] - eref[k]) / abs(eref[k])) for k in ("bond", "chi", "kappa")},
              "steps": 4, "position_max_over_L": float(dr / m.L), "velocity_normwise_rel": float(_rel(v, st.vel))}
    print("FP32_VS_ORACLE " + json.dumps(report))
    for k in ("bond", "chi", "kappa"):
        assert report["energy_rel"][k] < 1e-6


@pytest.mark.parametrize("n_chains", [500, 1000])
def test_dense_tiles_match_oracle(B, n_chains):
    """FP32 tiles denser than the bead kernel's staging chunk (512 beads) and,
    with 1,000 chains, denser than its 32-bit shared patches allow (1,023
    beads: those tiles spread straight into the 64-bit grid). 5,000 or
    10,000 beads on an 8^3-cell-tile grid of 2^3 tiles: density, forces,
    energies and a 5-step trajectory against the oracle."""
    spec = I.small_system(n_chains=n_chains, N=10, n_a=4, L=8.0, n=16, precision="fp32", chi=0.5, kappa=2.0,
                          seed=31)
    t, m, pos = _setup(B, spec, sort_every=2)
    tile = np.floor(pos / (spec.L / 2)).astype(int)
    per_tile = np.bincount((tile[:, 2] * 2 + tile[:, 1]) * 2 + tile[:, 0], minlength=8)
    assert per_tile.min() > (1023 if n_chains == 1000 else 512)
    rho = t.density()
    ref = O.spread(m, pos).transpose(0, 3, 2, 1)
    assert np.abs(rho - ref).max() <= 2e-6 * np.abs(ref).max()
    t.init_velocities()
    f, e = t.compute()
    assert _rel(f, O.forces(m, pos)) < 1e-5
    eref = O.energies(m, pos)
    for k in ("bond", "chi", "kappa"):
        assert abs(e[k] - eref[k]) <= 1e-6 * abs(eref[k]), (k, e[k], eref[k])
    t.step(5)
    st = O.run(m, O.initial_state(m, pos), 5)
    assert np.abs(O.minimum_image(t.positions() - st.pos, m.L)).max() < 1e-4 * m.L
    assert _rel(t.velocities(), st.vel) < 1e-4


def test_blend_6p4M_256_sampled_forces(B):
    """6.4M-bead ternary blend on 256^3 in FP32 (split xy passes)."""
    _sampled_force_check(B, I.config("blend_6p4M_256"), n_sample=3000)


def test_autotune_keeps_the_trajectory(B):
    """The autotuner only changes the re-binning period: state, step count
    and the following trajectory are bit-identical to an untuned run."""
    spec = I.small_system(n_chains=150, N=10, n_a=4, L=10.0, n=32, precision="fp32")
    t, m, pos = _setup(B, spec, sort_every=20)
    t.init_velocities()
    t.step(7)
    r7, v7 = t.positions(), t.velocities()
    k, ms = t.autotune(80)
    assert k in B.Tild.AUTOTUNE_PERIODS and all(v > 0 for v in ms.values())
    assert t.step_count() == 7
    assert np.array_equal(t.positions(), r7) and np.array_equal(t.velocities(), v7)
    t.step(30)
    t2, _, _ = _setup(B, spec, sort_every=20)
    t2.init_velocities()
    t2.step(37)
    assert np.array_equal(t.positions(), t2.positions())
