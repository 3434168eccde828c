"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test names what it pins. None of them re-types an oracle formula: they
compare against published vectors, hand-derived closed forms, direct
real-space sums, invariants or brute force on tiny inputs.
"""
import os

import numpy as np
import pytest

from oracle import tild_oracle as O
from paper_2302_02474_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _model(n_chains=6, N=5, n_a=2, L=4.0, n=8, P=2, chi=1.7, kappa=3.0, a=1.0, seed=3, **kw):
    mt = (I.MolType(n_chains, N, n_a),)
    sp = I.species_of_beads(mt)
    bonds = I.bond_pairs(mt)
    m = O.Model(L=L, n=n, P=P, species=sp.astype(np.int64), n_species=2, bonds=bonds, b=1.0,
                chi=np.array([[0.0, chi], [chi, 0.0]]), kappa=kappa, a=a, seed=seed, **kw)
    pos = I.random_walk_positions(mt, L, 1.0, seed)
    return m, pos


# --------------------------------------------------------------------- RNG


def test_philox_known_answers():
    """Philox4x32-10 reproduces the published known-answer vectors."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = O.philox4x32_10(*v[:6])
        assert [int(x) for x in out] == v[6:]


def test_gaussian_triplets_moments():
    """Box-Muller normals: zero mean, unit variance, uncorrelated, and a
    different stream for each (id, step)."""
    g = O.gaussian_triplets(np.arange(200000), 7, 99)
    assert abs(g.mean()) < 5e-3
    assert np.allclose(g.var(axis=0), 1.0, atol=1e-2)
    c = np.corrcoef(g.T)
    assert np.all(np.abs(c - np.eye(3)) < 1e-2)
    g2 = O.gaussian_triplets(np.arange(200000), 8, 99)
    assert abs(np.corrcoef(g[:, 0], g2[:, 0])[0, 1]) < 1e-2
    # fourth moment of a normal is 3
    assert abs(np.mean(g ** 4) - 3.0) < 0.05


# ----------------------------------------------------------------- weights


def test_assignment_weights_golden():
    """Deserno-Holm closed forms at t = 1/4 for P = 2..5."""
    for line in open(os.path.join(GOLDEN, "assignment_weights.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x) for x in line.split()]
        P, first, nums, den = v[0], v[1], v[2:-1], v[-1]
        j, w = O.stencil(np.array([3.25]), P)
        assert j[0, 0] == first
        np.testing.assert_allclose(w[0], np.array(nums) / den, rtol=0, atol=1e-15)


@pytest.mark.parametrize("P", [2, 3, 4, 5])
def test_assignment_weights_invariants(P):
    """Partition of unity, reproduction of linear functions (first moment),
    symmetry W(t) = W(-t), continuity across cell boundaries."""
    rng = np.random.default_rng(P)
    s = rng.uniform(0, 50, 5000)
    j, w = O.stencil(s, P)
    np.testing.assert_allclose(w.sum(1), 1.0, atol=1e-14)
    np.testing.assert_allclose((j * w).sum(1), s, atol=1e-12)
    assert np.all(w >= -1e-16)
    t = rng.uniform(-P / 2, P / 2, 1000)
    np.testing.assert_allclose(O.cardinal_bspline(t + P / 2, P), O.cardinal_bspline(-t + P / 2, P), atol=1e-14)
    # continuity: weights seen from just below and just above an integer agree
    for base in (3.0, 3.5):
        lo, hi = base - 1e-12, base + 1e-12
        jl, wl = O.stencil(np.array([lo]), P)
        jh, wh = O.stencil(np.array([hi]), P)
        fl = {int(a): b for a, b in zip(jl[0], wl[0])}
        fh = {int(a): b for a, b in zip(jh[0], wh[0])}
        for k in set(fl) | set(fh):
            assert abs(fl.get(k, 0.0) - fh.get(k, 0.0)) < 1e-10


def test_cic_is_two_nearest_points():
    """Order 1 maps a particle to the two nearest grid points per dimension
    with linear weights (Fig. pmm)."""
    j, w = O.stencil(np.array([5.3]), 2)
    assert list(j[0]) == [5, 6]
    np.testing.assert_allclose(w[0], [0.7, 0.3], atol=1e-14)


def test_bspline_derivative_matches_finite_difference():
    x = np.linspace(0.01, 3.99, 397)
    h = 1e-6
    fd = (O.cardinal_bspline(x + h, 4) - O.cardinal_bspline(x - h, 4)) / (2 * h)
    np.testing.assert_allclose(O.cardinal_bspline_derivative(x, 4), fd, atol=1e-8)


# ------------------------------------------------------------------ spread


@pytest.mark.parametrize("P", [2, 3, 4, 5])
def test_spread_conserves_mass(P):
    """sum_g rho_K dV = number of beads of species K (Eq. rhohat)."""
    m, pos = _model(P=P, n_chains=13, N=7, n_a=3, L=5.0, n=10)
    rho = O.spread(m, pos)
    dV = m.dx ** 3
    for K in range(2):
        assert abs(rho[K].sum() * dV - np.sum(m.species == K)) < 1e-12


def test_spread_bead_on_node_and_wrap():
    """A bead on a grid node (order 1) puts 1/dV on that node only; a bead
    at L - eps contributes to the node at index 0 through the wrap."""
    m = O.Model(L=4.0, n=8, P=2, species=np.array([0, 1]), n_species=2, bonds=np.zeros((0, 2), np.int64),
                b=1.0, chi=np.zeros((2, 2)), kappa=1.0, a=0.5)
    pos = np.array([[1.0, 1.5, 2.0], [4.0 - 1e-13, 0.0, 0.0]])
    rho = O.spread(m, pos)
    dV = 0.5 ** 3
    assert rho[0, 2, 3, 4] == pytest.approx(1 / dV, abs=1e-12)
    assert np.count_nonzero(np.abs(rho[0]) > 1e-15) == 1
    assert rho[1, 0, 0, 0] == pytest.approx(1 / dV, rel=1e-9)
    assert rho[1].sum() * dV == pytest.approx(1.0, abs=1e-14)
    # exactly L maps to 0
    assert O.wrap(np.array([4.0, -4.0, 8.0]), 4.0).tolist() == [0.0, 0.0, 0.0]


# ----------------------------------------------- convolution vs real space


def _periodic_gaussian(disp, L, sigma, n_img=3):
    """Unit 3D Gaussian u_G summed over periodic images, and its gradient,
    evaluated directly in real space (Eq. fh's u_G)."""
    u = np.zeros(disp.shape[:-1])
    g = np.zeros(disp.shape)
    norm = (2 * np.pi * sigma * sigma) ** -1.5
    rng = range(-n_img, n_img + 1)
    for ix in rng:
        for iy in rng:
            for iz in rng:
                r = disp + L * np.array([ix, iy, iz])
                e = norm * np.exp(-np.sum(r * r, axis=-1) / (2 * sigma * sigma))
                u += e
                g += -r / (sigma * sigma) * e[..., None]
    return u, g


def test_fft_convolution_matches_real_space_sum():
    """With a >= 2 dx (aliasing below 1e-16) the spectral potential field and
    its ik gradient equal the direct periodic real-space convolution
    w_K(g) = sum_K' eps_KK' dV sum_g' u_G(g - g') rho_K'(g') (Eqs. fh,
    HelfandP, PMM; sigma^2 = 2 a^2). Pins eps, u_hat(0)=1, the sigma-a
    relation, dV and 1/M factors, the sign of i k and the axis order."""
    m, pos = _model(L=4.0, n=8, a=1.0, P=3)
    rho = O.spread(m, pos)
    f = O.potential_fields(m, rho)
    n, dx = m.n, m.dx
    g = np.stack(np.meshgrid(*[np.arange(n) * dx] * 3, indexing="ij"), axis=-1).reshape(-1, 3)
    disp = g[:, None, :] - g[None, :, :]
    u, gu = _periodic_gaussian(disp, m.L, np.sqrt(2) * m.a)
    eps = m.eps()
    dV = dx ** 3
    for K in range(2):
        w_direct = sum(eps[K, Kp] * dV * (u @ rho[Kp].reshape(-1)) for Kp in range(2))
        np.testing.assert_allclose(f["w"][K].reshape(-1), w_direct, rtol=0, atol=1e-12 * np.abs(w_direct).max())
        for d in range(3):
            gd = sum(eps[K, Kp] * dV * (gu[..., d] @ rho[Kp].reshape(-1)) for Kp in range(2))
            np.testing.assert_allclose(f["grad_w"][K, d].reshape(-1), gd, rtol=0, atol=1e-11 * np.abs(gd).max())


def test_field_energies_match_real_space_double_sum():
    """E_chi = (chi/rho0) dV^2 sum_gg' rho_A u_G rho_B (Eq. fh) and
    E_kappa = (kappa/2rho0) dV^2 sum_gg' (rho_+ - rho0) u_G (rho_+ - rho0)
    (Eq. HelfandP), evaluated directly on the grid."""
    m, pos = _model(L=4.0, n=8, a=1.0, P=2)
    rho = O.spread(m, pos)
    e = O.field_energies(m, np.fft.fftn(rho, axes=(1, 2, 3)))
    n, dx = m.n, m.dx
    g = np.stack(np.meshgrid(*[np.arange(n) * dx] * 3, indexing="ij"), axis=-1).reshape(-1, 3)
    u, _ = _periodic_gaussian(g[:, None, :] - g[None, :, :], m.L, np.sqrt(2) * m.a)
    dV = dx ** 3
    ra, rb = rho[0].reshape(-1), rho[1].reshape(-1)
    chi = m.chi[0, 1]
    e_chi = chi / m.rho0 * dV * dV * ra @ u @ rb
    dp = ra + rb - m.rho0
    e_kap = m.kappa / (2 * m.rho0) * dV * dV * dp @ u @ dp
    assert e["chi"] == pytest.approx(e_chi, rel=1e-12)
    assert e["kappa"] == pytest.approx(e_kap, rel=1e-11)


# ------------------------------------------------------------ force checks


@pytest.mark.parametrize("P", [2, 3, 4, 5])
def test_net_nonbonded_force_vanishes(P):
    """ik differentiation with the same assignment weights conserves momentum."""
    m, pos = _model(P=P, n_chains=20, N=6, n_a=2, L=5.0, n=10, a=0.5)
    f = O.nonbonded_forces(m, pos, "ik")
    assert np.abs(f.sum(0)).max() < 1e-12 * np.abs(f).sum()
    fb = O.bond_forces(m, pos)
    assert np.abs(fb.sum(0)).max() < 1e-12 * max(1.0, np.abs(fb).sum())


def test_homogeneous_melt_has_no_field_force():
    """One A and one B bead on every node: uniform densities, zero field
    force, zero Helfand energy, E_chi = chi N_A N_B / (rho0 V)."""
    L, n = 4.0, 8
    g = np.stack(np.meshgrid(*[np.arange(n) * (L / n)] * 3, indexing="ij"), axis=-1).reshape(-1, 3)
    pos = np.concatenate([g, g])
    sp = np.concatenate([np.zeros(len(g), np.int64), np.ones(len(g), np.int64)])
    m = O.Model(L=L, n=n, P=2, species=sp, n_species=2, bonds=np.zeros((0, 2), np.int64), b=1.0,
                chi=np.array([[0.0, 2.0], [2.0, 0.0]]), kappa=5.0, a=0.5)
    f = O.nonbonded_forces(m, pos)
    assert np.abs(f).max() < 1e-12
    e = O.energies(m, pos)
    assert abs(e["kappa"]) < 1e-10
    assert e["chi"] == pytest.approx(2.0 * len(g) * len(g) / (m.rho0 * L ** 3), rel=1e-12)


def test_translation_by_grid_vector():
    """Shifting every bead by an integer number of grid spacings leaves the
    energies and the forces unchanged."""
    m, pos = _model(P=3, L=5.0, n=10, a=0.6)
    shift = m.dx * np.array([3, -2, 7])
    f0, f1 = O.forces(m, pos), O.forces(m, O.wrap(pos + shift, m.L))
    np.testing.assert_allclose(f1, f0, atol=1e-11 * np.abs(f0).max())
    e0, e1 = O.energies(m, pos), O.energies(m, O.wrap(pos + shift, m.L))
    for k in e0:
        assert e1[k] == pytest.approx(e0[k], rel=1e-11, abs=1e-12)


@pytest.mark.parametrize("P", [2, 3, 4, 5])
def test_analytic_forces_are_energy_gradient(P):
    """Central differences of E_bond + E_chi + E_kappa equal the analytic
    gradient of the gridded energy (bond force of Eq. bonds: -3/b^2 dr)."""
    m, pos = _model(P=P, n_chains=4, N=4, n_a=2, L=4.0, n=8, a=0.5)
    f = O.forces(m, pos, variant="analytic")

    def etot(p):
        e = O.energies(m, p)
        return e["bond"] + e["chi"] + e["kappa"]

    h = 1e-5
    for i in (0, 3, 9, 15):
        for d in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, d] += h
            pm[i, d] -= h
            fd = -(etot(pp) - etot(pm)) / (2 * h)
            assert abs(fd - f[i, d]) < 1e-7 * max(1.0, np.abs(f).max())


def test_ik_forces_converge_to_analytic_with_refinement():
    """The ik and analytic forces of the same gridded model approach each
    other as the grid is refined (both converge to the continuum force)."""
    errs = []
    for n in (8, 16, 32):
        m, pos = _model(P=4, n_chains=4, N=4, n_a=2, L=4.0, n=n, a=0.5)
        fa = O.nonbonded_forces(m, pos, "analytic")
        fi = O.nonbonded_forces(m, pos, "ik")
        errs.append(np.linalg.norm(fi - fa) / np.linalg.norm(fa))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 2e-3


def test_two_bead_bond_closed_form():
    """Eq. bonds for one bond: E = 3/(2b^2) d^2, F_1 = -3/b^2 d; across the
    periodic boundary the minimum image is used."""
    m = O.Model(L=10.0, n=8, P=2, species=np.array([0, 0]), n_species=1, bonds=np.array([[0, 1]]), b=1.3,
                chi=np.zeros((1, 1)), kappa=0.0, a=0.5)
    pos = np.array([[9.8, 1.0, 5.0], [0.4, 1.5, 4.0]])
    d = np.array([-0.6, -0.5, 1.0])
    assert O.bond_energy(m, pos) == pytest.approx(1.5 / 1.3 ** 2 * d @ d, rel=1e-13)
    f = O.bond_forces(m, pos)
    np.testing.assert_allclose(f[0], -3 / 1.3 ** 2 * d, atol=1e-13)
    np.testing.assert_allclose(f[1], 3 / 1.3 ** 2 * d, atol=1e-13)


# ------------------------------------------------------------- integrator


def test_gjf_harmonic_oscillator_configurational_temperature():
    """GJF samples <x^2> = kT/k exactly for any stable dt (Gronbech-Jensen &
    Farago 2013); with omega dt = 0.8 Euler-type schemes would be far off."""
    k = 4.0
    n = 4000
    m = O.Model(L=1000.0, n=8, P=2, species=np.zeros(n, np.int64), n_species=1, bonds=np.zeros((0, 2), np.int64),
                b=1.0, chi=np.zeros((1, 1)), kappa=0.0, a=0.5, dt=0.4, friction=1.0, kT=1.5, seed=11)
    c = 500.0

    def force(mm, p):
        return -k * (p - c)

    st = O.initial_state(m, np.full((n, 3), c), force_fn=force)
    xs = []
    for it in range(400):
        st = O.gjf_step(m, st, force)
        if it >= 100 and it % 5 == 0:
            xs.append(np.mean((st.pos - c) ** 2))
    x2 = np.mean(xs)
    assert abs(x2 - m.kT / k) < 0.03 * m.kT / k


@pytest.mark.slow
def test_ideal_chain_statistics_and_equipartition():
    """chi = kappa = 0: bonds only (Eq. bonds). Equilibrium ideal Gaussian
    chains: <|dr|^2> = b^2, <R_ee^2> = (N-1) b^2, <R_g^2> = b^2 (N^2-1)/(6N);
    kinetic temperature <v^2> = kT/m per component."""
    N, nc = 20, 400
    mt = (I.MolType(nc, N, N),)
    sp = I.species_of_beads(mt).astype(np.int64)
    m = O.Model(L=60.0, n=8, P=2, species=sp, n_species=1, bonds=I.bond_pairs(mt), b=1.0,
                chi=np.zeros((1, 1)), kappa=0.0, a=0.5, dt=0.05, friction=1.0, kT=1.0, seed=5)
    pos = I.random_walk_positions(mt, m.L, 1.0, 21)

    def force(mm, p):
        return O.bond_forces(mm, p)

    st = O.initial_state(m, pos, force_fn=force)
    b2, ree, rg, v2 = [], [], [], []
    for it in range(3000):
        st = O.gjf_step(m, st, force)
        if it >= 500 and it % 25 == 0:
            d = O.bond_vectors(m, st.pos).reshape(nc, N - 1, 3)
            r = np.concatenate([np.zeros((nc, 1, 3)), np.cumsum(d * -1, axis=1)], axis=1)
            b2.append(np.mean(np.sum(d * d, -1)))
            ree.append(np.mean(np.sum(r[:, -1] ** 2, -1)))
            rc = r - r.mean(1, keepdims=True)
            rg.append(np.mean(np.sum(rc * rc, -1)))
            v2.append(np.mean(st.vel ** 2))
    assert abs(np.mean(b2) - 1.0) < 0.03
    assert abs(np.mean(ree) - (N - 1)) < 0.06 * (N - 1)
    assert abs(np.mean(rg) - (N * N - 1) / (6 * N)) < 0.06 * (N * N - 1) / (6 * N)
    # GJF kinetic bias is O((omega dt)^2) ~ 3e-2 here at the stiffest mode
    assert abs(np.mean(v2) - 1.0) < 0.03


def test_gjf_free_particle_velocity_variance():
    """No forces: <v^2> = kT/m is stationary from the Maxwell-Boltzmann start."""
    n = 20000
    m = O.Model(L=50.0, n=8, P=2, species=np.zeros(n, np.int64), n_species=1, bonds=np.zeros((0, 2), np.int64),
                b=1.0, chi=np.zeros((1, 1)), kappa=0.0, a=0.5, dt=0.05, friction=2.0, kT=0.7, seed=2)

    def force(mm, p):
        return np.zeros_like(p)

    st = O.initial_state(m, np.full((n, 3), 1.0), force_fn=force)
    assert abs(np.mean(st.vel ** 2) - 0.7) < 0.02
    for _ in range(50):
        st = O.gjf_step(m, st, force)
    assert abs(np.mean(st.vel ** 2) - 0.7) < 0.02


# ----------------------------------------- Euler-Maruyama and velocity-Verlet


def _free_or_bonded(n_beads, bonds, **kw):
    return O.Model(L=kw.pop("L", 50.0), n=8, P=2, species=np.zeros(n_beads, np.int64), n_species=1,
                   bonds=bonds, b=1.0, chi=np.zeros((1, 1)), kappa=0.0, a=0.5, **kw)


def test_em_free_particle_diffusion_coefficient():
    """Brownian dynamics of free particles: <|r(t) - r(0)|^2> = 6 D t with
    the Einstein relation D = kT / alpha (exact for the EM discretisation)."""
    n, K = 20000, 50
    m = _free_or_bonded(n, np.zeros((0, 2), np.int64), dt=0.01, friction=2.0, kT=0.7, seed=4)

    def force(mm, p):
        return np.zeros_like(p)

    st = O.em_initial_state(m, np.full((n, 3), 25.0), force_fn=force)
    disp = np.zeros((n, 3))
    for _ in range(K):
        new = O.em_step(m, st, force)
        disp += O.minimum_image(new.pos - st.pos, m.L)
        st = new
    msd = np.mean(np.sum(disp * disp, axis=1))
    assert abs(msd - 6.0 * (0.7 / 2.0) * K * m.dt) < 0.03 * 6.0 * (0.7 / 2.0) * K * m.dt
    assert not np.any(st.vel)


def test_em_dimer_bond_length_closed_form():
    """Dimers with the bond force of Eq. bonds (k = 3/b^2) under EM: the
    bond vector is an AR(1) process d' = (1 - 2 k dt/alpha) d + noise of
    variance 4 kT dt/alpha per component, whose stationary mean square is
    <|d|^2> = 3 (kT/k) / (1 - k dt/alpha) (= b^2 as dt -> 0)."""
    nd = 10000
    bonds = np.stack([2 * np.arange(nd), 2 * np.arange(nd) + 1], axis=1).astype(np.int64)
    m = _free_or_bonded(2 * nd, bonds, L=400.0, dt=0.03, friction=1.0, kT=1.0, seed=8)

    def force(mm, p):
        return O.bond_forces(mm, p)

    rng = np.random.default_rng(3)
    pos = np.repeat(rng.uniform(10, 390, size=(nd, 3)), 2, axis=0)
    pos[1::2] += rng.normal(size=(nd, 3)) / np.sqrt(3.0)
    st = O.em_initial_state(m, pos, force_fn=force)
    d2 = []
    for it in range(400):
        st = O.em_step(m, st, force)
        if it >= 100 and it % 10 == 0:
            d = O.bond_vectors(m, st.pos)
            d2.append(np.mean(np.sum(d * d, axis=1)))
    expect = 3.0 * (1.0 / 3.0) / (1.0 - 3.0 * m.dt / m.friction)
    assert abs(np.mean(d2) - expect) < 0.015 * expect
    assert abs(expect - 1.0) > 0.08  # the pin distinguishes the discrete process from its continuum limit


def test_vv_is_time_reversible_without_friction():
    """alpha = 0: velocity-Verlet is time reversible for any position-only
    force (here the full field + bond force): n steps, reverse velocities,
    n steps returns to the start."""
    m, pos = _model(friction=0.0, dt=0.01)
    vel = np.random.default_rng(2).normal(size=pos.shape)
    st0 = O.vv_initial_state(m, pos, vel)
    st = O.run_with(O.vv_step, m, st0, 30)
    assert np.abs(O.minimum_image(st.pos - st0.pos, m.L)).max() > 0.1
    back = O.run_with(O.vv_step, m, O.State(st.pos, -st.vel, st.force, st.step), 30)
    assert np.abs(O.minimum_image(back.pos - st0.pos, m.L)).max() < 1e-9
    np.testing.assert_allclose(-back.vel, vel, atol=1e-8)


def test_vv_conserves_energy_without_friction():
    """alpha = 0, bonds only: E = kinetic + bond energy stays within the
    O((omega dt)^2) shadow-Hamiltonian band and does not drift."""
    mt = (I.MolType(200, 10, 10),)
    m = O.Model(L=40.0, n=8, P=2, species=I.species_of_beads(mt).astype(np.int64), n_species=1,
                bonds=I.bond_pairs(mt), b=1.0, chi=np.zeros((1, 1)), kappa=0.0, a=0.5, dt=0.01, friction=0.0,
                kT=1.0, seed=9)
    pos = I.random_walk_positions(mt, m.L, 1.0, 4)
    vel = np.random.default_rng(6).normal(size=pos.shape)

    def force(mm, p):
        return O.bond_forces(mm, p)

    st = O.vv_initial_state(m, pos, vel, force_fn=force)
    e = []
    for _ in range(500):
        st = O.vv_step(m, st, force)
        e.append(O.kinetic_energy(m, st.vel) + O.bond_energy(m, st.pos))
    e = np.array(e)
    assert np.abs(e - e[0]).max() < 1e-3 * abs(e[0])
    assert abs(e[-50:].mean() - e[:50].mean()) < 2e-4 * abs(e[0])


def test_vv_langevin_free_particle_velocity_variances():
    """Free particles under VV + Langevin force: the half-step velocity is
    an AR(1) process u' = (1 - alpha dt/m) u + (dt/m) sigma xi with
    stationary variance (kT/m) / (1 - alpha dt/2m), and the full-step
    velocity v = u + (dt/2m) F then has variance exactly kT/m."""
    n = 20000
    m = _free_or_bonded(n, np.zeros((0, 2), np.int64), dt=0.1, friction=2.0, kT=0.7, seed=12)

    def force(mm, p):
        return np.zeros_like(p)

    vel = np.sqrt(0.7) * np.random.default_rng(1).normal(size=(n, 3))
    st = O.vv_initial_state(m, np.full((n, 3), 25.0), vel, force_fn=force)
    v2, u2 = [], []
    for it in range(120):
        st = O.vv_step(m, st, force)
        if it >= 40 and it % 4 == 0:
            v2.append(np.mean(st.vel ** 2))
            u2.append(np.mean((st.vel - m.dt / 2 * st.force) ** 2))
    assert abs(np.mean(v2) - 0.7) < 0.01 * 0.7
    expect_u = 0.7 / (1.0 - 2.0 * 0.1 / 2.0)
    assert abs(np.mean(u2) - expect_u) < 0.01 * expect_u
    assert expect_u / 0.7 > 1.1  # distinguishes the half-step from the full-step variance


# ------------------------------------------------------------ electrostatics


def _charged_pair(r, n, L=24.0, ae=1.0, lb=1.0, P=4):
    """A +1 (species A) and a -1 (species B) charge at separation r along x."""
    m = O.Model(L=L, n=n, P=P, species=np.array([0, 1]), n_species=2, bonds=np.zeros((0, 2), np.int64), b=1.0,
                chi=np.zeros((2, 2)), kappa=0.0, a=0.5, charges=np.array([1.0, -1.0]), bjerrum=lb, charge_smear=ae)
    c = np.array([L / 2 + 0.13, L / 2 - 0.21, L / 2 + 0.07])
    return m, np.stack([c - [r / 2, 0, 0], c + [r / 2, 0, 0]])


def test_coulomb_pair_converges_to_the_smeared_closed_form():
    """Two opposite charges smeared over unit Gaussians of width a_e interact
    through -l_B erf(r / 2 a_e) / r (the convolution of two such Gaussians
    has variance 2 a_e^2 per axis). Differences of the gridded energy and the
    gridded force along the pair axis approach that closed form as the grid
    is refined (the particle-mesh smoothing of order-P splines is the
    method's own error): the error falls at least twofold from dx = 0.5 to
    dx = 0.25, where it is below 3% (the images of the neutral pair in
    L = 24 contribute about 1e-3). A wrong 4 pi, a missing 1/2, the smearing
    exponent a_e^2/2 or a flipped sign each miss by 20% or more."""
    from math import erf, exp, pi, sqrt

    def closed_e(r):
        return -erf(r / 2.0) / r

    def closed_f(r):  # force on the +1 charge along +x (attractive: towards the -1 charge)
        return -(erf(r / 2.0) / r ** 2 - exp(-r * r / 4.0) / (sqrt(pi) * r))

    errs = []
    for n in (48, 96):
        e = {}
        for r in (1.5, 3.0):
            m, pos = _charged_pair(r, n)
            e[r] = O.energies(m, pos)["elec"]
        de = e[1.5] - e[3.0]
        ref = closed_e(1.5) - closed_e(3.0)
        m, pos = _charged_pair(2.0, n)
        fx = O.nonbonded_forces(m, pos, "analytic")[0, 0]
        errs.append((abs(de / ref - 1.0), abs(fx / -closed_f(2.0) - 1.0)))
    assert errs[1][0] < 0.5 * errs[0][0] and errs[1][1] < 0.5 * errs[0][1]
    assert errs[1][0] < 0.03 and errs[1][1] < 0.03


def test_charged_forces_are_energy_gradient():
    """With charges, central differences of the total energy (bond, chi,
    kappa and electrostatic) equal the analytic force."""
    m, pos = _model(P=3, n_chains=4, N=4, n_a=2, L=4.0, n=8, a=0.5, charges=np.array([0.7, -1.1]), bjerrum=2.0,
                    charge_smear=0.4)
    f = O.forces(m, pos, variant="analytic")

    def etot(p):
        e = O.energies(m, p)
        return e["bond"] + e["chi"] + e["kappa"] + e["elec"]

    assert abs(O.energies(m, pos)["elec"]) > 1e-3
    h = 1e-5
    for i in (0, 5, 10):
        for d in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, d] += h
            pm[i, d] -= h
            fd = -(etot(pp) - etot(pm)) / (2 * h)
            assert abs(fd - f[i, d]) < 1e-7 * max(1.0, np.abs(f).max())


def test_neutral_homogeneous_melt_has_no_electrostatics():
    """A +1 and a -1 bead on every node: zero charge density, no
    electrostatic energy or force."""
    L, n = 4.0, 8
    g = np.stack(np.meshgrid(*[np.arange(n) * (L / n)] * 3, indexing="ij"), axis=-1).reshape(-1, 3)
    pos = np.concatenate([g, g])
    sp = np.concatenate([np.zeros(len(g), np.int64), np.ones(len(g), np.int64)])
    m = O.Model(L=L, n=n, P=2, species=sp, n_species=2, bonds=np.zeros((0, 2), np.int64), b=1.0,
                chi=np.zeros((2, 2)), kappa=0.0, a=0.5, charges=np.array([1.0, -1.0]), bjerrum=3.0, charge_smear=0.5)
    assert abs(O.energies(m, pos)["elec"]) < 1e-12
    assert np.abs(O.nonbonded_forces(m, pos)).max() < 1e-12


# ------------------------------------------------------- force vector-Jacobian


@pytest.mark.parametrize("P", [2, 3, 4, 5])
def test_force_vjp_matches_finite_differences(P):
    """J^T lam of the ik force equals central differences of sum_i lam_i . F_i
    with respect to positions, chi, kappa and a (with charges on)."""
    m, pos = _model(P=P, n_chains=4, N=4, n_a=2, L=4.0, n=8, a=0.6, charges=np.array([0.5, -0.8]), bjerrum=1.5,
                    charge_smear=0.5)
    lam = np.random.default_rng(7).normal(size=pos.shape)
    v = O.force_vjp(m, pos, lam)

    def lf(mm, p):
        return float(np.sum(lam * O.forces(mm, p)))

    h = 1e-5
    scale = max(1.0, np.abs(v["r"]).max())
    for i in (0, 5, 11):
        for d in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, d] += h
            pm[i, d] -= h
            fd = (lf(m, pp) - lf(m, pm)) / (2 * h)
            assert abs(fd - v["r"][i, d]) < 1e-6 * scale
    import dataclasses
    for name, attr, get in (("chi", "chi", lambda mm: mm.chi[0, 1]), ("kappa", "kappa", None), ("a", "a", None)):
        mp, mm_ = dataclasses.replace(m), dataclasses.replace(m)
        if name == "chi":
            mp.chi = m.chi + h * np.array([[0, 1], [1, 0]])
            mm_.chi = m.chi - h * np.array([[0, 1], [1, 0]])
        else:
            setattr(mp, attr, getattr(m, attr) + h)
            setattr(mm_, attr, getattr(m, attr) - h)
        fd = (lf(mp, pos) - lf(mm_, pos)) / (2 * h)
        assert fd == pytest.approx(v[name], rel=1e-6, abs=1e-8)


def test_gjf_trajectory_vjp_matches_finite_differences():
    """Reverse-mode derivatives of L = sum w . r^K after K GJF steps (noise
    fixed) equal central differences of L with respect to chi, kappa, a, an
    initial position and an initial velocity."""
    import dataclasses

    m, pos = _model(P=2, n_chains=4, N=4, n_a=2, L=4.0, n=8, a=0.6, dt=0.02)
    vel = O.initial_state(m, pos).vel
    K = 6
    w = np.random.default_rng(9).normal(size=pos.shape)
    g = O.gjf_trajectory_vjp(m, pos, vel, K, w)

    def loss(mm, p, v):
        st = O.State(O.wrap(p, mm.L), v, O.forces(mm, O.wrap(p, mm.L)), 0)
        st = O.run(mm, st, K)
        r = st.pos
        # unwrap against the start so a boundary crossing does not jump
        return float(np.sum(w * (O.wrap(pos, mm.L) + O.minimum_image(r - O.wrap(pos, mm.L), mm.L))))

    h = 1e-6
    for name in ("chi", "kappa", "a"):
        mp, mm_ = dataclasses.replace(m), dataclasses.replace(m)
        if name == "chi":
            mp.chi, mm_.chi = m.chi + h * np.array([[0, 1], [1, 0]]), m.chi - h * np.array([[0, 1], [1, 0]])
        else:
            setattr(mp, name, getattr(m, name) + h)
            setattr(mm_, name, getattr(m, name) - h)
        fd = (loss(mp, pos, vel) - loss(mm_, pos, vel)) / (2 * h)
        assert fd == pytest.approx(g[name], rel=1e-5, abs=1e-9), name
    for i, d in ((0, 1), (7, 2)):
        pp, pm = pos.copy(), pos.copy()
        pp[i, d] += h
        pm[i, d] -= h
        assert (loss(m, pp, vel) - loss(m, pm, vel)) / (2 * h) == pytest.approx(g["r0"][i, d], rel=1e-5, abs=1e-9)
        vp, vm = vel.copy(), vel.copy()
        vp[i, d] += h
        vm[i, d] -= h
        assert (loss(m, pos, vp) - loss(m, pos, vm)) / (2 * h) == pytest.approx(g["v0"][i, d], rel=1e-5, abs=1e-9)


def _fd_trajectory_pins(m, pos, vel, g, loss, check_v0=True):
    """Central differences of `loss(model, pos, vel)` against the reverse-mode
    derivatives g (chi, kappa, a, two initial positions and velocities)."""
    import dataclasses

    h = 1e-6
    for name in ("chi", "kappa", "a"):
        mp, mm_ = dataclasses.replace(m), dataclasses.replace(m)
        if name == "chi":
            mp.chi, mm_.chi = m.chi + h * np.array([[0, 1], [1, 0]]), m.chi - h * np.array([[0, 1], [1, 0]])
        else:
            setattr(mp, name, getattr(m, name) + h)
            setattr(mm_, name, getattr(m, name) - h)
        fd = (loss(mp, pos, vel) - loss(mm_, pos, vel)) / (2 * h)
        assert fd == pytest.approx(g[name], rel=1e-5, abs=1e-9), name
    for i, d in ((0, 1), (7, 2)):
        pp, pm = pos.copy(), pos.copy()
        pp[i, d] += h
        pm[i, d] -= h
        assert (loss(m, pp, vel) - loss(m, pm, vel)) / (2 * h) == pytest.approx(g["r0"][i, d], rel=1e-5, abs=1e-9)
        if check_v0:
            vp, vm = vel.copy(), vel.copy()
            vp[i, d] += h
            vm[i, d] -= h
            assert (loss(m, pos, vp) - loss(m, pos, vm)) / (2 * h) == pytest.approx(g["v0"][i, d], rel=1e-5, abs=1e-9)


def test_em_trajectory_vjp_matches_finite_differences():
    """Reverse-mode derivatives of L = sum w . r^K after K Euler-Maruyama
    steps (noise fixed) equal central differences of L with respect to chi,
    kappa, a and initial positions; dL/dv^0 is zero (no velocity)."""
    m, pos = _model(P=2, n_chains=4, N=4, n_a=2, L=4.0, n=8, a=0.6, dt=0.01, friction=2.0)
    K = 6
    w = np.random.default_rng(10).normal(size=pos.shape)
    g = O.em_trajectory_vjp(m, pos, K, w)
    assert not np.any(g["v0"])

    def loss(mm, p, v):
        st = O.run_with(O.em_step, mm, O.em_initial_state(mm, p), K)
        r0 = O.wrap(pos, mm.L)
        return float(np.sum(w * (r0 + O.minimum_image(st.pos - r0, mm.L))))

    _fd_trajectory_pins(m, pos, np.zeros_like(pos), g, loss, check_v0=False)


def test_vv_trajectory_vjp_matches_finite_differences():
    """Reverse-mode derivatives of L = sum w . r^K + sum u . v^K after K
    velocity-Verlet steps with the Langevin force (noise fixed) equal central
    differences of L with respect to chi, kappa, a, initial positions and
    initial velocities."""
    m, pos = _model(P=2, n_chains=4, N=4, n_a=2, L=4.0, n=8, a=0.6, dt=0.02, friction=0.7)
    vel = O.initial_state(m, pos).vel
    K = 6
    rng = np.random.default_rng(11)
    w, u = rng.normal(size=pos.shape), rng.normal(size=pos.shape)
    g = O.vv_trajectory_vjp(m, pos, vel, K, w, u)

    def loss(mm, p, v):
        st = O.run_with(O.vv_step, mm, O.vv_initial_state(mm, p, v), K)
        r0 = O.wrap(pos, mm.L)
        return float(np.sum(w * (r0 + O.minimum_image(st.pos - r0, mm.L))) + np.sum(u * st.vel))

    _fd_trajectory_pins(m, pos, vel, g, loss)


def test_gjf_trajectory_vjp_with_velocity_loss_matches_finite_differences():
    """As the GJF pin above, with a velocity term in the loss:
    L = sum w . r^K + sum u . v^K."""
    m, pos = _model(P=2, n_chains=4, N=4, n_a=2, L=4.0, n=8, a=0.6, dt=0.02)
    vel = O.initial_state(m, pos).vel
    K = 5
    rng = np.random.default_rng(12)
    w, u = rng.normal(size=pos.shape), rng.normal(size=pos.shape)
    g = O.gjf_trajectory_vjp(m, pos, vel, K, w, u)

    def loss(mm, p, v):
        st = O.run(mm, O.State(O.wrap(p, mm.L), v, O.forces(mm, O.wrap(p, mm.L)), 0), K)
        r0 = O.wrap(pos, mm.L)
        return float(np.sum(w * (r0 + O.minimum_image(st.pos - r0, mm.L))) + np.sum(u * st.vel))

    _fd_trajectory_pins(m, pos, vel, g, loss)


@pytest.mark.parametrize("P", [2, 3, 4, 5])
def test_spread_vjp_matches_finite_differences(P):
    """spread_vjp is the gradient of the linear functional sum_{K,g}
    psi_K(g) rho_K(g) of the positions: central differences of that sum
    (computed with the spread itself) agree to O(h^2)."""
    m, pos = _model(P=P, n_chains=5, N=4, n_a=2, L=4.0, n=8, a=0.5)
    rng = np.random.default_rng(P)
    psi = rng.normal(size=(2, m.n, m.n, m.n))
    g = O.spread_vjp(m, pos, psi)

    def f(p):
        return float(np.sum(psi * O.spread(m, p)))

    h = 1e-6
    for i in (0, 7, 13):
        for d in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, d] += h
            pm[i, d] -= h
            fd = (f(pp) - f(pm)) / (2 * h)
            assert abs(fd - g[i, d]) < 1e-6 * max(1.0, np.abs(g).max())
