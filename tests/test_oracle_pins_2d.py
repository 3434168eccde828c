"""Pins of the oracle's two-dimensional form (Sec. "TILD Branch": periodic
boxes in two or three dimensions; Listing infile runs D = 2 on a 65 x 65
grid), each against a fact fixed outside the oracle: bead counts, a direct
periodic real-space double sum with the 2D unit Gaussian written out, a
homogeneous melt, momentum conservation, finite differences of the energy,
and the GJF harmonic-oscillator configurational temperature in 2D.
"""
import numpy as np
import pytest

from oracle import tild_oracle as O


def _model2d(N=60, L=5.0, n=10, P=2, chi=1.4, kappa=4.0, a=0.8, seed=2):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, L, size=(N, 2))
    sp = (np.arange(N) % 3 == 0).astype(np.int64)
    bonds = np.stack([np.arange(0, N - 1, 2), np.arange(1, N, 2)], axis=1).astype(np.int64)
    m = O.Model(L=L, n=n, P=P, species=sp, n_species=2, bonds=bonds, b=1.0,
                chi=np.array([[0.0, chi], [chi, 0.0]]), kappa=kappa, a=a, seed=seed, dim=2)
    return m, pos


@pytest.mark.parametrize("P", [2, 3, 4, 5])
def test_2d_spread_conserves_mass_and_odd_grid(P):
    for n in (10, 13, 65):
        m, pos = _model2d(n=n, P=P, L=9.0)
        rho = O.spread(m, pos)
        assert rho.shape == (2, n, n)
        dA = m.dx ** 2
        for K in range(2):
            assert rho[K].sum() * dA == pytest.approx(np.sum(m.species == K), rel=1e-13)


def test_2d_bead_on_node_puts_one_over_cell_area_there():
    m, _ = _model2d(N=2, n=13, L=6.5)
    pos = np.array([[3 * m.dx, 7 * m.dx], [0.0, 0.0]])
    rho = O.spread(m, pos)
    assert rho[1, 3, 7] == pytest.approx(1.0 / m.dx ** 2, rel=1e-12)
    assert np.count_nonzero(np.abs(rho[1]) > 1e-14) == 1


def _periodic_gaussian_2d(disp, L, sigma, n_img=4):
    """Unit 2D Gaussian (2 pi sigma^2)^-1 exp(-r^2 / 2 sigma^2) (Eq. fh's u_G
    with D = 2) summed over periodic images, and its gradient."""
    u = np.zeros(disp.shape[:-1])
    g = np.zeros(disp.shape)
    norm = 1.0 / (2 * np.pi * sigma * sigma)
    for ix in range(-n_img, n_img + 1):
        for iy in range(-n_img, n_img + 1):
            r = disp + L * np.array([ix, iy])
            e = norm * np.exp(-np.sum(r * r, axis=-1) / (2 * sigma * sigma))
            u += e
            g += -r / (sigma * sigma) * e[..., None]
    return u, g


@pytest.mark.parametrize("n", [10, 9])
def test_2d_spectral_fields_and_energies_match_real_space_sums(n):
    """Potential, ik gradient and Flory/Helfand energies on the grid equal
    the direct periodic real-space sums with the 2D unit Gaussian (odd and
    even n; a >= 2 dx so aliasing is below 1e-16)."""
    m, pos = _model2d(n=n, L=4.5, a=1.0, P=3)
    rho = O.spread(m, pos)
    f = O.potential_fields(m, rho)
    dx = m.dx
    g = np.stack(np.meshgrid(*[np.arange(n) * dx] * 2, indexing="ij"), axis=-1).reshape(-1, 2)
    u, gu = _periodic_gaussian_2d(g[:, None, :] - g[None, :, :], m.L, np.sqrt(2) * m.a)
    eps = m.eps()
    dA = dx * dx
    for K in range(2):
        w = sum(eps[K, Kp] * dA * (u @ rho[Kp].reshape(-1)) for Kp in range(2))
        np.testing.assert_allclose(f["w"][K].reshape(-1), w, rtol=0, atol=1e-12 * np.abs(w).max())
        if n % 2 == 1:  # no Nyquist column: the ik gradient is the exact derivative of the sum
            for d in range(2):
                gd = sum(eps[K, Kp] * dA * (gu[..., d] @ rho[Kp].reshape(-1)) for Kp in range(2))
                np.testing.assert_allclose(f["grad_w"][K, d].reshape(-1), gd, rtol=0, atol=1e-11 * np.abs(gd).max())
    e = O.energies(m, pos)
    ra, rb = rho[0].reshape(-1), rho[1].reshape(-1)
    assert e["chi"] == pytest.approx(m.chi[0, 1] / m.rho0 * dA * dA * ra @ u @ rb, rel=1e-12)
    dp = ra + rb - m.rho0
    assert e["kappa"] == pytest.approx(m.kappa / (2 * m.rho0) * dA * dA * dp @ u @ dp, rel=1e-11)
    assert m.rho0 == pytest.approx(m.n_beads / m.L ** 2)


def test_2d_homogeneous_melt_has_no_field_force():
    L, n = 4.0, 8
    g = np.stack(np.meshgrid(*[np.arange(n) * (L / n)] * 2, indexing="ij"), axis=-1).reshape(-1, 2)
    pos = np.concatenate([g, g])
    sp = np.concatenate([np.zeros(len(g), np.int64), np.ones(len(g), np.int64)])
    m = O.Model(L=L, n=n, P=2, species=sp, n_species=2, bonds=np.zeros((0, 2), np.int64), b=1.0,
                chi=np.array([[0.0, 2.0], [2.0, 0.0]]), kappa=5.0, a=0.5, dim=2)
    assert np.abs(O.nonbonded_forces(m, pos)).max() < 1e-12
    e = O.energies(m, pos)
    assert abs(e["kappa"]) < 1e-10
    assert e["chi"] == pytest.approx(2.0 * len(g) * len(g) / (m.rho0 * L ** 2), rel=1e-12)


@pytest.mark.parametrize("P", [2, 3, 4, 5])
def test_2d_net_force_vanishes_and_analytic_force_is_energy_gradient(P):
    m, pos = _model2d(n=11, P=P, L=5.5, a=0.6)
    f = O.nonbonded_forces(m, pos, "ik")
    assert f.shape == (m.n_beads, 2)
    assert np.abs(f.sum(0)).max() < 1e-12 * np.abs(f).sum()
    fa = O.forces(m, pos, variant="analytic")

    def etot(p):
        e = O.energies(m, p)
        return e["bond"] + e["chi"] + e["kappa"]

    h = 1e-5
    for i in (0, 5, 17):
        for d in range(2):
            pp, pm = pos.copy(), pos.copy()
            pp[i, d] += h
            pm[i, d] -= h
            assert abs(-(etot(pp) - etot(pm)) / (2 * h) - fa[i, d]) < 1e-7 * max(1.0, np.abs(fa).max())


def test_2d_gjf_harmonic_oscillator_configurational_temperature():
    """GJF samples the Boltzmann distribution of a harmonic potential
    exactly for any stable dt, in any dimension: for 2D dimers joined by one
    bond of energy (3/2b^2)|d|^2 (Eq. bonds), each component of the bond
    vector d has variance kT b^2 / 3."""
    n_dimers = 400
    L = 40.0
    rng = np.random.default_rng(4)
    pos = rng.uniform(0, L, size=(2 * n_dimers, 2))
    pos[1::2] = pos[0::2] + 0.3
    bonds = np.stack([np.arange(0, 2 * n_dimers, 2), np.arange(1, 2 * n_dimers, 2)], axis=1).astype(np.int64)
    m = O.Model(L=L, n=8, P=2, species=np.zeros(2 * n_dimers, np.int64), n_species=1, bonds=bonds, b=1.0,
                chi=np.zeros((1, 1)), kappa=0.0, a=0.5, dt=0.05, friction=1.0, kT=1.0, seed=11, dim=2)
    st = O.initial_state(m, pos, force_fn=O.bond_forces)
    st = O.run(m, st, 200, force_fn=O.bond_forces)
    acc = []
    for _ in range(600):
        st = O.gjf_step(m, st, force_fn=O.bond_forces)
        acc.append(np.mean(O.bond_vectors(m, st.pos) ** 2))
    assert float(np.mean(acc)) == pytest.approx(1.0 / 3.0, rel=0.08)
