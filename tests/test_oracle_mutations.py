"""The pins can fail: each plausible mistake below is planted in a copy of the
oracle (on the CPU, by replacing one line of its source) and at least one
pin of tests/test_oracle_pins.py must then fail. The oracle itself is never
modified."""
import os
import sys
import types

import pytest

import test_oracle_pins as pins
import test_oracle_pins_2d as pins2d

ORACLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "tild_oracle.py")

# (mistake, line as written, line with the mistake, pins that must catch it)
MUTATIONS = [
    ("flipped ik sign",
     "grad[K, d] = np.fft.ifftn(1j * kvec[d] * w_hat[K]).real",
     "grad[K, d] = np.fft.ifftn(-1j * kvec[d] * w_hat[K]).real",
     [("test_ik_forces_converge_to_analytic_with_refinement",)]),
    ("the 1/2 dropped from the kernel exponent",
     "return np.exp(-_k2(n, L, dim) * a * a)",
     "return np.exp(-2.0 * _k2(n, L, dim) * a * a)",
     [("test_fft_convolution_matches_real_space_sum",)]),
    ("x and z axes transposed in the spread",
     "flat = ((jx[sel, a] % n) * n + (jy[sel, b] % n)) * n + (jz[sel, c] % n)",
     "flat = ((jz[sel, c] % n) * n + (jy[sel, b] % n)) * n + (jx[sel, a] % n)",
     [("test_spread_bead_on_node_and_wrap",), ("test_analytic_forces_are_energy_gradient", 3)]),
    ("wrong power of the cell volume",
     "return rho.reshape(m.n_species, n, n, n) / m.dx ** 3",
     "return rho.reshape(m.n_species, n, n, n) / m.dx ** 2",
     [("test_spread_conserves_mass", 2)]),
    ("doubled kappa in the pair matrix",
     "return (chi + self.kappa) / self.rho0",
     "return (chi + 2.0 * self.kappa) / self.rho0",
     [("test_analytic_forces_are_energy_gradient", 2)]),
    ("stencil shifted by one point",
     "j0 = np.floor(s - P / 2.0).astype(np.int64) + 1",
     "j0 = np.floor(s - P / 2.0).astype(np.int64) + 2",
     [("test_cic_is_two_nearest_points",), ("test_assignment_weights_invariants", 2)]),
    ("bond constant 1/b^2 instead of 3/b^2",
     "k = 3.0 / m.b ** 2",
     "k = 1.0 / m.b ** 2",
     [("test_two_bead_bond_closed_form",)]),
    ("wrong GJF coefficient b",
     "gb = 1.0 / (1.0 + alpha * dt / (2 * mass))\n    beta",
     "gb = 1.0 / (1.0 + alpha * dt / mass)\n    beta",
     [("test_gjf_harmonic_oscillator_configurational_temperature",), ("test_gjf_free_particle_velocity_variance",)]),
    ("the k = 0 Helfand term kept",
     "p[(0,) * m.dim] = 0.0",
     "p[(0,) * m.dim] = p[(0,) * m.dim]",
     [("test_homogeneous_melt_has_no_field_force",)]),
    ("two Philox output words swapped",
     "c0, c1, c2, c3 = hi1 ^ c1 ^ k0.astype(np.uint32), lo1, hi0 ^ c3 ^ k1.astype(np.uint32), lo0",
     "c0, c1, c2, c3 = hi1 ^ c1 ^ k0.astype(np.uint32), lo0, hi0 ^ c3 ^ k1.astype(np.uint32), lo1",
     [("test_philox_known_answers",)]),
    ("friction sign flipped in the VV adjoint",
     "vhb = vb - al * ft + m.dt * rt",
     "vhb = vb + al * ft + m.dt * rt",
     [("test_vv_trajectory_vjp_matches_finite_differences",)]),
    ("initial-force weight of the VV adjoint dropped",
     "q = 1.0 / (1.0 - al * h)",
     "q = 1.0",
     [("test_vv_trajectory_vjp_matches_finite_differences",)]),
    ("EM adjoint takes the force VJP at the wrong state",
     "v = force_vjp(m, traj[n].pos, c * rb)",
     "v = force_vjp(m, traj[n + 1].pos, c * rb)",
     [("test_em_trajectory_vjp_matches_finite_differences",)]),
]

# mistakes in the two-dimensional form, caught by tests/test_oracle_pins_2d.py
MUTATIONS_2D = [
    ("cell volume instead of cell area in 2D",
     "return rho.reshape(m.n_species, n, n) / m.dx ** 2",
     "return rho.reshape(m.n_species, n, n) / m.dx ** 3",
     [("test_2d_spread_conserves_mass_and_odd_grid", 2)]),
    ("x and y swapped in the 2D spread",
     "flat = (jx[sel, a] % n) * n + (jy[sel, b] % n)",
     "flat = (jy[sel, b] % n) * n + (jx[sel, a] % n)",
     [("test_2d_bead_on_node_puts_one_over_cell_area_there",)]),
    ("3D volume in the 2D model",
     "return self.L ** self.dim",
     "return self.L ** 3",
     [("test_2d_spectral_fields_and_energies_match_real_space_sums", 10)]),
]


def _mutant(old: str, new: str) -> types.ModuleType:
    src = open(ORACLE).read()
    assert src.count(old) == 1, f"the line to mutate must occur once: {old!r}"
    mod = types.ModuleType("oracle_mutant")
    sys.modules["oracle_mutant"] = mod  # dataclasses look their module up while the class is built
    try:
        exec(compile(src.replace(old, new), ORACLE + " (mutant)", "exec"), mod.__dict__)
    finally:
        del sys.modules["oracle_mutant"]
    return mod


@pytest.mark.parametrize("mistake,old,new,catchers", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(mistake, old, new, catchers, monkeypatch):
    monkeypatch.setattr(pins, "O", _mutant(old, new))
    caught = []
    for name, *args in catchers:
        try:
            getattr(pins, name)(*args)
        except AssertionError:
            caught.append(name)
    assert caught, f"no pin caught: {mistake}"


@pytest.mark.parametrize("mistake,old,new,catchers", MUTATIONS_2D, ids=[m[0] for m in MUTATIONS_2D])
def test_planted_2d_mistake_fails_a_pin(mistake, old, new, catchers, monkeypatch):
    monkeypatch.setattr(pins2d, "O", _mutant(old, new))
    caught = []
    for name, *args in catchers:
        try:
            getattr(pins2d, name)(*args)
        except AssertionError:
            caught.append(name)
    assert caught, f"no pin caught: {mistake}"


def test_unmutated_oracle_passes_the_same_pins():
    """The catchers pass on the oracle as written (so a failure above is the
    planted mistake's doing)."""
    for _, _, _, catchers in MUTATIONS:
        for name, *args in catchers:
            getattr(pins, name)(*args)
    for _, _, _, catchers in MUTATIONS_2D:
        for name, *args in catchers:
            getattr(pins2d, name)(*args)
