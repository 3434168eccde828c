"""Plain FP64 CPU oracle of the TILD timestep (MATILDA.FT, arXiv 2302.02474).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module. It shares no code with the CUDA path and imports nothing from it;
both sides receive the same seeded arrays from the input generator.

What it computes, in the paper's notation (Sec. "Structure of
theoretically-informed coarse-grained and field-theoretic models" and
Sec. "Long-range interactions"):

* microscopic densities rho_K (Eq. rhohat) assigned to a periodic grid with
  the Deserno-Holm / cardinal B-spline weights of order P = pmeorder + 1
  (Sec. "Long-range interactions"; the same weights interpolate forces back,
  caption of Fig. pmm);
* the Gaussian-smeared Flory (Eq. fh) and Helfand (Eq. HelfandP) energies,
  with u_G a unit Gaussian of width sigma, sigma^2 = 2 a^2 (Eqs. smearRho,
  fhF, HelfandF), evaluated by FFT convolution (Eq. PMM);
* the harmonic bond energy with spring constant 3/b^2 (Eq. bonds);
* the Gronbech-Jensen-Farago Langevin integrator (named in the Integrator
  Class list and used by Listing infile), with Philox4x32-10 random numbers
  and Box-Muller normals, and the two other integrators of that list:
  Euler-Maruyama and velocity-Verlet with a Langevin thermostat force.

Readings where the paper is silent are listed with each function.
Everything here is FP64; the only library primitives are numpy's FFT and
``bincount``.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, Optional

import numpy as np

# ---------------------------------------------------------------------------
# Periodic box
# ---------------------------------------------------------------------------


def wrap(x: np.ndarray, L: float) -> np.ndarray:
    """Map coordinates into [0, L). A value that rounds to L maps to 0."""
    y = x - L * np.floor(x / L)
    return np.where(y >= L, 0.0, y)


def minimum_image(d: np.ndarray, L: float) -> np.ndarray:
    """Minimum-image displacement in a cubic periodic box of edge L.

    Reading: the paper does not say how bonds that cross the boundary are
    measured; bonds are much shorter than L/2, so the minimum image is the
    bond vector.
    """
    return d - L * np.round(d / L)


# ---------------------------------------------------------------------------
# Assignment weights (Sec. "Long-range interactions": spline weights from the
# appendix of Deserno & Holm 1998, orders 1..4; Fig. pmm: order 1 uses the
# two nearest grid points per dimension)
# ---------------------------------------------------------------------------


def cardinal_bspline(x: np.ndarray, P: int) -> np.ndarray:
    """Cardinal B-spline M_P(x), the P-fold convolution of the unit box on [0, 1).

    Cox-de Boor recursion: M_1 = 1 on [0, 1);
    M_P(x) = (x M_{P-1}(x) + (P - x) M_{P-1}(x - 1)) / (P - 1).
    """
    x = np.asarray(x, dtype=np.float64)
    if P == 1:
        return ((x >= 0.0) & (x < 1.0)).astype(np.float64)
    return (x * cardinal_bspline(x, P - 1) + (P - x) * cardinal_bspline(x - 1.0, P - 1)) / (P - 1)


def cardinal_bspline_derivative(x: np.ndarray, P: int) -> np.ndarray:
    """dM_P/dx = M_{P-1}(x) - M_{P-1}(x - 1)  (P >= 2)."""
    return cardinal_bspline(x, P - 1) - cardinal_bspline(x - 1.0, P - 1)


def stencil(s: np.ndarray, P: int):
    """Grid points and weights along one axis for positions s in grid units.

    The Deserno-Holm charge-assignment function of order P is the centred
    cardinal B-spline W(t) = M_P(t + P/2); a particle at s gives grid point j
    the weight W(s - j). Its support |s - j| < P/2 holds P points, the first
    being floor(s - P/2) + 1. Returns (j, w) with shape (len(s), P); j is
    not yet reduced modulo the grid size.
    """
    j0 = np.floor(s - P / 2.0).astype(np.int64) + 1
    j = j0[:, None] + np.arange(P, dtype=np.int64)[None, :]
    w = cardinal_bspline(s[:, None] - j + P / 2.0, P)
    return j, w


def stencil_derivative(s: np.ndarray, P: int):
    """Same points as ``stencil``; d W(s - j) / d s (grid units)."""
    j, _ = stencil(s, P)
    dw = cardinal_bspline_derivative(s[:, None] - j + P / 2.0, P)
    return j, dw


# ---------------------------------------------------------------------------
# System description
# ---------------------------------------------------------------------------


@dataclasses.dataclass
class Model:
    """Parameters of one TILD system (reduced units).

    chi: S x S symmetric matrix with zero diagonal (Eq. fh generalised to S
    species pairs). rho0 = total bead number density N_b / V (Eq. HelfandP,
    rho_0 = nN/V). a: smearing width of h, sigma^2 = 2 a^2 (Eqs. fhF/HelfandF).
    """

    L: float
    n: int
    P: int
    species: np.ndarray          # (N_b,) int
    n_species: int
    bonds: np.ndarray            # (n_bonds, 2) int
    b: float
    chi: np.ndarray              # (S, S)
    kappa: float
    a: float
    dt: float = 0.005
    friction: float = 1.0
    kT: float = 1.0
    mass: float = 1.0
    seed: int = 0
    # electrostatics (Sec. "Long-range interactions"; charges smeared over a
    # unit Gaussian): charge per species in units of e, Bjerrum length l_B
    # (0: none) and charge spreading length a_e
    charges: Optional[np.ndarray] = None
    bjerrum: float = 0.0
    charge_smear: float = 0.5
    # dimensionality D (Sec. "TILD Branch": two- or three-dimensional
    # periodic boxes; Listing infile runs D = 2): positions are (N, D), grids
    # n^D, cell volume dx^D, and u_G the unit Gaussian in D dimensions
    dim: int = 3

    @property
    def n_beads(self) -> int:
        return int(self.species.shape[0])

    @property
    def dx(self) -> float:
        return self.L / self.n

    @property
    def volume(self) -> float:
        return self.L ** self.dim

    @property
    def rho0(self) -> float:
        return self.n_beads / self.volume

    def eps(self) -> np.ndarray:
        """Pair matrix of U_nb = 1/2 sum_KK' eps_KK' int int rho_K u_G rho_K'.

        Expanding Eq. fh plus Eq. HelfandP (rho_+ = sum_K rho_K) gives
        eps_KK' = (chi_KK' + kappa) / rho0 with chi_KK = 0, up to a constant.
        """
        S = self.n_species
        chi = np.zeros((S, S))
        chi[: self.chi.shape[0], : self.chi.shape[1]] = self.chi[:S, :S]
        return (chi + self.kappa) / self.rho0


def model_from_spec(spec, species: np.ndarray, bonds: np.ndarray) -> Model:
    """Build a Model from an input-generator SystemSpec (duck-typed)."""
    S = 2 if int(species.max(initial=0)) >= 1 else 1
    chi = np.zeros((S, S))
    if S == 2:
        chi[0, 1] = chi[1, 0] = spec.chi
    return Model(L=spec.L, n=spec.n, P=spec.pmeorder + 1, species=species.astype(np.int64), n_species=S,
                 bonds=bonds.astype(np.int64), b=spec.b, chi=chi, kappa=spec.kappa, a=spec.a, dt=spec.dt,
                 friction=spec.friction, kT=spec.kT, mass=spec.mass, seed=spec.dyn_seed)


# ---------------------------------------------------------------------------
# Wavevectors
# ---------------------------------------------------------------------------


def wavenumbers(n: int, L: float) -> np.ndarray:
    """k = 2 pi m / L with m in {0, .., n/2-1, -n/2, .., -1} (numpy FFT order)."""
    m = np.fft.fftfreq(n, d=1.0 / n)
    return 2.0 * np.pi * m / L


def gradient_wavenumbers(n: int, L: float) -> np.ndarray:
    """Wavenumbers for spectral differentiation: the Nyquist entry (m = -n/2,
    even n) is set to zero so that the derivative of a real field stays real.
    """
    k = wavenumbers(n, L).copy()
    if n % 2 == 0:
        k[n // 2] = 0.0
    return k


def _k2(n: int, L: float, dim: int) -> np.ndarray:
    """|k|^2 on the n^dim grid of wavevectors, axes (x, y[, z])."""
    k = wavenumbers(n, L)
    if dim == 2:
        return k[:, None] ** 2 + k[None, :] ** 2
    return k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2


def gaussian_kernel_hat(n: int, L: float, a: float, dim: int = 3) -> np.ndarray:
    """u_hat(k) = exp(-|k|^2 sigma^2 / 2) = exp(-|k|^2 a^2): the continuous
    Fourier transform of the unit Gaussian u_G (Eq. fh; normalised to unit
    integral in D dimensions) with sigma^2 = 2 a^2; u_hat(0) = 1 in any D.
    Axes (x, y[, z])."""
    return np.exp(-_k2(n, L, dim) * a * a)


def coulomb_kernel_hat(n: int, L: float, lb: float, ae: float) -> np.ndarray:
    """Fourier transform of the Coulomb interaction l_B / r between two
    charges each smeared over a unit Gaussian of width a_e (variance a_e^2
    per axis): 4 pi l_B exp(-|k|^2 a_e^2) / |k|^2, and 0 at k = 0 (the
    neutralising background of a periodic box). Axes (x, y, z). Reading:
    the paper gives the Bjerrum length and the charge spreading length but
    no formula; this is the standard smeared-charge Coulomb kernel with the
    same smearing convention as the pair kernel."""
    k = wavenumbers(n, L)
    k2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2
    out = np.zeros_like(k2)
    nz = k2 > 0
    out[nz] = 4.0 * np.pi * lb * np.exp(-k2[nz] * ae * ae) / k2[nz]
    return out


def _has_charges(m: "Model") -> bool:
    return m.bjerrum > 0 and m.charges is not None and np.any(np.asarray(m.charges) != 0)


# ---------------------------------------------------------------------------
# Particle-to-mesh
# ---------------------------------------------------------------------------


def spread(m: Model, pos: np.ndarray) -> np.ndarray:
    """Grid densities rho_K(g) = (1/dV) sum_{i in K} prod_d W(s_id - g_d)
    (Eq. rhohat assigned with the spline weights). Array axes (K, x, y[, z])."""
    if m.dim == 2:
        return _spread_2d(m, pos)
    n, P = m.n, m.P
    s = wrap(pos, m.L) / m.dx
    jx, wx = stencil(s[:, 0], P)
    jy, wy = stencil(s[:, 1], P)
    jz, wz = stencil(s[:, 2], P)
    rho = np.zeros((m.n_species, n * n * n))
    for K in range(m.n_species):
        sel = m.species == K
        for a in range(P):
            for b in range(P):
                for c in range(P):
                    flat = ((jx[sel, a] % n) * n + (jy[sel, b] % n)) * n + (jz[sel, c] % n)
                    w = wx[sel, a] * wy[sel, b] * wz[sel, c]
                    rho[K] += np.bincount(flat, weights=w, minlength=n ** 3)
    return rho.reshape(m.n_species, n, n, n) / m.dx ** 3


def _spread_2d(m: Model, pos: np.ndarray) -> np.ndarray:
    """spread for D = 2: rho_K(g) = (1/dA) sum_{i in K} W(s_ix - g_x) W(s_iy - g_y)."""
    n, P = m.n, m.P
    s = wrap(pos[:, :2], m.L) / m.dx
    jx, wx = stencil(s[:, 0], P)
    jy, wy = stencil(s[:, 1], P)
    rho = np.zeros((m.n_species, n * n))
    for K in range(m.n_species):
        sel = m.species == K
        for a in range(P):
            for b in range(P):
                flat = (jx[sel, a] % n) * n + (jy[sel, b] % n)
                rho[K] += np.bincount(flat, weights=wx[sel, a] * wy[sel, b], minlength=n * n)
    return rho.reshape(m.n_species, n, n) / m.dx ** 2


def gather(m: Model, pos: np.ndarray, field: np.ndarray, which: Optional[np.ndarray] = None) -> np.ndarray:
    """Interpolate per-species grid vectors field[K, d, x, y, z] to the beads
    with the same weights as ``spread`` (caption of Fig. pmm). Returns (N, D)."""
    idx = np.arange(m.n_beads) if which is None else np.asarray(which)
    n, P = m.n, m.P
    if m.dim == 2:
        s = wrap(pos[idx, :2], m.L) / m.dx
        jx, wx = stencil(s[:, 0], P)
        jy, wy = stencil(s[:, 1], P)
        K = m.species[idx]
        out = np.zeros((len(idx), field.shape[1]))
        for a in range(P):
            for b in range(P):
                w = wx[:, a] * wy[:, b]
                for d in range(field.shape[1]):
                    out[:, d] += w * field[K, d, jx[:, a] % n, jy[:, b] % n]
        return out
    s = wrap(pos[idx], m.L) / m.dx
    jx, wx = stencil(s[:, 0], P)
    jy, wy = stencil(s[:, 1], P)
    jz, wz = stencil(s[:, 2], P)
    K = m.species[idx]
    D = field.shape[1]
    out = np.zeros((len(idx), D))
    for a in range(P):
        for b in range(P):
            for c in range(P):
                w = wx[:, a] * wy[:, b] * wz[:, c]
                gx, gy, gz = jx[:, a] % n, jy[:, b] % n, jz[:, c] % n
                for d in range(D):
                    out[:, d] += w * field[K, d, gx, gy, gz]
    return out


def potential_fields(m: Model, rho: np.ndarray) -> Dict[str, np.ndarray]:
    """Spectral evaluation of Eq. PMM for the smeared pair kernel.

    rho_hat_K(k) = sum_g rho_K(g) exp(-i k.g)          (unnormalised DFT)
    w_hat_K(k)   = u_hat(k) sum_K' eps_KK' rho_hat_K'(k)
    w_K(g)       = (1/M) sum_k w_hat_K(k) exp(i k.g)      (potential field)
    grad w_K(g)  = (1/M) sum_k i k~ w_hat_K(k) exp(i k.g) (k~: Nyquist zeroed)

    The continuum convolution int u(r - r') rho(r') dr' becomes this sum
    because the Fourier coefficient of rho is dV * rho_hat and V = M dV.
    """
    n, L, D = m.n, m.L, m.dim
    axes = tuple(range(1, D + 1))
    rho_hat = np.fft.fftn(rho, axes=axes)
    u_hat = gaussian_kernel_hat(n, L, m.a, D)
    eps = m.eps()
    w_hat = np.einsum("kl,l...->k...", eps, rho_hat) * u_hat[None]
    if _has_charges(m) and D != 3:
        raise NotImplementedError("electrostatics: three dimensions only")
    if _has_charges(m):
        # electrostatic potential phi = l_B (1/r * h_e * h_e * rho_q): w_K += q_K phi
        q = np.asarray(m.charges, dtype=float)[: m.n_species]
        rho_q_hat = np.einsum("l,l...->...", q, rho_hat)
        w_hat = w_hat + q[:, None, None, None] * (coulomb_kernel_hat(n, L, m.bjerrum, m.charge_smear) * rho_q_hat)[None]
    kt = gradient_wavenumbers(n, L)
    if D == 2:
        kvec = (kt[:, None], kt[None, :])
    else:
        kvec = (kt[:, None, None], kt[None, :, None], kt[None, None, :])
    grad = np.empty((m.n_species, D) + (n,) * D)
    for K in range(m.n_species):
        for d in range(D):
            grad[K, d] = np.fft.ifftn(1j * kvec[d] * w_hat[K]).real
    w = np.fft.ifftn(w_hat, axes=axes).real
    return {"rho_hat": rho_hat, "w_hat": w_hat, "w": w, "grad_w": grad, "u_hat": u_hat}


# ---------------------------------------------------------------------------
# Energies (Eqs. bonds, fh, HelfandP) and forces
# ---------------------------------------------------------------------------


def bond_vectors(m: Model, pos: np.ndarray) -> np.ndarray:
    return minimum_image(pos[m.bonds[:, 0]] - pos[m.bonds[:, 1]], m.L)


def bond_energy(m: Model, pos: np.ndarray) -> float:
    """beta U_0 = (3 / 2b^2) sum_bonds |r_i - r_j|^2  (Eq. bonds). Reading: the
    equation has the factor 3/2b^2 with no dimension in it; it is kept as
    written in two dimensions too."""
    d = bond_vectors(m, pos)
    return float(1.5 / m.b ** 2 * np.sum(d * d))


def bond_forces(m: Model, pos: np.ndarray) -> np.ndarray:
    """-dU_0/dr_i = -(3/b^2) sum_{j bonded to i} (r_i - r_j)."""
    d = bond_vectors(m, pos)
    f = np.zeros((m.n_beads, pos.shape[1]))
    k = 3.0 / m.b ** 2
    np.add.at(f, m.bonds[:, 0], -k * d)
    np.add.at(f, m.bonds[:, 1], k * d)
    return f


def field_energies(m: Model, rho_hat: np.ndarray) -> Dict[str, float]:
    """Flory and Helfand energies from the density spectra (Parseval).

    With rho'_K(k) = dV rho_hat_K(k) (Fourier coefficients of the gridded
    density) the periodic double integrals of Eqs. fh and HelfandP become
      E_chi   = sum_{K<K'} (chi_KK'/rho0) (1/V) sum_k u_hat Re[conj(rho'_K) rho'_K'],
      E_kappa = (kappa / 2 rho0) (1/V) sum_{k != 0} u_hat |sum_K rho'_K|^2.
    The k = 0 Helfand term cancels the -rho0 shift exactly because the
    weights conserve mass (reading: E_chi keeps k = 0 as Eq. fh does).
    """
    dV = m.dx ** m.dim
    V = m.volume
    u_hat = gaussian_kernel_hat(m.n, m.L, m.a, m.dim)
    rp = dV * rho_hat
    e_chi = 0.0
    for K in range(m.n_species):
        for Kp in range(K + 1, m.n_species):
            chi = m.chi[K, Kp] if K < m.chi.shape[0] and Kp < m.chi.shape[1] else 0.0
            e_chi += chi / m.rho0 / V * float(np.sum(u_hat * np.real(np.conj(rp[K]) * rp[Kp])))
    tot = rp.sum(axis=0)
    p = u_hat * np.abs(tot) ** 2
    p[(0,) * m.dim] = 0.0
    e_kappa = m.kappa / (2.0 * m.rho0) / V * float(np.sum(p))
    out = {"chi": e_chi, "kappa": e_kappa, "elec": 0.0}
    if _has_charges(m):
        # E_el = (1/2V) sum_k c(k) |rho'_q(k)|^2, rho_q = sum_K q_K rho_K
        q = np.asarray(m.charges, dtype=float)[: m.n_species]
        rq = np.einsum("l,l...->...", q, rp)
        c = coulomb_kernel_hat(m.n, m.L, m.bjerrum, m.charge_smear)
        out["elec"] = 0.5 / V * float(np.sum(c * np.abs(rq) ** 2))
    return out


def nonbonded_forces(m: Model, pos: np.ndarray, variant: str = "ik") -> np.ndarray:
    """Particle-mesh force of Eq. PMM.

    variant "ik" (the method): F_i = -sum_g W(r_i - g) grad w_K(g), the
    spectral gradient interpolated with the assignment weights.
    variant "analytic": F_i = -sum_g grad_r W(r_i - g) w_K(g), the exact
    gradient of the gridded energy (used to check forces against finite
    differences of the energy).
    """
    rho = spread(m, pos)
    f = potential_fields(m, rho)
    if variant == "ik":
        return -gather(m, pos, f["grad_w"])
    if variant != "analytic":
        raise ValueError(variant)
    n, P, dx = m.n, m.P, m.dx
    if m.dim == 2:
        s = wrap(pos[:, :2], m.L) / dx
        jx, wx = stencil(s[:, 0], P)
        jy, wy = stencil(s[:, 1], P)
        _, dwx = stencil_derivative(s[:, 0], P)
        _, dwy = stencil_derivative(s[:, 1], P)
        wf = f["w"][m.species]
        out = np.zeros((m.n_beads, 2))
        rows = np.arange(m.n_beads)
        for a in range(P):
            for b in range(P):
                val = wf[rows, jx[:, a] % n, jy[:, b] % n]
                out[:, 0] -= dwx[:, a] / dx * wy[:, b] * val
                out[:, 1] -= wx[:, a] * dwy[:, b] / dx * val
        return out
    s = wrap(pos, m.L) / dx
    js, ws, dws = [], [], []
    for d in range(3):
        j, w = stencil(s[:, d], P)
        _, dw = stencil_derivative(s[:, d], P)
        js.append(j % n)
        ws.append(w)
        dws.append(dw / dx)
    w_field = f["w"][m.species]
    out = np.zeros((m.n_beads, 3))
    rows = np.arange(m.n_beads)
    for a in range(P):
        for b in range(P):
            for c in range(P):
                val = w_field[rows, js[0][:, a], js[1][:, b], js[2][:, c]]
                out[:, 0] -= dws[0][:, a] * ws[1][:, b] * ws[2][:, c] * val
                out[:, 1] -= ws[0][:, a] * dws[1][:, b] * ws[2][:, c] * val
                out[:, 2] -= ws[0][:, a] * ws[1][:, b] * dws[2][:, c] * val
    return out


def forces(m: Model, pos: np.ndarray, variant: str = "ik") -> np.ndarray:
    return nonbonded_forces(m, pos, variant) + bond_forces(m, pos)


def energies(m: Model, pos: np.ndarray) -> Dict[str, float]:
    rho = spread(m, pos)
    e = field_energies(m, np.fft.fftn(rho, axes=tuple(range(1, m.dim + 1))))
    e["bond"] = bond_energy(m, pos)
    return e


# ---------------------------------------------------------------------------
# Random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) and
# Box-Muller normals. Counter (bead id, step lo, step hi, 0), key (seed lo,
# seed hi). Reading: the paper says only that GJF draws its thermal noise
# internally; any such generator defines a different (equally valid)
# trajectory, so this choice is part of the definition of parity.
# ---------------------------------------------------------------------------

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint32(0x9E3779B9)
_W1 = np.uint32(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox-4x32 rounds. All arguments uint32 arrays (broadcastable)."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint32) for v in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64)
    k1 = np.asarray(k1, dtype=np.uint64)
    for r in range(10):
        if r > 0:  # key schedule: add the Weyl constants modulo 2^32
            k0 = (k0 + np.uint64(_W0)) & _MASK
            k1 = (k1 + np.uint64(_W1)) & _MASK
        p0 = _M0 * c0.astype(np.uint64)
        p1 = _M1 * c2.astype(np.uint64)
        hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
        lo0 = (p0 & _MASK).astype(np.uint32)
        hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
        lo1 = (p1 & _MASK).astype(np.uint32)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0.astype(np.uint32), lo1, hi0 ^ c3 ^ k1.astype(np.uint32), lo0
    return c0, c1, c2, c3


def gaussian_triplets(ids: np.ndarray, step: int, seed: int) -> np.ndarray:
    """Three standard normals per bead id from one Philox block.

    u_j = (x_j + 1/2) 2^-32 in (0, 1); (n0, n1) = Box-Muller(u0, u1),
    n2 = sqrt(-2 ln u2) cos(2 pi u3). step is taken modulo 2^64.
    """
    step = int(step) % (1 << 64)
    ids = np.asarray(ids, dtype=np.uint64)
    x = philox4x32_10(ids & _MASK, np.uint32(step & 0xFFFFFFFF), np.uint32(step >> 32), np.uint32(0),
                      np.uint32(seed & 0xFFFFFFFF), np.uint32((seed >> 32) & 0xFFFFFFFF))
    u = [(xi.astype(np.float64) + 0.5) * 2.0 ** -32 for xi in x]
    r1 = np.sqrt(-2.0 * np.log(u[0]))
    r2 = np.sqrt(-2.0 * np.log(u[2]))
    return np.stack([r1 * np.cos(2 * np.pi * u[1]), r1 * np.sin(2 * np.pi * u[1]),
                     r2 * np.cos(2 * np.pi * u[3])], axis=1)


VELOCITY_INIT_STEP = (1 << 64) - 1


# ---------------------------------------------------------------------------
# Gronbech-Jensen-Farago integrator (Mol. Phys. 111, 983 (2013))
# ---------------------------------------------------------------------------


@dataclasses.dataclass
class State:
    pos: np.ndarray      # (N, 3) wrapped positions r^n
    vel: np.ndarray      # (N, 3) velocities v^n
    force: np.ndarray    # (N, 3) total force F^n = F(r^n)
    step: int            # n


def initial_state(m: Model, pos: np.ndarray, force_fn=None) -> State:
    """v^0 ~ N(0, kT/m) per component (Philox block at step 2^64-1);
    F^0 evaluated at r^0. ``force_fn(m, pos)`` defaults to ``forces``."""
    force_fn = forces if force_fn is None else force_fn
    ids = np.arange(m.n_beads)
    vel = np.sqrt(m.kT / m.mass) * gaussian_triplets(ids, VELOCITY_INIT_STEP, m.seed)[:, : m.dim]
    p = wrap(pos, m.L)
    return State(p, vel, force_fn(m, p), 0)


def gjf_step(m: Model, st: State, force_fn=None) -> State:
    """One GJF step:
      r^{n+1} = r^n + b dt v^n + (b dt^2 / 2m) F^n + (b dt / 2m) beta^{n+1}
      v^{n+1} = a v^n + (dt / 2m)(a F^n + F^{n+1}) + (b / m) beta^{n+1}
    with a = (1 - alpha dt/2m)/(1 + alpha dt/2m), b = 1/(1 + alpha dt/2m) and
    beta^{n+1} ~ N(0, 2 alpha kT dt) per component (drawn with counter step
    n+1). alpha is the friction coefficient.
    """
    dt, mass, alpha = m.dt, m.mass, m.friction
    ga = (1.0 - alpha * dt / (2 * mass)) / (1.0 + alpha * dt / (2 * mass))
    gb = 1.0 / (1.0 + alpha * dt / (2 * mass))
    beta = np.sqrt(2.0 * alpha * m.kT * dt) * gaussian_triplets(np.arange(m.n_beads), st.step + 1, m.seed)[:, : m.dim]
    r_new = st.pos + gb * dt * st.vel + gb * dt * dt / (2 * mass) * st.force + gb * dt / (2 * mass) * beta
    r_new = wrap(r_new, m.L)
    f_new = (forces if force_fn is None else force_fn)(m, r_new)
    v_new = ga * st.vel + dt / (2 * mass) * (ga * st.force + f_new) + gb / mass * beta
    return State(r_new, v_new, f_new, st.step + 1)


def run(m: Model, st: State, n_steps: int, force_fn=None) -> State:
    for _ in range(n_steps):
        st = gjf_step(m, st, force_fn)
    return st


def kinetic_energy(m: Model, vel: np.ndarray) -> float:
    return float(0.5 * m.mass * np.sum(vel * vel))


# ---------------------------------------------------------------------------
# The other integrators of the Integrator Class list (Sec. "Integrator
# Class"): Euler-Maruyama (EM) and velocity-Verlet (VV) coupled to the
# Langevin thermostat force of the ExtraForce list.
# ---------------------------------------------------------------------------


def em_step(m: Model, st: State, force_fn=None) -> State:
    """One Euler-Maruyama step of overdamped Langevin (Brownian) dynamics:
      r^{n+1} = r^n + (dt / alpha) F^n + sqrt(2 kT dt / alpha) xi^{n+1}
    with xi^{n+1} ~ N(0, 1) per component (counter step n+1) and alpha the
    friction coefficient. Reading: the paper names EM as the scheme that
    draws its noise during the update; for particles that is the EM
    discretisation of dr = F/alpha dt + sqrt(2 kT/alpha) dW. There is no
    velocity in this dynamics; ``vel`` stays zero.
    """
    dt, alpha = m.dt, m.friction
    xi = gaussian_triplets(np.arange(m.n_beads), st.step + 1, m.seed)[:, : m.dim]
    r_new = wrap(st.pos + dt / alpha * st.force + np.sqrt(2.0 * m.kT * dt / alpha) * xi, m.L)
    f_new = (forces if force_fn is None else force_fn)(m, r_new)
    return State(r_new, np.zeros_like(st.vel), f_new, st.step + 1)


def em_initial_state(m: Model, pos: np.ndarray, force_fn=None) -> State:
    force_fn = forces if force_fn is None else force_fn
    p = wrap(pos, m.L)
    return State(p, np.zeros((m.n_beads, m.dim)), force_fn(m, p), 0)


def langevin_force(m: Model, v_half: np.ndarray, step: int) -> np.ndarray:
    """Langevin thermostat force of step n: -alpha v + sqrt(2 alpha kT / dt)
    xi^n, xi^n ~ N(0, 1) per component (counter step n). Reading: the force
    acts on the half-step velocity v^{n-1/2} = v^n - (dt/2m) F^n, the
    velocity a velocity-Verlet step holds when forces are evaluated."""
    sigma = np.sqrt(2.0 * m.friction * m.kT / m.dt)
    return -m.friction * v_half + sigma * gaussian_triplets(np.arange(m.n_beads), step, m.seed)[:, : m.dim]


def vv_initial_state(m: Model, pos: np.ndarray, vel: np.ndarray, force_fn=None, step: int = 0) -> State:
    """Velocity-Verlet state at step n (default 0) from r^n, v^n. F^n =
    F_c(r^n) + Langevin force on v^{n-1/2} = v^n - (dt/2m) F^n, which is
    linear in F^n:
      v^{n-1/2} = (v^n - (dt/2m)(F_c + sigma xi^n)) / (1 - alpha dt/2m)."""
    force_fn = forces if force_fn is None else force_fn
    p = wrap(pos, m.L)
    fc = force_fn(m, p)
    h = m.dt / (2.0 * m.mass)
    noise = langevin_force(m, np.zeros_like(vel), step)
    v_half = (vel - h * (fc + noise)) / (1.0 - m.friction * h)
    return State(p, vel.copy(), fc + langevin_force(m, v_half, step), step)


def vv_step(m: Model, st: State, force_fn=None) -> State:
    """One velocity-Verlet step with the Langevin force (friction alpha,
    temperature kT; alpha = 0 gives plain NVE velocity-Verlet):
      v^{n+1/2} = v^n + (dt/2m) F^n
      r^{n+1}   = r^n + dt v^{n+1/2}
      F^{n+1}   = F_c(r^{n+1}) - alpha v^{n+1/2} + sqrt(2 alpha kT/dt) xi^{n+1}
      v^{n+1}   = v^{n+1/2} + (dt/2m) F^{n+1}
    """
    h = m.dt / (2.0 * m.mass)
    v_half = st.vel + h * st.force
    r_new = wrap(st.pos + m.dt * v_half, m.L)
    f_new = (forces if force_fn is None else force_fn)(m, r_new) + langevin_force(m, v_half, st.step + 1)
    return State(r_new, v_half + h * f_new, f_new, st.step + 1)


def run_with(step_fn, m: Model, st: State, n_steps: int, force_fn=None) -> State:
    for _ in range(n_steps):
        st = step_fn(m, st, force_fn)
    return st


# ---------------------------------------------------------------------------
# Differentiable form: vector-Jacobian product of the density assignment
# ---------------------------------------------------------------------------


def spread_vjp(m: Model, pos: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """d/dr_i of sum_{K,g} psi_K(g) rho_K(g) for a grid adjoint psi with the
    axes of ``spread`` (K, x, y, z): Eq. rhohat with the spline weights
    differentiated, (1/dV) sum_g grad_r W(r_i - g) psi_{K_i}(g). (N, 3)."""
    n, P, dx = m.n, m.P, m.dx
    s = wrap(pos, m.L) / dx
    js, ws, dws = [], [], []
    for d in range(3):
        j, w = stencil(s[:, d], P)
        _, dw = stencil_derivative(s[:, d], P)
        js.append(j % n)
        ws.append(w)
        dws.append(dw / dx)
    field = psi[m.species]
    rows = np.arange(m.n_beads)
    out = np.zeros((m.n_beads, 3))
    for a in range(P):
        for b in range(P):
            for c in range(P):
                v = field[rows, js[0][:, a], js[1][:, b], js[2][:, c]]
                out[:, 0] += dws[0][:, a] * ws[1][:, b] * ws[2][:, c] * v
                out[:, 1] += ws[0][:, a] * dws[1][:, b] * ws[2][:, c] * v
                out[:, 2] += ws[0][:, a] * ws[1][:, b] * dws[2][:, c] * v
    return out / dx ** 3


# ---------------------------------------------------------------------------
# Differentiable form: vector-Jacobian product of the ik force
# ---------------------------------------------------------------------------


def force_vjp(m: Model, pos: np.ndarray, lam: np.ndarray) -> Dict[str, object]:
    """J^T lam for the ik particle-mesh + bond force F(r; chi, kappa, a):
    d/dr_j of sum_i lam_i . F_i, and the derivatives of sum_i lam_i . F_i with
    respect to chi, kappa and a.

    With W_i(g) = W(r_i - g), mu_K(g) = sum_{i in K} W_i(g) lam_i, C the
    convolution with the smeared kernel (u_hat), D the i k~ derivative (anti-
    self-adjoint; Nyquist zeroed) and psi_K = sum_K' eps_KK' C (D . mu_K'):
      (J^T lam)_j = - sum_g grad W_j(g) (lam_j . D w_{K_j})(g)
                    + (1/dV) sum_g grad W_j(g) psi_{K_j}(g)
                    - (3/b^2) sum_{i ~ j} (lam_j - lam_i),
      d/dchi   = sum_K sum_g (D . mu_K)(g) dw_K/dchi(g)  (dw_A/dchi = C rho_B / rho0),
      d/dkappa = ... with dw_K/dkappa = C (rho_A + rho_B) / rho0,
      d/da     = ... with dw_K/da = sum_K' eps_KK' C_a rho_K', C_a: -2 a |k|^2 u_hat.
    Charges add their Coulomb term to C for the position part (the parameter
    part covers chi, kappa, a only)."""
    n, L, P, dx = m.n, m.L, m.P, m.dx
    S = m.n_species
    rho = spread(m, pos)
    f = potential_fields(m, rho)
    s = wrap(pos, L) / dx
    js, ws, dws = [], [], []
    for d in range(3):
        j, w = stencil(s[:, d], P)
        _, dw = stencil_derivative(s[:, d], P)
        js.append(j % n)
        ws.append(w)
        dws.append(dw / dx)
    # mu_K (vector field per species, no 1/dV)
    mu = np.zeros((S, 3, n * n * n))
    for a in range(P):
        for b in range(P):
            for c in range(P):
                flat = (js[0][:, a] * n + js[1][:, b]) * n + js[2][:, c]
                w = ws[0][:, a] * ws[1][:, b] * ws[2][:, c]
                for K in range(S):
                    sel = m.species == K
                    for d in range(3):
                        mu[K, d] += np.bincount(flat[sel], weights=w[sel] * lam[sel, d], minlength=n ** 3)
    mu = mu.reshape(S, 3, n, n, n)
    kt = gradient_wavenumbers(n, L)
    kvec = (kt[:, None, None], kt[None, :, None], kt[None, None, :])
    div_hat = np.zeros((S, n, n, n), dtype=complex)  # DFT of D . mu_K
    for K in range(S):
        for d in range(3):
            div_hat[K] += 1j * kvec[d] * np.fft.fftn(mu[K, d])
    u_hat = f["u_hat"]
    kernel = m.eps()[:, :, None, None, None] * u_hat[None, None]
    if _has_charges(m):
        q = np.asarray(m.charges, dtype=float)[:S]
        kernel = kernel + q[:, None, None, None, None] * q[None, :, None, None, None] * \
            coulomb_kernel_hat(n, L, m.bjerrum, m.charge_smear)[None, None]
    psi = np.fft.ifftn(np.einsum("kl...,l...->k...", kernel, div_hat), axes=(1, 2, 3)).real
    dV = dx ** 3
    # lam_j . D w_{K_j} at every grid point, per bead
    gw = f["grad_w"]  # (S, 3, n, n, n)
    out = np.zeros((m.n_beads, 3))
    rows = np.arange(m.n_beads)
    K = m.species
    for a in range(P):
        for b in range(P):
            for c in range(P):
                gx, gy, gz = js[0][:, a], js[1][:, b], js[2][:, c]
                ldw = sum(lam[:, d] * gw[K, d, gx, gy, gz] for d in range(3))
                val = psi[K, gx, gy, gz] / dV - ldw
                out[:, 0] += dws[0][:, a] * ws[1][:, b] * ws[2][:, c] * val
                out[:, 1] += ws[0][:, a] * dws[1][:, b] * ws[2][:, c] * val
                out[:, 2] += ws[0][:, a] * ws[1][:, b] * dws[2][:, c] * val
    # bonds
    kb = 3.0 / m.b ** 2
    dl = lam[m.bonds[:, 0]] - lam[m.bonds[:, 1]]
    np.add.at(out, m.bonds[:, 0], -kb * dl)
    np.add.at(out, m.bonds[:, 1], kb * dl)
    # parameters (Parseval: sum_g f h = (1/M) sum_k conj(f~) h~ for real f, h)
    M = n ** 3
    rho_hat = f["rho_hat"]
    k = wavenumbers(n, L)
    k2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2
    out_t = {"chi": 0.0, "kappa": 0.0, "a": 0.0}
    if S == 2:
        out_t["chi"] = float(np.real(np.sum(np.conj(div_hat[0]) * u_hat * rho_hat[1] +
                                            np.conj(div_hat[1]) * u_hat * rho_hat[0]))) / (m.rho0 * M)
    tot = rho_hat.sum(axis=0)
    out_t["kappa"] = float(np.real(np.sum(np.conj(div_hat.sum(axis=0)) * u_hat * tot))) / (m.rho0 * M)
    eps_rho = np.einsum("kl,l...->k...", m.eps(), rho_hat)
    out_t["a"] = float(np.real(np.sum(np.conj(div_hat) * (-2.0 * m.a * k2 * u_hat)[None] * eps_rho))) / M
    return {"r": out, **out_t}


def gjf_trajectory_vjp(m: Model, pos0: np.ndarray, vel0: np.ndarray, n_steps: int, r_bar: np.ndarray,
                       v_bar: Optional[np.ndarray] = None) -> Dict[str, object]:
    """Reverse-mode derivative of L(r^K, v^K) through K GJF steps (noise held
    fixed: the same Philox counters), given dL/dr^K = r_bar and dL/dv^K =
    v_bar. Returns dL/dr^0, dL/dv^0 and dL/dchi, dL/dkappa, dL/da.

    One step maps (r, v, F) to (r', v', F') with F' = F(r') and
      r' = r + b dt v + (b dt^2/2m) F + (b dt/2m) beta,
      v' = a v + (dt/2m)(a F + F'),
    so with h = dt/2m its adjoint is
      Fb'_tot = Fb' + h vb',  rb'_tot = rb' + J(r')^T Fb'_tot,
      rb = rb'_tot,  vb = b dt rb'_tot + a vb',  Fb = (b dt^2/2m) rb'_tot + h a vb',
    and the parameters collect (dF/dtheta)(r')^T Fb'_tot at every step and at
    r^0 (F^0 = F(r^0))."""
    dt, mass, alpha = m.dt, m.mass, m.friction
    h = dt / (2 * mass)
    ga = (1.0 - alpha * h) / (1.0 + alpha * h)
    gb = 1.0 / (1.0 + alpha * h)
    st = State(wrap(pos0, m.L), vel0.copy(), forces(m, wrap(pos0, m.L)), 0)
    traj = [st]
    for _ in range(n_steps):
        st = gjf_step(m, st)
        traj.append(st)
    rb = r_bar.copy()
    vb = np.zeros_like(rb) if v_bar is None else v_bar.copy()
    fb = np.zeros_like(rb)
    tb = {"chi": 0.0, "kappa": 0.0, "a": 0.0}
    for n in range(n_steps, 0, -1):
        ft = fb + h * vb
        v = force_vjp(m, traj[n].pos, ft)
        rt = rb + v["r"]
        for k in tb:
            tb[k] += v[k]
        rb, vb, fb = rt, gb * dt * rt + ga * vb, gb * dt * dt / (2 * mass) * rt + h * ga * vb
    v = force_vjp(m, traj[0].pos, fb)
    for k in tb:
        tb[k] += v[k]
    return {"r0": rb + v["r"], "v0": vb, **tb}



def em_trajectory_vjp(m: Model, pos0: np.ndarray, n_steps: int, r_bar: np.ndarray) -> Dict[str, object]:
    """Reverse-mode derivative of L(r^K) through K Euler-Maruyama steps (noise
    held fixed), given dL/dr^K = r_bar. One step is
      r' = r + (dt/alpha) F(r) + sqrt(2 kT dt/alpha) xi,
    so its adjoint is rb = rb' + J(r)^T ((dt/alpha) rb'), and the parameters
    collect (dF/dtheta)(r)^T ((dt/alpha) rb') at r^0 .. r^{K-1}. There is no
    velocity: dL/dv^0 is zero."""
    c = m.dt / m.friction
    st = em_initial_state(m, pos0)
    traj = [st]
    for _ in range(n_steps):
        st = em_step(m, st)
        traj.append(st)
    rb = r_bar.copy()
    tb = {"chi": 0.0, "kappa": 0.0, "a": 0.0}
    for n in range(n_steps - 1, -1, -1):
        v = force_vjp(m, traj[n].pos, c * rb)
        for k in tb:
            tb[k] += v[k]
        rb = rb + v["r"]
    return {"r0": rb, "v0": np.zeros_like(rb), **tb}


def vv_trajectory_vjp(m: Model, pos0: np.ndarray, vel0: np.ndarray, n_steps: int, r_bar: np.ndarray,
                      v_bar: Optional[np.ndarray] = None) -> Dict[str, object]:
    """Reverse-mode derivative of L(r^K, v^K) through K velocity-Verlet steps
    with the Langevin force (noise held fixed), given dL/dr^K = r_bar and
    dL/dv^K = v_bar. One step (see vv_step) maps (r, v, F) to (r', v', F'):
      vh = v + h F,  r' = r + dt vh,  F' = F_c(r') - alpha vh + s xi',
      v' = vh + h F',   h = dt/2m,
    so its adjoint is
      Fb'_tot = Fb' + h vb',  rb'_tot = rb' + J_c(r')^T Fb'_tot,
      vhb = vb' - alpha Fb'_tot + dt rb'_tot,  rb = rb'_tot,  vb = vhb,  Fb = h vhb.
    The initial force (see vv_initial_state) is
      F^0 = (F_c(r^0) - alpha v^0) / (1 - alpha h) + (terms in the noise),
    which closes the chain at r^0 with weight q = 1/(1 - alpha h). The
    parameters collect (dF_c/dtheta)^T of the same adjoint vectors."""
    h = m.dt / (2.0 * m.mass)
    al = m.friction
    st = vv_initial_state(m, pos0, vel0)
    traj = [st]
    for _ in range(n_steps):
        st = vv_step(m, st)
        traj.append(st)
    rb = r_bar.copy()
    vb = np.zeros_like(rb) if v_bar is None else v_bar.copy()
    fb = np.zeros_like(rb)
    tb = {"chi": 0.0, "kappa": 0.0, "a": 0.0}
    for n in range(n_steps, 0, -1):
        ft = fb + h * vb
        v = force_vjp(m, traj[n].pos, ft)
        for k in tb:
            tb[k] += v[k]
        rt = rb + v["r"]
        vhb = vb - al * ft + m.dt * rt
        rb, vb, fb = rt, vhb, h * vhb
    q = 1.0 / (1.0 - al * h)
    v = force_vjp(m, traj[0].pos, q * fb)
    for k in tb:
        tb[k] += v[k]
    return {"r0": rb + v["r"], "v0": vb - al * q * fb, **tb}