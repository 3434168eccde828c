"""Seeded synthetic inputs for TILD systems (shared by the CUDA path's tests,
the benchmark and the CPU oracle).

This module holds no arithmetic of the method itself: it only describes
systems (chain architectures, box, grid, interaction parameters) and draws
initial coordinates. Both the oracle and the GPU path receive the arrays it
returns.

System model (MATILDA.FT, arXiv 2302.02474, Sec. "Structure of
theoretically-informed coarse-grained and field-theoretic models"): linear
bead-spring chains of species A and B (Eq. rhohat), joined by harmonic bonds
of statistical segment length b (Eq. bonds).

Initial coordinates ("uniform random-walk chain initialisation"): the first
bead of every chain is uniform in the periodic box; each following bead sits
at distance exactly b from its predecessor along a direction uniform on the
sphere. Drawn with numpy's PCG64 in FP64 and wrapped into [0, L).
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence, Tuple

import numpy as np


@dataclasses.dataclass(frozen=True)
class MolType:
    """One molecule type: ``n_chains`` linear chains of ``N`` beads.

    ``n_a`` leading beads of each chain are species 0 (A); the remaining
    ``N - n_a`` are species 1 (B). ``n_a == N`` gives an A homopolymer and
    ``n_a == 0`` a B homopolymer.
    """

    n_chains: int
    N: int
    n_a: int


@dataclasses.dataclass(frozen=True)
class SystemSpec:
    """A complete TILD system description (all in reduced units kT=m=b=1)."""

    name: str
    moltypes: Tuple[MolType, ...]
    L: float            # cubic box edge
    n: int              # grid points per edge
    pmeorder: int       # assignment order p (p+1 stencil points per dimension)
    a: float            # Gaussian smearing width (sigma^2 = 2 a^2)
    chi: float          # Flory-Huggins chi between A and B
    kappa: float        # Helfand compressibility
    dt: float
    friction: float
    kT: float
    mass: float
    b: float            # statistical segment length (bond constant 3/b^2)
    steps: int          # length of the run the configuration is quoted for
    precision: str      # "fp32" or "fp64"
    input_seed: int
    dyn_seed: int

    @property
    def n_beads(self) -> int:
        return sum(m.n_chains * m.N for m in self.moltypes)

    @property
    def n_species(self) -> int:
        has_a = any(m.n_a > 0 and m.n_chains > 0 for m in self.moltypes)
        has_b = any(m.n_a < m.N and m.n_chains > 0 for m in self.moltypes)
        return 2 if (has_a and has_b) else 1 if has_a else 2

    def with_(self, **kw) -> "SystemSpec":
        return dataclasses.replace(self, **kw)


def config(name: str) -> SystemSpec:
    """Named workloads.

    ``diblock_20k_32``   AB diblock melt, 1,000 x A10-B10 (20,000 beads), L=20, 32^3, FP64.
    ``diblock_1p6M_128`` AB diblock melt, 80,000 x A8-B12 (1.6M beads), L=64, 128^3, FP32.
    ``blend_6p4M_256``   A/B homopolymer blend (N=32) + A16-B16 compatibiliser,
                         6.4M beads in 40/40/20 bead fractions, L=128, 256^3, FP32.
    ``diblock_200k_64``  AB diblock melt, 10,000 x A10-B10 (200,000 beads), L=32, 64^3.
    """
    if name == "diblock_20k_32":
        return SystemSpec(name, (MolType(1000, 20, 10),), 20.0, 32, 1, 0.5, 1.0, 20.0,
                          0.005, 1.0, 1.0, 1.0, 1.0, 100, "fp64", 12345 + 1, 777 + 1)
    if name == "diblock_1p6M_128":
        return SystemSpec(name, (MolType(80000, 20, 8),), 64.0, 128, 1, 0.5, 0.8, 25.0,
                          0.005, 1.0, 1.0, 1.0, 1.0, 10000, "fp32", 12345 + 2, 777 + 2)
    if name == "blend_6p4M_256":
        return SystemSpec(name, (MolType(80000, 32, 32), MolType(80000, 32, 0), MolType(40000, 32, 16)),
                          128.0, 256, 1, 0.6, 0.5, 30.0, 0.005, 1.0, 1.0, 1.0, 1.0, 2000, "fp32",
                          12345 + 3, 777 + 3)
    if name == "diblock_200k_64":
        return SystemSpec(name, (MolType(10000, 20, 10),), 32.0, 64, 1, 0.5, 1.0, 25.0,
                          0.005, 1.0, 1.0, 1.0, 1.0, 200, "fp32", 12345 + 4, 777 + 4)
    raise KeyError(name)


def small_system(n_chains: int = 40, N: int = 10, n_a: int = 4, L: float = 6.0, n: int = 12,
                 pmeorder: int = 1, precision: str = "fp64", chi: float = 1.3, kappa: float = 7.0,
                 a: float = 0.5, seed: int = 5, **kw) -> SystemSpec:
    """A small diblock melt for fast tests (ragged sizes allowed)."""
    base = SystemSpec("small", (MolType(n_chains, N, n_a),), float(L), int(n), int(pmeorder), float(a),
                      float(chi), float(kappa), 0.005, 1.0, 1.0, 1.0, 1.0, 10, precision, seed, seed + 1000)
    return base.with_(**kw) if kw else base


def species_of_beads(moltypes: Sequence[MolType]) -> np.ndarray:
    """Species index (0=A, 1=B) of every bead, beads numbered chain by chain."""
    out: List[np.ndarray] = []
    for m in moltypes:
        one = np.concatenate([np.zeros(m.n_a, np.int8), np.ones(m.N - m.n_a, np.int8)])
        out.append(np.tile(one, m.n_chains))
    return np.concatenate(out) if out else np.zeros(0, np.int8)


def bond_pairs(moltypes: Sequence[MolType]) -> np.ndarray:
    """(n_bonds, 2) int64 array of bonded bead pairs (i, i+1) along every chain."""
    out: List[np.ndarray] = []
    start = 0
    for m in moltypes:
        if m.N >= 2 and m.n_chains > 0:
            first = start + np.arange(m.n_chains, dtype=np.int64)[:, None] * m.N
            i = (first + np.arange(m.N - 1, dtype=np.int64)[None, :]).reshape(-1)
            out.append(np.stack([i, i + 1], axis=1))
        start += m.n_chains * m.N
    return np.concatenate(out) if out else np.zeros((0, 2), np.int64)


def random_walk_positions(moltypes: Sequence[MolType], L: float, b: float, seed: int) -> np.ndarray:
    """(n_beads, 3) float64 coordinates wrapped into [0, L), chain by chain."""
    rng = np.random.Generator(np.random.PCG64(seed))
    chunks: List[np.ndarray] = []
    for m in moltypes:
        if m.n_chains == 0:
            continue
        first = rng.uniform(0.0, L, size=(m.n_chains, 1, 3))
        u = rng.normal(size=(m.n_chains, m.N - 1, 3))
        u /= np.linalg.norm(u, axis=2, keepdims=True)
        steps = np.concatenate([np.zeros((m.n_chains, 1, 3)), b * u], axis=1)
        chunks.append((first + np.cumsum(steps, axis=1)).reshape(-1, 3))
    r = np.concatenate(chunks) if chunks else np.zeros((0, 3))
    r = np.mod(r, L)
    r[r >= L] = 0.0
    return r


def initial_positions(spec: SystemSpec) -> np.ndarray:
    return random_walk_positions(spec.moltypes, spec.L, spec.b, spec.input_seed)


def random_positions(n_beads: int, L: float, seed: int) -> np.ndarray:
    """Uniform positions in [0, L)^3 (for kernel-level tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(0.0, L, size=(n_beads, 3))


def batch_configs(n_replicas: int = 256, seed: int = 12345 + 5, steps: int = 5000) -> List[SystemSpec]:
    """Uneven replicas of AB diblock melts (A10-B10, N = 20): bead counts
    uniform in [4000, 40000] rounded to whole chains, box L uniform in
    [16, 32], grid spacing uniform in [0.5, 0.67] with n the nearest of
    {24, 32, 40, 48, 64} to L/dx, chi uniform in [0.2, 1.5], kappa = 25,
    a = 0.5, independent seeds; FP32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.array([24, 32, 40, 48, 64])
    out: List[SystemSpec] = []
    for r in range(n_replicas):
        beads = rng.uniform(4000, 40000)
        n_chains = max(1, int(round(beads / 20)))
        L = float(rng.uniform(16.0, 32.0))
        dx = float(rng.uniform(0.5, 0.67))
        n = int(sizes[np.argmin(np.abs(sizes - L / dx))])
        chi = float(rng.uniform(0.2, 1.5))
        out.append(SystemSpec(f"batch{r}", (MolType(n_chains, 20, 10),), L, n, 1, 0.5, chi, 25.0, 0.005, 1.0, 1.0, 1.0,
                              1.0, steps, "fp32", seed * 1000 + 2 * r, seed * 1000 + 2 * r + 1))
    return out


@dataclasses.dataclass(frozen=True)
class Topology:
    """Explicit species and bonds of a system (beads numbered 0..n-1):
    ``species`` (n,) int32 in [0, n_species), ``bonds`` (n_bonds, 2) int32
    bead-id pairs and ``positions`` (n, 3) float64 in [0, L)."""

    n_species: int
    species: np.ndarray
    bonds: np.ndarray
    positions: np.ndarray


def ring_star_system(n_rings: int, ring_N: int, n_stars: int, arms: int, arm_N: int, n_linear: int, lin_N: int,
                     L: float, b: float = 1.0, n_species: int = 3, seed: int = 9) -> Topology:
    """A mixture of ring polymers, star polymers and linear chains with up
    to four species, for topology tests (Sec. "Input file": a data file gives
    each bead's type and the bond list).

    Rings: ring_N beads on a closed loop, the first half species 0 and the
    rest species 1, beads on a circle of circumference ring_N * b (so every
    bond, the closing one included, is about b long) around a uniform centre,
    in a uniformly oriented plane.
    Stars: one centre bead (species 2 when n_species > 2, else 0) with
    ``arms`` random-walk arms of arm_N beads (species 1, or 3 for the odd arms
    when n_species == 4), each arm bonded to the centre: the centre has
    ``arms`` bonds.
    Linear chains: lin_N-bead random walks, species 0 then 1 (halves).
    Molecules are numbered rings, stars, linear chains."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sp: List[int] = []
    bonds: List[Tuple[int, int]] = []
    pos: List[np.ndarray] = []
    idx = 0
    for _ in range(n_rings):
        c = rng.uniform(0.0, L, size=3)
        e1 = rng.normal(size=3)
        e1 /= np.linalg.norm(e1)
        e2 = rng.normal(size=3)
        e2 -= e1 * np.dot(e1, e2)
        e2 /= np.linalg.norm(e2)
        rad = ring_N * b / (2.0 * np.pi)
        ang = 2.0 * np.pi * np.arange(ring_N) / ring_N
        pos.append(c + rad * (np.cos(ang)[:, None] * e1 + np.sin(ang)[:, None] * e2))
        sp += [0] * (ring_N // 2) + [1] * (ring_N - ring_N // 2)
        bonds += [(idx + k, idx + (k + 1) % ring_N) for k in range(ring_N)]
        idx += ring_N
    for _ in range(n_stars):
        c = rng.uniform(0.0, L, size=3)
        centre = idx
        pos.append(c[None, :])
        sp.append(2 if n_species > 2 else 0)
        idx += 1
        for a in range(arms):
            u = rng.normal(size=(arm_N, 3))
            u /= np.linalg.norm(u, axis=1, keepdims=True)
            pos.append(c + np.cumsum(b * u, axis=0))
            sp += [3 if (n_species == 4 and a % 2 == 1) else 1] * arm_N
            bonds.append((centre, idx))
            bonds += [(idx + k, idx + k + 1) for k in range(arm_N - 1)]
            idx += arm_N
    for _ in range(n_linear):
        c = rng.uniform(0.0, L, size=3)
        u = rng.normal(size=(lin_N - 1, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        pos.append(c + np.concatenate([np.zeros((1, 3)), np.cumsum(b * u, axis=0)]))
        sp += [0] * (lin_N // 2) + [1] * (lin_N - lin_N // 2)
        bonds += [(idx + k, idx + k + 1) for k in range(lin_N - 1)]
        idx += lin_N
    r = np.mod(np.concatenate(pos), L)
    r[r >= L] = 0.0
    return Topology(n_species, np.asarray(sp, np.int32), np.asarray(bonds, np.int32).reshape(-1, 2), r)


def random_walk_positions_2d(moltypes: Sequence[MolType], L: float, b: float, seed: int) -> np.ndarray:
    """Two-dimensional version of random_walk_positions (Listing infile's
    "Dim 2"): (n_beads, 3) float64 with z = 0; the first bead of each chain
    uniform in the square [0, L)^2, each following bead at distance b along a
    uniformly random direction in the plane."""
    rng = np.random.Generator(np.random.PCG64(seed))
    chunks: List[np.ndarray] = []
    for m in moltypes:
        if m.n_chains == 0:
            continue
        first = rng.uniform(0.0, L, size=(m.n_chains, 1, 2))
        ang = rng.uniform(0.0, 2.0 * np.pi, size=(m.n_chains, m.N - 1))
        steps = np.concatenate([np.zeros((m.n_chains, 1, 2)), b * np.stack([np.cos(ang), np.sin(ang)], axis=2)], axis=1)
        chunks.append((first + np.cumsum(steps, axis=1)).reshape(-1, 2))
    r = np.concatenate(chunks) if chunks else np.zeros((0, 2))
    r = np.mod(r, L)
    r[r >= L] = 0.0
    return np.concatenate([r, np.zeros((len(r), 1))], axis=1)
