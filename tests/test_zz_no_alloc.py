"""The allocation-free density entry point (tild_spread_density_noalloc).

It serves callers that cannot allocate device memory: code running while a
framework's caching allocator owns the device memory, plug-ins held to a
fixed memory budget, or loops where a cudaMalloc (which can synchronise the
device) is not acceptable. Its scratch grid is a static device array shared
by every call, so the tests make two calls in a row with different inputs
and check each against the FP64 oracle's spread (within the FP32 density
tolerance of the other parity tests) and against the context-based
tild_get_density, and check that a call after the first takes no device
memory.
"""
import ctypes

import numpy as np
import pytest

from oracle import tild_oracle as O
from paper_2302_02474_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_02474_gb300 import _build, binding

    _build.build()
    return binding


def _call(B, lib, xyz, species, n_beads, L, n, pmeorder, out):
    return lib.tild_spread_density_noalloc(ctypes.c_void_p(xyz.data_ptr()), ctypes.c_void_p(species.data_ptr()),
                                           n_beads, L, n, pmeorder, ctypes.c_void_p(out.data_ptr()), None)


def test_noalloc_density_matches_oracle_and_context_on_two_calls(B):
    import torch

    lib = B.load()
    for spec in (I.small_system(n_chains=150, N=12, n_a=5, L=12.0, n=32, pmeorder=1, precision="fp32", seed=21),
                 I.small_system(n_chains=90, N=20, n_a=8, L=16.0, n=64, pmeorder=3, precision="fp32", seed=22)):
        pos = I.initial_positions(spec).astype(np.float32)
        sp = I.species_of_beads(spec.moltypes).astype(np.uint8)
        m = O.model_from_spec(spec, I.species_of_beads(spec.moltypes), I.bond_pairs(spec.moltypes))
        ref = O.spread(m, pos.astype(np.float64)).transpose(0, 3, 2, 1)  # -> [K][z][y][x]
        with B.Tild.from_spec(spec) as t:
            t.set_positions(pos)
            ctx_rho = t.density(dtype=np.float32)
        xyz = torch.from_numpy(pos).cuda()
        species = torch.from_numpy(sp).cuda()
        out = torch.full((2 * spec.n ** 3,), float("nan"), dtype=torch.float32, device="cuda")
        st = _call(B, lib, xyz, species, spec.n_beads, spec.L, spec.n, spec.pmeorder, out)
        assert st == B.TILD_OK, lib.tild_last_error(None)
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(2, spec.n, spec.n, spec.n)
        assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max()
        assert np.abs(got - ctx_rho).max() <= 2e-6 * np.abs(ctx_rho).max()
        dV = (spec.L / spec.n) ** 3
        for K in range(2):
            assert abs(got[K].sum() * dV - np.sum(sp == K)) < 1e-6 * len(sp)


def test_noalloc_second_call_takes_no_device_memory(B):
    import torch

    lib = B.load()
    spec = I.small_system(n_chains=50, N=10, n_a=4, L=8.0, n=16, pmeorder=2, precision="fp32", seed=23)
    xyz = torch.from_numpy(I.initial_positions(spec).astype(np.float32)).cuda()
    species = torch.from_numpy(I.species_of_beads(spec.moltypes).astype(np.uint8)).cuda()
    out = torch.empty(2 * spec.n ** 3, dtype=torch.float32, device="cuda")
    assert _call(B, lib, xyz, species, spec.n_beads, spec.L, spec.n, spec.pmeorder, out) == B.TILD_OK
    torch.cuda.synchronize()
    first = out.clone()
    free0, _ = torch.cuda.mem_get_info()
    assert _call(B, lib, xyz, species, spec.n_beads, spec.L, spec.n, spec.pmeorder, out) == B.TILD_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.equal(out, first)


def test_noalloc_rejects_grids_beyond_its_scratch(B):
    import torch

    lib = B.load()
    xyz = torch.zeros(3, dtype=torch.float32, device="cuda")
    species = torch.zeros(1, dtype=torch.uint8, device="cuda")
    out = torch.zeros(2 * 128 ** 3, dtype=torch.float32, device="cuda")
    st = _call(B, lib, xyz, species, 1, 10.0, 128, 1, out)
    assert st == B.TILD_EINVAL
    assert b"[8, 64]" in lib.tild_last_error(None)
