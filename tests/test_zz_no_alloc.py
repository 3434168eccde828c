"""The allocation-free density entry point against the context-based one.

tild_spread_density_noalloc serves callers that cannot allocate device
memory (a framework allocator owns it, a fixed memory budget, or a loop
where a possibly synchronising cudaMalloc is not acceptable). It keeps its
scratch grid in a static device array shared by every call, so this test
makes two calls in a row with different inputs and checks each against the
density that tild_get_density returns for the same beads.
"""
import ctypes

import numpy as np
import pytest

from paper_2302_02474_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_noalloc_density_matches_context_density_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_02474_gb300 import _build, binding as B

    _build.build()
    lib = B.load()
    for spec in (I.small_system(n_chains=150, N=12, n_a=5, L=12.0, n=32, pmeorder=1, precision="fp32", seed=21),
                 I.small_system(n_chains=90, N=20, n_a=8, L=16.0, n=64, pmeorder=3, precision="fp32", seed=22)):
        pos = I.initial_positions(spec).astype(np.float32)
        sp = I.species_of_beads(spec.moltypes).astype(np.uint8)
        with B.Tild.from_spec(spec) as t:
            t.set_positions(pos)
            ref = t.density(dtype=np.float32)
        xyz = torch.from_numpy(pos).cuda()
        species = torch.from_numpy(sp).cuda()
        out = torch.full((2 * spec.n ** 3,), float("nan"), dtype=torch.float32, device="cuda")
        st = lib.tild_spread_density_noalloc(ctypes.c_void_p(xyz.data_ptr()), ctypes.c_void_p(species.data_ptr()),
                                             spec.n_beads, spec.L, spec.n, spec.pmeorder,
                                             ctypes.c_void_p(out.data_ptr()), None)
        assert st == B.TILD_OK, lib.tild_last_error(None)
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(2, spec.n, spec.n, spec.n)
        assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max()


def test_noalloc_rejects_grids_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_02474_gb300 import binding as B

    lib = B.load()
    xyz = torch.zeros(3, dtype=torch.float32, device="cuda")
    species = torch.zeros(1, dtype=torch.uint8, device="cuda")
    out = torch.zeros(2 * 128 ** 3, dtype=torch.float32, device="cuda")
    st = lib.tild_spread_density_noalloc(ctypes.c_void_p(xyz.data_ptr()), ctypes.c_void_p(species.data_ptr()), 1,
                                         10.0, 128, 1, ctypes.c_void_p(out.data_ptr()), None)
    assert st == B.TILD_EINVAL
    assert b"[8, 64]" in lib.tild_last_error(None)
