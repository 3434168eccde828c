"""Batched form: replicas stepped together through tild_batch_* give, bit for
bit, the trajectories of the same systems stepped one by one (and those are
checked against the oracle elsewhere)."""
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


REPLICAS = [  # (n_chains, N, n_a, L, n, pmeorder, chi, seed)
    (40, 20, 10, 9.6, 24, 1, 0.3, 11),
    (55, 20, 8, 12.0, 32, 1, 1.2, 12),
    (31, 20, 10, 10.0, 32, 1, 0.7, 13),
    (70, 20, 10, 16.0, 48, 1, 1.5, 14),
    (25, 20, 5, 8.0, 16, 2, 0.9, 15),
    (60, 20, 12, 16.0, 40, 1, 0.4, 16),
]


def _spec(r, prec):
    nc, N, na, L, n, order, chi, seed = r
    return I.small_system(n_chains=nc, N=N, n_a=na, L=L, n=n, pmeorder=order, precision=prec, chi=chi, kappa=25.0,
                          seed=seed)


def _ctx(B, spec, sort_every, pos):
    t = B.Tild.from_spec(spec, sort_every=sort_every)
    t.set_positions(pos)
    t.init_velocities()
    return t


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batch_matches_individual_replicas_bitwise(B, prec):
    specs = [_spec(r, prec) for r in REPLICAS]
    pos = [I.initial_positions(s) for s in specs]
    batch_ctx = [_ctx(B, s, 5, p) for s, p in zip(specs, pos)]
    alone = [_ctx(B, s, 7, p) for s, p in zip(specs, pos)]
    with B.TildBatch(batch_ctx) as bt:
        bt.step(3)
        bt.step(30)  # includes whole re-binning cycles replayed as a graph
        bt.step(2)
        bt.synchronize()
        assert bt.launches(10) > 0
    for t in alone:
        t.step(35)
        t.synchronize()
    for tb, ta in zip(batch_ctx, alone):
        assert tb.step_count() == ta.step_count() == 35
        assert np.array_equal(tb.positions(), ta.positions())
        assert np.array_equal(tb.velocities(), ta.velocities())


def test_batch_replica_matches_oracle(B):
    spec = _spec(REPLICAS[0], "fp64")
    pos = I.initial_positions(spec)
    other = _spec(REPLICAS[3], "fp64")
    ts = [_ctx(B, spec, 4, pos), _ctx(B, other, 4, I.initial_positions(other))]
    with B.TildBatch(ts) as bt:
        bt.step(12)
        bt.synchronize()
    m = O.model_from_spec(spec, I.species_of_beads(spec.moltypes), I.bond_pairs(spec.moltypes))
    st = O.run(m, O.initial_state(m, pos), 12)
    assert np.abs(O.minimum_image(ts[0].positions() - st.pos, m.L)).max() < 1e-10


def test_batch_rejects_bad_input(B):
    spec = _spec(REPLICAS[1], "fp32")
    t = B.Tild.from_spec(spec)
    t.set_positions(I.initial_positions(spec))
    with pytest.raises(B.TildError):
        B.TildBatch([t])  # no velocities yet
    t.init_velocities()
    with pytest.raises(B.TildError):
        B.TildBatch([t, t])
    t64 = B.Tild.from_spec(_spec(REPLICAS[1], "fp64"))
    t64.set_positions(I.initial_positions(spec))
    t64.init_velocities()
    with pytest.raises(B.TildError):
        B.TildBatch([t, t64])


PERSISTENT = [r for r in REPLICAS if r[5] == 1 and r[4] in (24, 32, 40, 48, 64)] + [
    (90, 20, 10, 20.0, 64, 1, 1.1, 17)]


def test_persistent_batch_matches_individual_replicas_bitwise(B):
    """Eligible replicas (FP32, pmeorder 1, grids 24..64) step through the one
    persistent launch per re-binning run; same bits as stepping alone."""
    specs = [_spec(r, "fp32") for r in PERSISTENT]
    pos = [I.initial_positions(s) for s in specs]
    batch_ctx = [_ctx(B, s, 5, p) for s, p in zip(specs, pos)]
    alone = [_ctx(B, s, 9, p) for s, p in zip(specs, pos)]
    with B.TildBatch(batch_ctx) as bt:
        assert bt.persistent
        bt.step(3)
        bt.step(30)  # whole re-binning cycles (graph replay of sorts + persistent launches)
        bt.step(4)
        bt.synchronize()
        # one launch per run of steps between re-binnings (K = 5: at most
        # three runs in 10 steps), plus 8 per replica per re-binning (two)
        assert bt.launches(10) <= 3 + 2 * 8 * len(specs)
    for t in alone:
        t.step(37)
        t.synchronize()
    for tb, ta in zip(batch_ctx, alone):
        assert tb.step_count() == ta.step_count() == 37
        assert np.array_equal(tb.positions(), ta.positions())
        assert np.array_equal(tb.velocities(), ta.velocities())


def test_persistent_wait_runs_out(B):
    """Fault injection on the host side: the persistent kernel's grid barrier
    is told to wait for one CTA more than the launch has, so every wait runs
    out after its limit; the kernel returns, the batch reports TILD_ETIMEOUT,
    and the device stays usable."""
    specs = [_spec(r, "fp32") for r in PERSISTENT[:2]]
    ts = [_ctx(B, s, 5, I.initial_positions(s)) for s in specs]
    with B.TildBatch(ts) as bt:
        assert bt.persistent
        bt.set_wait_limit(20_000_000, extra=1)  # 20 ms
        bt.step(2)
        with pytest.raises(B.TildError) as ei:
            bt.synchronize()
        assert ei.value.status == B.TILD_ETIMEOUT
    # the context and device still work
    t = _ctx(B, specs[0], 5, I.initial_positions(specs[0]))
    t.step(3)
    t.synchronize()


def test_plane_threads_1024_and_row_passes_same_bits(B):
    """80^3 FP32: 1024-thread plane CTAs, 512 and the row/column passes give
    the same trajectory bits."""
    spec = I.small_system(n_chains=300, N=10, n_a=4, L=32.0, n=80, precision="fp32")
    pos = I.initial_positions(spec)
    out = []
    for pt in (512, 1024, 0):
        t = _ctx(B, spec, 5, pos)
        t.set_launch_shapes(pt, t.launch_shapes()[1])
        assert t.launch_shapes()[0] == pt
        t.step(12)
        out.append((t.positions(), t.velocities()))
    for o in out[1:]:
        assert np.array_equal(o[0], out[0][0]) and np.array_equal(o[1], out[0][1])


def test_plane_shapes_same_bits_at_128(B):
    """128^3 FP32 (the benchmarked grid): 512- and 1024-thread planes, the
    row/column passes and both z tiles give the same trajectory and field bits."""
    spec = I.small_system(n_chains=1500, N=10, n_a=4, L=48.0, n=128, precision="fp32")
    pos = I.initial_positions(spec)
    out = []
    for pt, alt in ((512, False), (1024, True), (1024, False), (0, True)):
        t = _ctx(B, spec, 4, pos)
        zdef = t.launch_shapes()[1]
        t.set_launch_shapes(pt, zdef // 2 if alt else zdef)
        assert t.launch_shapes()[0] == pt
        t.step(9)
        out.append((t.positions(), t.velocities(), t.field_gradient()))
    for o in out[1:]:
        for a, b in zip(o, out[0]):
            assert np.array_equal(a, b)


def test_launch_shapes_do_not_change_results(B):
    spec = _spec(REPLICAS[3], "fp32")  # 48^3
    pos = I.initial_positions(spec)
    out = []
    for pt, alt in ((512, False), (256, False), (128, True), (0, False), (0, True)):
        t = _ctx(B, spec, 5, pos)
        zdef = t.launch_shapes()[1]
        try:
            t.set_launch_shapes(pt, zdef if not alt else max(2, zdef // 2))
        except B.TildError:
            continue
        t.step(12)
        out.append((t.positions(), t.velocities()))
    assert len(out) >= 4  # 512, 256 and the row/column passes (0) exist for 48^3
    for o in out[1:]:
        assert np.array_equal(o[0], out[0][0]) and np.array_equal(o[1], out[0][1])
