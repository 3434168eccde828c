"""Differentiable form on the GPU: the force vector-Jacobian product
(tild_force_vjp) and derivatives through GJF, Euler-Maruyama and
velocity-Verlet trajectories with checkpoints (tild_trajectory_vjp), against
the oracle's force_vjp and its per-scheme trajectory adjoints (themselves
pinned by finite differences)."""
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
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def _setup(B, spec, charges=None):
    pos = I.initial_positions(spec)
    if spec.precision == "fp32":
        pos = pos.astype(np.float32).astype(np.float64)
    t = B.Tild.from_spec(spec, sort_every=3)
    m = O.model_from_spec(spec, I.species_of_beads(spec.moltypes), I.bond_pairs(spec.moltypes))
    if charges is not None:
        t.set_electrostatics(charges[0], charges[1], 1.5, 0.6)
        m.charges, m.bjerrum, m.charge_smear = np.array(charges), 1.5, 0.6
    t.set_positions(pos)
    return t, m, pos


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("order,charges", [(1, None), (2, (0.7, -1.2)), (4, None)])
def test_force_vjp_matches_oracle(B, prec, order, charges):
    spec = I.small_system(n_chains=70, N=10, n_a=4, L=8.0, n=16, pmeorder=order, precision=prec, chi=1.1, kappa=6.0)
    t, m, pos = _setup(B, spec, charges)
    lam = np.random.default_rng(3).normal(size=pos.shape)
    if prec == "fp32":
        lam = lam.astype(np.float32)
    got, th = t.force_vjp(lam)
    ref = O.force_vjp(m, pos, lam.astype(np.float64))
    tol = 1e-10 if prec == "fp64" else 1e-4
    assert _rel(got, ref["r"]) < tol
    for k in ("chi", "kappa", "a"):
        assert th[k] == pytest.approx(ref[k], rel=tol, abs=tol * 1e-3 * abs(ref["a"])), k


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_force_vjp_is_reproducible_and_exactly_homogeneous(B, prec):
    # lam is spread in fixed point with a power-of-two scale taken from
    # max|lam|: repeated calls agree bitwise, and J^T (2^k lam) is exactly
    # 2^k J^T lam (the same integers, rescaled), as is d(lam . F)/dtheta.
    spec = I.small_system(n_chains=70, N=10, n_a=4, L=8.0, n=16, pmeorder=2, precision=prec, chi=1.1, kappa=6.0)
    t, m, pos = _setup(B, spec)
    dt = np.float64 if prec == "fp64" else np.float32
    lam = np.random.default_rng(5).normal(size=pos.shape).astype(dt)
    a, tha = t.force_vjp(lam)
    b, thb = t.force_vjp(lam)
    assert a.tobytes() == b.tobytes() and tha == thb
    for k in (40, -40):
        c, thc = t.force_vjp(lam * dt(2.0**k))
        assert np.array_equal(c, a * dt(2.0**k)), k
        for key in ("chi", "kappa", "a"):
            assert thc[key] == tha[key] * 2.0**k, (k, key)


def test_force_vjp_non_finite_lam_gives_nan(B):
    spec = I.small_system(n_chains=70, N=10, n_a=4, L=8.0, n=16, pmeorder=2, precision="fp32", chi=1.1, kappa=6.0)
    t, m, pos = _setup(B, spec)
    lam = np.random.default_rng(6).normal(size=pos.shape).astype(np.float32)
    lam[17, 1] = np.nan
    got, th = t.force_vjp(lam)
    assert np.isnan(got).all() and all(np.isnan(th[k]) for k in ("chi", "kappa", "a"))
    lam[17, 1] = 0.5  # the context is still usable
    got, th = t.force_vjp(lam)
    assert np.isfinite(got).all()


@pytest.mark.parametrize("scheme", ["gjf", "em", "vv"])
def test_trajectory_vjp_matches_oracle(B, scheme):
    """Derivatives through 7 steps of each scheme (checkpoints every 3)
    against the oracle's reverse sweep for that scheme, with a velocity term
    in the loss where the scheme has velocities; K = 0 is the identity."""
    from paper_2302_02474_gb300.trajectory import trajectory_vjp

    friction = {"gjf": 1.0, "em": 2.0, "vv": 0.7}[scheme]
    spec = I.small_system(n_chains=40, N=10, n_a=4, L=7.0, n=16, pmeorder=1, precision="fp64", chi=1.0, kappa=6.0,
                          dt=0.01, friction=friction)
    pos = I.initial_positions(spec)
    t = B.Tild.from_spec(spec, sort_every=3)
    t.set_scheme(scheme)
    t.set_positions(pos)
    m = O.model_from_spec(spec, I.species_of_beads(spec.moltypes), I.bond_pairs(spec.moltypes))
    t.init_velocities()
    vel0 = O.initial_state(m, pos).vel
    K = 7
    rng = np.random.default_rng(5)
    w = rng.normal(size=pos.shape)
    u = None if scheme == "em" else rng.normal(size=pos.shape)
    g = trajectory_vjp(t, K, w, u, checkpoint_every=3)
    if scheme == "gjf":
        ref = O.gjf_trajectory_vjp(m, pos, vel0, K, w, u)
        st = O.run(m, O.initial_state(m, pos), K)
    elif scheme == "em":
        ref = O.em_trajectory_vjp(m, pos, K, w)
        st = O.run_with(O.em_step, m, O.em_initial_state(m, pos), K)
    else:
        ref = O.vv_trajectory_vjp(m, pos, vel0, K, w, u)
        st = O.run_with(O.vv_step, m, O.vv_initial_state(m, pos, vel0), K)
    assert t.step_count() == K
    assert np.abs(O.minimum_image(t.positions() - st.pos, m.L)).max() < 1e-10
    assert _rel(g["r0"], ref["r0"]) < 1e-9
    if scheme == "em":
        assert not np.any(g["v0"])
    else:
        assert _rel(g["v0"], ref["v0"]) < 1e-9
    for k in ("chi", "kappa", "a"):
        assert g[k] == pytest.approx(ref[k], rel=1e-9), k
    g0 = trajectory_vjp(t, 0, w, u)
    assert t.step_count() == K
    assert np.allclose(g0["r0"], w, rtol=0, atol=1e-12)
    if u is not None:
        assert np.allclose(g0["v0"], u, rtol=0, atol=1e-12)


def test_trajectory_vjp_with_checkpoints_beyond_the_window(B):
    """checkpoint_every larger than the trajectory: one segment, same result."""
    from paper_2302_02474_gb300.trajectory import trajectory_vjp

    spec = I.small_system(n_chains=30, N=10, n_a=4, L=6.0, n=16, pmeorder=1, precision="fp64", chi=1.0, kappa=6.0,
                          dt=0.01)
    t, m, pos = _setup(B, spec)
    t.init_velocities()
    vel0 = O.initial_state(m, pos).vel
    w = np.random.default_rng(8).normal(size=pos.shape)
    g = trajectory_vjp(t, 4, w, checkpoint_every=1000)
    ref = O.gjf_trajectory_vjp(m, pos, vel0, 4, w)
    assert t.step_count() == 4
    assert _rel(g["r0"], ref["r0"]) < 1e-9 and _rel(g["v0"], ref["v0"]) < 1e-9


def test_trajectory_autograd_matches_oracle(B):
    """tild_trajectory as a torch.autograd function: r^K, v^K equal the
    oracle's trajectory, and backward of sum w . r^K + sum u . v^K equals the
    oracle's reverse sweep for the initial positions, velocities, chi, kappa
    and a; the context is left where the forward left it."""
    import torch

    from paper_2302_02474_gb300.autograd import tild_trajectory

    spec = I.small_system(n_chains=30, N=10, n_a=4, L=6.0, n=16, pmeorder=1, precision="fp64", chi=1.0, kappa=6.0,
                          dt=0.01)
    pos = I.initial_positions(spec)
    t = B.Tild.from_spec(spec, sort_every=3)
    m = O.model_from_spec(spec, I.species_of_beads(spec.moltypes), I.bond_pairs(spec.moltypes))
    vel0 = O.initial_state(m, pos).vel
    K = 5
    rng = np.random.default_rng(13)
    w, u = rng.normal(size=pos.shape), rng.normal(size=pos.shape)
    f64 = dict(dtype=torch.float64)
    r0 = torch.tensor(pos, device="cuda", requires_grad=True, **f64)
    v0 = torch.tensor(vel0, device="cuda", requires_grad=True, **f64)
    chi, kappa, a = (torch.tensor(float(x), requires_grad=True, **f64) for x in (spec.chi, spec.kappa, spec.a))
    r_k, v_k = tild_trajectory(t, K, r0, v0, chi, kappa, a, checkpoint_every=2)
    st = O.run(m, O.State(O.wrap(pos, m.L), vel0, O.forces(m, O.wrap(pos, m.L)), 0), K)
    assert np.abs(O.minimum_image(r_k.detach().cpu().numpy() - st.pos, m.L)).max() < 1e-10
    assert _rel(v_k.detach().cpu().numpy(), st.vel) < 1e-10
    loss = (torch.as_tensor(w, device="cuda") * r_k).sum() + (torch.as_tensor(u, device="cuda") * v_k).sum()
    loss.backward()
    ref = O.gjf_trajectory_vjp(m, pos, vel0, K, w, u)
    assert _rel(r0.grad.cpu().numpy(), ref["r0"]) < 1e-9
    assert _rel(v0.grad.cpu().numpy(), ref["v0"]) < 1e-9
    for name, p in (("chi", chi), ("kappa", kappa), ("a", a)):
        assert float(p.grad) == pytest.approx(ref[name], rel=1e-9), name
    assert t.step_count() == K


def test_trajectory_autograd_backward_keeps_the_current_parameters(B):
    """Parameters set after the forward (and before backward) are the ones
    the context holds after backward: a step then equals the same step of a
    context that never ran the backward."""
    import torch

    from paper_2302_02474_gb300.autograd import tild_trajectory

    spec = I.small_system(n_chains=20, N=10, n_a=4, L=6.0, n=16, pmeorder=1, precision="fp64", chi=1.0, kappa=6.0)
    pos = I.initial_positions(spec)
    m = O.model_from_spec(spec, I.species_of_beads(spec.moltypes), I.bond_pairs(spec.moltypes))
    vel0 = O.initial_state(m, pos).vel
    f64 = dict(dtype=torch.float64, device="cuda")
    t = B.Tild.from_spec(spec, sort_every=3)
    r0 = torch.tensor(pos, requires_grad=True, **f64)
    v0 = torch.tensor(vel0, **f64)
    r_k, _ = tild_trajectory(t, 3, r0, v0, spec.chi, spec.kappa, spec.a, checkpoint_every=2)
    t.set_interactions(2.0, 9.0, 0.6)
    r_k.sum().backward()
    assert t.interactions == (2.0, 9.0, 0.6)
    t.step(2)
    ref = B.Tild.from_spec(spec, sort_every=3)
    ref.set_positions(pos)
    ref.set_velocities(vel0)
    ref.step(3)
    ref.set_interactions(2.0, 9.0, 0.6)
    ref.step(2)
    assert np.array_equal(t.positions(), ref.positions())
    assert r0.grad.is_cuda


def test_force_vjp_needs_the_ik_force(B):
    spec = I.small_system(n_chains=20, N=10, n_a=4, L=6.0, n=16, precision="fp64")
    t, m, pos = _setup(B, spec)
    t.set_force_method("analytic")
    with pytest.raises(B.TildError, match="EUNSUPPORTED"):
        t.force_vjp(np.zeros(pos.shape))


def test_device_checkpoints_match_host_blobs(B):
    import torch

    spec = I.small_system(n_chains=30, N=10, n_a=4, L=6.0, n=16, precision="fp32")
    t, m, pos = _setup(B, spec)
    t.init_velocities()
    t.step(5)
    host = t.get_state()
    dev = t.get_state(out=torch.empty(t.state_bytes(), dtype=torch.uint8, device="cuda"))
    assert dev.cpu().numpy().tobytes() == host
    t.step(4)
    r9 = t.positions()
    t.set_state(dev)
    assert t.step_count() == 5
    t.step(4)
    assert np.array_equal(t.positions(), r9)
