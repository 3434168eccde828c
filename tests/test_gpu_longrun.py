"""Long-run observables of the GPU path within statistical error (FP32, the
production precision): equipartition in a chi/kappa melt and ideal-chain
statistics with the field interactions off. The oracle's own pins check the
same observables on the CPU at smaller sizes."""
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


def test_equipartition_in_a_diblock_melt(B):
    """<m v^2 / 2> = (3/2) kT per bead (the GJF on-site velocity bias is
    O((omega dt)^2) ~ 1e-4 here, below the statistical error)."""
    spec = I.config("diblock_200k_64")
    t = B.Tild.from_spec(spec)
    t.set_positions(I.initial_positions(spec))
    t.init_velocities()
    t.step(8000)  # the random-walk start releases field energy; let the thermostat remove it
    ke = []
    for _ in range(40):
        t.step(50)
        _, e = t.compute(forces=False)
        ke.append(e["kinetic"] / (1.5 * spec.n_beads * spec.kT))
    # 200k beads: each sample has relative spread ~ sqrt(2/3/N) ~ 2e-3
    assert abs(np.mean(ke) - 1.0) < 3e-3, ke


def test_ideal_chain_statistics(B):
    """chi = kappa = 0: bonds only (Eq. bonds). <|dr|^2> = b^2,
    <R_ee^2> = (N-1) b^2, <R_g^2> = b^2 (N^2 - 1)/(6 N)."""
    N, nc = 20, 2000
    spec = I.small_system(n_chains=nc, N=N, n_a=N, L=60.0, n=32, precision="fp32", chi=0.0, kappa=0.0, dt=0.05)
    t = B.Tild.from_spec(spec)
    t.set_positions(I.initial_positions(spec))
    t.init_velocities()
    t.step(600)
    b2, ree, rg = [], [], []
    for _ in range(30):
        t.step(40)
        r = t.positions().reshape(nc, N, 3)
        d = O.minimum_image(r[:, 1:] - r[:, :-1], spec.L)
        x = np.concatenate([np.zeros((nc, 1, 3)), np.cumsum(d, axis=1)], axis=1)
        b2.append(np.mean(np.sum(d * d, -1)))
        ree.append(np.mean(np.sum(x[:, -1] ** 2, -1)))
        xc = x - x.mean(1, keepdims=True)
        rg.append(np.mean(np.sum(xc * xc, -1)))
    assert abs(np.mean(b2) - 1.0) < 0.02
    assert abs(np.mean(ree) - (N - 1)) < 0.05 * (N - 1)
    assert abs(np.mean(rg) - (N * N - 1) / (6 * N)) < 0.05 * (N * N - 1) / (6 * N)
