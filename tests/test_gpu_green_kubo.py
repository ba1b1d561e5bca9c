"""Green-Kubo viscosity (Eq. viscosity) through the C ABI against the oracle, on seeded
synthetic stress series (correlated noise in all six independent tensor entries plus an
isotropic pressure), several trajectories, lags up to a tenth of the series."""
import numpy as np
import pytest

from oracle import green_kubo

pytestmark = pytest.mark.gpu


def _series(seed, n_traj, n_steps, tau=12.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    a = np.exp(-1.0 / tau)
    x = np.empty((n_traj, n_steps, 6))
    x[:, 0] = rng.normal(size=(n_traj, 6))
    noise = rng.normal(size=(n_traj, n_steps, 6)) * np.sqrt(1.0 - a * a)
    for i in range(1, n_steps):
        x[:, i] = a * x[:, i - 1] + noise[:, i]
    sig = np.empty((n_traj, n_steps, 3, 3))
    iu = [(0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (0, 2)]
    for k, (p, q) in enumerate(iu):
        sig[..., p, q] = 0.01 * x[..., k]
        sig[..., q, p] = 0.01 * x[..., k]
    sig += (-0.12 + 0.003 * rng.normal(size=(n_traj, n_steps)))[..., None, None] * np.eye(3)
    return sig


@pytest.mark.parametrize("n_traj,n_steps,max_lag", [(1, 50, 0), (3, 2000, 200), (10, 5000, 499)])
def test_green_kubo_matches_oracle(n_traj, n_steps, max_lag):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2006_03697_gb300 import build
    build.build()
    from paper_2006_03697_gb300 import sq

    sig = _series(7 + n_traj, n_traj, n_steps)
    dt, vol, kT = 16.5, 1728.0, 3.17          # 0.4 fs sampling, the 64 H cell, 10^6 K
    eta_ref, acf_ref = green_kubo.viscosity(sig, dt, vol, kT, max_lag)
    eta, acf = sq.sq_green_kubo(sig, dt, vol, kT, max_lag)
    np.testing.assert_allclose(acf, acf_ref, rtol=1e-11, atol=1e-20)
    np.testing.assert_allclose(eta, eta_ref, rtol=1e-11, atol=1e-20)
