"""Green-Kubo shear viscosity from a stress time series (Sec. 5.2, Eq. viscosity).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): the plain NumPy restatement the library's
sq_green_kubo is compared with.

  eta(t) = |Omega| / (k_B T) * int_0^t (1/5) sum_i <s_i(t') s_i(0)> dt'
  s_i = sigma_12, sigma_23, sigma_31, (sigma_11 - sigma_22) / 2, (sigma_22 - sigma_33) / 2

Readings (the paper names the estimator only as an ensemble average): <s_i(k dt) s_i(0)> is the
mean of s_i(t + k) s_i(t) over every time origin t = 0 .. n_steps - 1 - k of every trajectory
(stationarity; trajectories are independent initial conditions), the five components are
averaged, and the time integral is the trapezoid rule on the sampled lags. Atomic units.
"""
from __future__ import annotations

import numpy as np


def deviatoric_components(sigma: np.ndarray) -> np.ndarray:
    """(..., 3, 3) stress tensors -> (..., 5) independent deviatoric components s_i."""
    s = np.asarray(sigma, dtype=np.float64)
    return np.stack([s[..., 0, 1], s[..., 1, 2], s[..., 2, 0],
                     0.5 * (s[..., 0, 0] - s[..., 1, 1]), 0.5 * (s[..., 1, 1] - s[..., 2, 2])], axis=-1)


def stress_acf(sigma: np.ndarray, max_lag: int) -> np.ndarray:
    """sigma: (n_traj, n_steps, 3, 3). Returns C[k] = (1/5) sum_i <s_i(t + k) s_i(t)>, k = 0..max_lag,
    averaged over all origins of all trajectories."""
    s = deviatoric_components(sigma)                     # (n_traj, n_steps, 5)
    n = s.shape[1]
    out = np.empty(max_lag + 1)
    for k in range(max_lag + 1):
        prod = s[:, k:, :] * s[:, : n - k, :]            # origins t = 0 .. n - 1 - k
        out[k] = prod.mean(axis=(0, 1)).mean()
    return out


def viscosity(sigma: np.ndarray, dt: float, volume: float, kT: float, max_lag: int):
    """Running Green-Kubo integral eta[k] = (|Omega| / kT) * trapezoid of C over [0, k dt]."""
    c = stress_acf(sigma, max_lag)
    eta = np.zeros(max_lag + 1)
    for k in range(1, max_lag + 1):
        eta[k] = eta[k - 1] + 0.5 * dt * (c[k - 1] + c[k])
    return volume / kT * eta, c
