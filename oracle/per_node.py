"""Per-node spectral bounds mode of the SQ sweep (Sec. 4): chi_q and zeta_q from the extreme
eigenvalues of each nodal Hamiltonian H_q, the literal reading of the method (the library's
default shares one interval over all nodes).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Per node q: k-step Lanczos on H_q from the node's own start vector (the same procedure as the
shared interval: full reorthogonalisation, Ritz extremes widened by their residual norms), then
widened by 1 % of the node's own width; the Chebyshev columns of node q use that node's
(chi_q, zeta_q). The Fermi level solves N(mu) = 2 sum_q sum'_j c_q^j(mu) rho_q^j = N_e with each
node's coefficients (same bisection rule as the shared mode), and the contraction uses each
node's c_q^j, d_q^j, s_q^j and (chi_q, zeta_q).
"""
from __future__ import annotations

import numpy as np

from .sq_oracle import (K_PAIRS, NodeRegion, Problem, fd_coefficients, lanczos_extremes, lanczos_start,
                        node_moments, primed)


def node_bounds(prob: Problem, q: int, k: int = 40):
    """(lambda_lo, lambda_hi) of node q's H_q: Lanczos extremes with residual widening, then 1 %."""
    region = NodeRegion(prob, prob.node_coords(q))
    shape = region.shape
    v0 = lanczos_start(region.chi.shape[1], q)
    lo, hi = lanczos_extremes(lambda x: region.apply_H(x.reshape(shape)).reshape(-1), v0,
                              min(k, region.chi.shape[1]))
    wdt = hi - lo
    return lo - 0.01 * wdt, hi + 0.01 * wdt


def moments(prob: Problem, bounds: np.ndarray) -> np.ndarray:
    """Moment table (N_d, n_pl + 1, 17), node q scaled by its own bounds[q]."""
    return np.array([node_moments(prob, prob.node_coords(q), bounds[q, 0], bounds[q, 1]) for q in range(prob.Nd)])


def _coefficients(prob: Problem, bounds: np.ndarray, mu: float):
    """Per-node (c, d, s) coefficient tables, each (N_d, n_pl + 1)."""
    c = np.empty((prob.Nd, prob.n_pl + 1))
    d = np.empty_like(c)
    s = np.empty_like(c)
    for q in range(prob.Nd):
        lo, hi = bounds[q]
        c[q], d[q], s[q] = fd_coefficients(mu, prob.kT, 0.5 * (hi + lo), 0.5 * (hi - lo), prob.n_pl, prob.M)
    return c, d, s


def electron_count(prob: Problem, mom: np.ndarray, bounds: np.ndarray, mu: float) -> float:
    c, _, _ = _coefficients(prob, bounds, mu)
    wp = primed(prob.n_pl)
    return 2.0 * float(np.sum(mom[:, :, 0] * c * wp))


def fermi_bisect(prob: Problem, mom: np.ndarray, bounds: np.ndarray) -> float:
    """The shared mode's bisection rule on [min lo - 40 kT, max hi + 40 kT]: halve towards
    N(mid) < N_e, stop when the bracket is below 1e-13 max(1, |mid|) or after 200 steps, return
    the midpoint."""
    lo = float(bounds[:, 0].min()) - 40.0 * prob.kT
    hi = float(bounds[:, 1].max()) + 40.0 * prob.kT
    if not (electron_count(prob, mom, bounds, lo) < prob.n_e < electron_count(prob, mom, bounds, hi)):
        raise ValueError("N(mu) - N_e has no sign change on the bisection bracket")
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if electron_count(prob, mom, bounds, mid) < prob.n_e:
            lo = mid
        else:
            hi = mid
        if hi - lo < 1e-13 * max(1.0, abs(mid)):
            break
    return 0.5 * (lo + hi)


def contract(prob: Problem, mom: np.ndarray, bounds: np.ndarray, mu: float):
    """Sec. 4 contraction with every node's own coefficients and (chi_q, zeta_q)."""
    c, d, s = _coefficients(prob, bounds, mu)
    wp = primed(prob.n_pl)
    cw, dw, sw = c * wp, d * wp, s * wp
    chi_q = 0.5 * (bounds[:, 1] + bounds[:, 0])
    zeta_q = 0.5 * (bounds[:, 1] - bounds[:, 0])
    rho_j = mom[:, :, 0]
    rho = 2.0 / prob.dV * np.sum(rho_j * cw, axis=1)
    E_band = 2.0 * float(np.sum(rho_j * (chi_q[:, None] * cw + zeta_q[:, None] * dw)))
    E_s = 2.0 * prob.kT * float(np.sum(rho_j * sw))
    E_nl = 2.0 * float(np.sum(mom[:, :, 7] * cw))
    sig_I = np.zeros((3, 3))
    for slot, (a, b) in enumerate(K_PAIRS):
        v = 2.0 * float(np.sum(mom[:, :, 1 + slot] * cw))
        sig_I[a, b] = v
        sig_I[b, a] = v
    sig_III = np.zeros((3, 3))
    for a in range(3):
        for b in range(3):
            S_ab = float(np.sum(mom[:, :, 8 + 3 * a + b] * cw))
            sig_III[a, b] = -2.0 * ((E_nl / 2.0 if a == b else 0.0) + 2.0 * S_ab)
    sigma = (sig_I + sig_III) / prob.vol
    return {"rho": rho, "E_band": E_band, "E_s": E_s, "E_nl": E_nl, "F": E_band + E_s,
            "N_check": prob.dV * float(np.sum(rho)), "sigma": sigma}


def run(inst: dict, k: int = 40):
    """Per-node bounds, moments, Fermi level and contraction of one instance."""
    prob = Problem(inst)
    bounds = np.array([node_bounds(prob, q, k) for q in range(prob.Nd)])
    mom = moments(prob, bounds)
    mu = fermi_bisect(prob, mom, bounds)
    out = contract(prob, mom, bounds, mu)
    out.update({"mu": mu, "bounds": bounds, "moments": mom})
    return out
