"""Gauss Spectral Quadrature for the electron density (the variant the paper uses inside the SCF
iteration, Sec. 5; the paper cites it without formulas).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Reading: for node q, k steps of Lanczos on H_q started from the node's unit vector e_q (full
reorthogonalisation by classical Gram-Schmidt applied twice, as for the spectral bounds) give
the tridiagonal T_q with eigenpairs (theta_qi, y_qi); the k-point Gauss quadrature of the
spectral measure of e_q is
    [f(H_q)]_qq ~ sum_i w_qi f(theta_qi),   w_qi = (first component of y_qi)^2,
exact for polynomials f of degree <= 2k - 1. Then rho_q = (2 / |dOmega|) sum_i w_qi g(theta_qi),
the Fermi level solves 2 sum_q sum_i w_qi g(theta_qi) = N_e (the shared bisection rule), and
the band energy is 2 sum_q sum_i w_qi theta_qi g(theta_qi).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from .sq_oracle import NodeRegion, Problem, fermi


def lanczos_tridiagonal(apply, v0: np.ndarray, k: int, reorth: bool = True):
    """(alpha, beta) of k-step Lanczos from v0 (normalised); stops early when
    beta <= 1e-12 max(1, |alpha|) (the Krylov space is exhausted). reorth: full
    reorthogonalisation by classical Gram-Schmidt applied twice; otherwise the plain three-term
    recurrence w = H v_i - alpha_i v_i - beta_{i-1} v_{i-1}, alpha_i = v_i^T H v_i."""
    V = [v0 / np.linalg.norm(v0)]
    alpha, beta = [], []
    for i in range(k):
        w = apply(V[i])
        if reorth:
            Vm = np.array(V)
            c1 = Vm @ w
            w = w - Vm.T @ c1
            c2 = Vm @ w
            w = w - Vm.T @ c2
            a = float(c1[i] + c2[i])
        else:
            a = float(V[i] @ w)
            w = w - a * V[i] - (beta[i - 1] * V[i - 1] if i > 0 else 0.0)
        b = float(np.linalg.norm(w))
        alpha.append(a)
        if i == k - 1 or b <= 1e-12 * max(1.0, abs(a)):
            break
        beta.append(b)
        V.append(w / b)
    return np.array(alpha), np.array(beta)


def node_quadrature(prob: Problem, q: int, k: int, reorth: bool = True):
    """Gauss nodes theta_qi and weights w_qi of node q (k-step Lanczos from e_q)."""
    region = NodeRegion(prob, prob.node_coords(q))
    shape = region.shape
    e = region.unit().reshape(-1)
    alpha, beta = lanczos_tridiagonal(lambda x: region.apply_H(x.reshape(shape)).reshape(-1), e,
                                      min(k, e.size), reorth)
    theta, Y = scipy.linalg.eigh_tridiagonal(alpha, beta)
    return theta, Y[0, :] ** 2


def electron_count(prob: Problem, quad, mu: float) -> float:
    return 2.0 * sum(float(np.sum(w * fermi((t - mu) / prob.kT))) for t, w in quad)


def fermi_bisect(prob: Problem, quad) -> float:
    lo = min(float(t.min()) for t, _ in quad) - 40.0 * prob.kT
    hi = max(float(t.max()) for t, _ in quad) + 40.0 * prob.kT
    if not (electron_count(prob, quad, lo) < prob.n_e < electron_count(prob, quad, hi)):
        raise ValueError("N(mu) - N_e has no sign change on the bisection bracket")
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if electron_count(prob, quad, mid) < prob.n_e:
            lo = mid
        else:
            hi = mid
        if hi - lo < 1e-13 * max(1.0, abs(mid)):
            break
    return 0.5 * (lo + hi)


def run(inst: dict, k: int = 40, reorth: bool = True):
    """Gauss SQ density, Fermi level and band energy of one instance."""
    prob = Problem(inst)
    quad = [node_quadrature(prob, q, k, reorth) for q in range(prob.Nd)]
    mu = fermi_bisect(prob, quad)
    g = [w * fermi((t - mu) / prob.kT) for t, w in quad]
    rho = np.array([2.0 / prob.dV * float(np.sum(gi)) for gi in g])
    E_band = 2.0 * sum(float(np.sum(gi * t)) for gi, (t, _) in zip(g, quad))
    return {"mu": mu, "rho": rho, "E_band": E_band, "N_check": prob.dV * float(np.sum(rho)), "quadrature": quad}
