"""Closed forms for the free-electron grid (V_eff = 0, no projectors).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Infinite crystal: the discrete kinetic operator is diagonal in Bloch waves, with
  eps(theta) = sum_a s(theta_a) / (2 h_a^2),  s(t) = -w0 - 2 sum_p w_p cos(p t),
and the first-derivative stencil has symbol i G(t) / h, G(t) = 2 sum_p g_p sin(p t). So
  rho            = (2/dV) <g(eps)>
  sigma^I_aa     = -(2/dV) <g(eps) G(theta_a)^2> / h_a^2        (paper form, grad_a grad_a)
  sigma^I_aa     = -(2/dV) <g(eps) s(theta_a)>  / h_a^2         (second-difference form)
  E_band / Omega = (2/dV) <g eps>,  E_s / Omega = (2 kT / dV) <s_ent>
where <.> is the average over theta in [-pi, pi)^3 (the integrands are smooth and periodic,
so the uniform-grid rule converges spectrally). Off-diagonal stresses vanish by symmetry.

Truncated region: with V = 0 the nodal Hamiltonian is a Kronecker sum of three 1-D
matrices, so the exact [f(H_q)]_qq and [grad_a grad_a f(H_q)]_qq follow from three 1-D
eigendecompositions, even for large regions.
"""
from __future__ import annotations

import math

import numpy as np

from .sq_oracle import entropy_fn, fd_weights, fermi


def _symbols(n_o, nq):
    w, g = fd_weights(n_o)
    t = 2.0 * math.pi * np.arange(nq) / nq - math.pi
    s = -w[0] - 2.0 * sum(w[p] * np.cos(p * t) for p in range(1, n_o + 1))
    G = 2.0 * sum(g[p] * np.sin(p * t) for p in range(1, n_o + 1))
    return t, s, G


def bz_values(mu, kT, h, n_o, nq=96):
    """Infinite free-electron grid at chemical potential mu: rho, energy densities and
    the diagonal kinetic stresses (paper form and second-difference form)."""
    h = np.asarray(h, dtype=np.float64)
    _, s, G = _symbols(n_o, nq)
    sz, sy, sx = np.meshgrid(s / (2 * h[2] ** 2), s / (2 * h[1] ** 2), s / (2 * h[0] ** 2), indexing="ij")
    eps = sx + sy + sz
    x = (eps - mu) / kT
    gg = fermi(x)
    dV = float(np.prod(h))
    out = {
        "rho": 2.0 / dV * float(np.mean(gg)),
        "E_band_density": 2.0 / dV * float(np.mean(gg * eps)),
        "E_s_density": 2.0 * kT / dV * float(np.mean(entropy_fn(x))),
    }
    sig_paper = np.zeros(3)
    sig_d2 = np.zeros(3)
    for a in range(3):
        ax = 2 - a
        shape = [1, 1, 1]
        shape[ax] = nq
        G2 = (G * G).reshape(shape)
        sa = s.reshape(shape)
        sig_paper[a] = -2.0 / dV * float(np.mean(gg * G2)) / h[a] ** 2
        sig_d2[a] = -2.0 / dV * float(np.mean(gg * sa)) / h[a] ** 2
    out["sigma_paper_diag"] = sig_paper
    out["sigma_d2_diag"] = sig_d2
    return out


def _restricted_1d(n_o, h, m):
    w, g = fd_weights(n_o)
    n = 2 * m + 1
    D2 = w[0] * np.eye(n)
    G1 = np.zeros((n, n))
    for p in range(1, n_o + 1):
        D2 += w[p] * (np.eye(n, k=p) + np.eye(n, k=-p))
        G1 += g[p] * (np.eye(n, k=p) - np.eye(n, k=-p))
    return -0.5 * D2 / h ** 2, G1 / h


def separable_region(f, h, n_o, m):
    """Exact [f(H_q)]_qq and [grad_a grad_a f(H_q)]_qq (a = x, y, z) for V = 0 on the
    region of half-widths m (3,), by three 1-D eigendecompositions."""
    lam, p, k = [], [], []
    for a in range(3):
        A, G1 = _restricted_1d(n_o, float(h[a]), int(m[a]))
        e, U = np.linalg.eigh(A)
        c = int(m[a])
        lam.append(e)
        p.append(U[c, :] ** 2)
        k.append((G1 @ G1 @ U)[c, :] * U[c, :])
    lz, ly, lx = np.meshgrid(lam[2], lam[1], lam[0], indexing="ij")
    fv = f(lx + ly + lz)
    diag = float(np.einsum("zyx,z,y,x->", fv, p[2], p[1], p[0]))
    kin = np.array([
        float(np.einsum("zyx,z,y,x->", fv, p[2], p[1], k[0])),
        float(np.einsum("zyx,z,y,x->", fv, p[2], k[1], p[0])),
        float(np.einsum("zyx,z,y,x->", fv, k[2], p[1], p[0])),
    ])
    return diag, kin
