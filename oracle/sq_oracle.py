"""FP64 CPU oracle of the infinite-cell Clenshaw-Curtis SQ sweep (Sec. 4 of the paper).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py). Plain, slow and meant to be read
against the paper: every nodal quantity is built from its definition on the node's
region of influence, with no blocking, batching or fusion across nodes.

Notation (paper -> code)
  K_Omega, N_d          prob.n (nodes per side), prob.Nd
  |dOmega| = h1 h2 h3   prob.dV ;  |Omega| = prob.vol
  region of influence   cube of side 2 R_cut around node q: offsets k in [-m, m]^3,
                        m_a = floor(R_cut / h_a + 1e-9)  (N_c = prod(2 m_a + 1))
  H_q                   restriction (zero extension) of H = -1/2 Lap_h + V_eff + V_nl
  chi_q, zeta_q         spectral centre / half-width: (lambda_max +- lambda_min) / 2
  t_q^j                 q-th column of T_j(Hhat_q), Hhat_q = (H_q - chi_q I) / zeta_q
  c^j, d^j, s^j         Chebyshev coefficients of g(r), r g(r) and the entropy function
  chi_Ilm, gamma_Jl     Kleinman-Bylander projectors (Gaussian s / p) and energies

Moment table layout, per node and per j = 0..n_pl (17 doubles):
  0        rho^j        = w_q^T t^j
  1..6     K^j_ab       = w_q^T grad_a,q grad_b,q t^j  for ab = xx, yy, zz, yz, xz, xy
  7        N^j          = w_q^T V_nl,q t^j
  8..16    S^j_ab       = sum_I w_q^T V^I_nl,q (X_b,q - R_I,b) grad_a,q t^j   (index 8+3a+b)
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import scipy.linalg
import scipy.sparse

N_MOM = 17
K_PAIRS = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))   # moment slots 1..6


# ----------------------------------------------------------------------------------------
# Finite differences (the paper's "twelfth-order" discretisation is the n_o = 6 member of
# the central 2 n_o-order family; the weights below are the closed forms of that family).
# ----------------------------------------------------------------------------------------
def fd_weights(n_o: int):
    """Central 2n_o-order weights.

    Second derivative: f''(x) h^2 ~ w[0] f(x) + sum_p w[p] (f(x+ph) + f(x-ph)),
        w[p] = 2 (-1)^(p+1) (n_o!)^2 / (p^2 (n_o-p)! (n_o+p)!),  w[0] = -2 sum_p w[p].
    First derivative:  f'(x) h ~ sum_p g[p] (f(x+ph) - f(x-ph)),
        g[p] = (-1)^(p+1) (n_o!)^2 / (p (n_o-p)! (n_o+p)!).
    """
    if not 1 <= n_o <= 8:
        raise ValueError("n_o out of range")
    w = [Fraction(0)] * (n_o + 1)
    g = [Fraction(0)] * (n_o + 1)
    fno = math.factorial(n_o)
    for p in range(1, n_o + 1):
        base = Fraction(fno * fno, math.factorial(n_o - p) * math.factorial(n_o + p))
        sgn = 1 if p % 2 == 1 else -1
        w[p] = 2 * sgn * base / (p * p)
        g[p] = sgn * base / p
    w[0] = -2 * sum(w[1:])
    return np.array([float(x) for x in w]), np.array([float(x) for x in g])


# ----------------------------------------------------------------------------------------
# Gaussian Kleinman-Bylander projectors (stand-in for the paper's pseudopotential
# projectors; normalised so that the continuum integral of chi^2 is 1).
# ----------------------------------------------------------------------------------------
def projector_value(l: int, ch: int, width: float, rcut: float, d: np.ndarray) -> np.ndarray:
    """chi_lm(d) for displacement d = x - R (shape (..., 3)); zero beyond |d| > rcut.
    l = 0: (pi w^2)^(-3/4) exp(-r^2 / (2 w^2));  l = 1, ch = x|y|z: sqrt(2)/w * d_ch * (same)."""
    r2 = np.sum(d * d, axis=-1)
    base = (math.pi * width * width) ** (-0.75) * np.exp(-r2 / (2.0 * width * width))
    if l == 0:
        val = base
    elif l == 1:
        val = math.sqrt(2.0) / width * d[..., ch] * base
    else:
        raise ValueError("only s and p projectors")
    return np.where(r2 <= rcut * rcut, val, 0.0)


def projector_gradient(l: int, ch: int, width: float, rcut: float, d: np.ndarray) -> np.ndarray:
    """Analytic gradient d chi_lm / d d_alpha, shape (..., 3) (zero beyond rcut)."""
    r2 = np.sum(d * d, axis=-1)
    w2 = width * width
    base = (math.pi * w2) ** (-0.75) * np.exp(-r2 / (2.0 * w2))
    if l == 0:
        grad = -d / w2 * base[..., None]
    else:
        c = math.sqrt(2.0) / width
        grad = -d / w2 * (c * d[..., ch] * base)[..., None]
        grad[..., ch] += c * base
    return np.where((r2 <= rcut * rcut)[..., None], grad, 0.0)


class Problem:
    """An SQ instance (dict from workloads.sq_workloads) with derived grid quantities."""

    def __init__(self, inst: dict):
        self.inst = inst
        self.L = np.asarray(inst["L"], dtype=np.float64)
        self.n = np.asarray(inst["n"], dtype=np.int64)
        self.n_o = int(inst["n_o"])
        self.h = self.L / self.n
        self.dV = float(np.prod(self.h))
        self.vol = float(np.prod(self.L))
        self.Nd = int(np.prod(self.n))
        self.r_cut = float(inst["r_cut"])
        self.m = np.array([int(math.floor(self.r_cut / self.h[a] + 1e-9)) for a in range(3)])
        self.Nc = int(np.prod(2 * self.m + 1))
        self.kT = float(inst["kT"])
        self.n_e = float(inst["n_e"])
        self.n_pl = int(inst["n_pl"])
        self.M = int(inst.get("M", 2048))
        self.v = np.asarray(inst["v_eff"], dtype=np.float64).reshape(self.n[2], self.n[1], self.n[0])
        self.pos = np.asarray(inst["pos"], dtype=np.float64).reshape(-1, 3)
        self.species = np.asarray(inst["species"], dtype=np.int64).reshape(-1)
        self.w, self.g = fd_weights(self.n_o)
        # one row per (atom, projector, channel): (atom, l, ch, width, gamma, rcut)
        self.rows = []
        for J in range(self.pos.shape[0]):
            for pj in inst["proj"][int(self.species[J])]:
                rc = pj.get("rcut", 0.0)
                rc = 7.0 * pj["width"] if rc is None or rc <= 0.0 else rc
                for ch in range(2 * pj["l"] + 1):
                    self.rows.append((J, pj["l"], ch, pj["width"], pj["gamma"], rc))
        if np.any(self.m < 1):
            raise ValueError("truncation region must contain neighbours (m >= 1)")

    # node q given as integer lattice coordinates (qx, qy, qz); index = qx + n0 (qy + n1 qz)
    def node_coords(self, idx: int):
        qx = idx % self.n[0]
        qy = (idx // self.n[0]) % self.n[1]
        qz = idx // (self.n[0] * self.n[1])
        return np.array([qx, qy, qz], dtype=np.int64)


# ----------------------------------------------------------------------------------------
# The nodal Hamiltonian H_q (Sec. 4): restriction of the infinite-crystal grid Hamiltonian
# to the region of influence of q, i.e. zero extension outside the region.
# Region arrays are indexed [kz, ky, kx]; Cartesian axis a lives on numpy axis 2 - a.
# ----------------------------------------------------------------------------------------
def _shift(t: np.ndarray, p: int, a: int) -> np.ndarray:
    """s[k] = t[k + p e_a], zero where k + p e_a leaves the region."""
    ax = 2 - a
    s = np.zeros_like(t)
    nax = t.shape[ax]
    if abs(p) >= nax:
        return s
    dst = [slice(None)] * 3
    src = [slice(None)] * 3
    if p > 0:
        dst[ax] = slice(0, nax - p)
        src[ax] = slice(p, nax)
    else:
        dst[ax] = slice(-p, nax)
        src[ax] = slice(0, nax + p)
    s[tuple(dst)] = t[tuple(src)]
    return s


class NodeRegion:
    """Operators restricted to the region of influence of one node q."""

    def __init__(self, prob: Problem, q, half=None):
        self.prob = prob
        self.q = np.asarray(q, dtype=np.int64)
        self.m = prob.m if half is None else np.asarray(half, dtype=np.int64)
        self.shape = tuple(int(2 * self.m[2 - ax] + 1) for ax in range(3))   # (z, y, x)
        self.center = tuple(int(self.m[2 - ax]) for ax in range(3))
        # absolute (unwrapped) lattice coordinates of the region points
        offs = [np.arange(-self.m[a], self.m[a] + 1) + self.q[a] for a in range(3)]
        self.lat = offs
        uz, uy, ux = np.meshgrid(offs[2], offs[1], offs[0], indexing="ij")
        self.X = np.stack([ux * prob.h[0], uy * prob.h[1], uz * prob.h[2]], axis=-1)  # (z,y,x,3)
        self.V = prob.v[np.mod(uz, prob.n[2]), np.mod(uy, prob.n[1]), np.mod(ux, prob.n[0])]
        self._build_projectors()

    def _build_projectors(self):
        """All projector rows chi_Ilm of atom images I in R^3 whose support meets the region
        (the set D^c of Sec. 4), sampled at the unwrapped region coordinates."""
        prob = self.prob
        lo = np.array([self.lat[a][0] for a in range(3)]) * prob.h
        hi = np.array([self.lat[a][-1] for a in range(3)]) * prob.h
        vals, gam, cen, img_R, meta = [], [], [], [], []
        xq = self.q * prob.h
        for (J, l, ch, width, gamma, rc) in prob.rows:
            R0 = prob.pos[J]
            rng = []
            for a in range(3):
                s_lo = int(math.floor((lo[a] - rc - R0[a]) / prob.L[a])) - 1
                s_hi = int(math.ceil((hi[a] + rc - R0[a]) / prob.L[a])) + 1
                rng.append(range(s_lo, s_hi + 1))
            for sz in rng[2]:
                for sy in rng[1]:
                    for sx in rng[0]:
                        R = R0 + np.array([sx, sy, sz]) * prob.L
                        # distance from R to the region box
                        dbox = np.maximum(0.0, np.maximum(lo - R, R - hi))
                        if np.dot(dbox, dbox) > rc * rc:
                            continue
                        v = projector_value(l, ch, width, rc, self.X - R)
                        if not np.any(v):
                            continue
                        vals.append(v.reshape(-1))
                        gam.append(gamma)
                        cen.append(float(projector_value(l, ch, width, rc, (xq - R)[None, :])[0]))
                        img_R.append(R)
                        meta.append((J, l, ch, width, rc))
        nc = int(np.prod(self.shape))
        if vals:
            self.chi = scipy.sparse.csr_matrix(np.vstack(vals))
        else:
            self.chi = scipy.sparse.csr_matrix((0, nc))
        self.gamma = np.asarray(gam, dtype=np.float64)
        self.chi_at_q = np.asarray(cen, dtype=np.float64)
        self.R_img = np.asarray(img_R, dtype=np.float64).reshape(-1, 3)
        self.meta = meta
        # w_q^T V^I_nl,q = sum_lm gamma h^3 chi_Ilm(x_q) chi_Ilm^T ; contract over rows once:
        a_r = self.gamma * prob.dV * self.chi_at_q
        self.W0 = np.asarray(self.chi.T @ a_r).reshape(self.shape)            # for N^j
        self.Wb = []
        Xf = self.X.reshape(-1, 3)
        for b in range(3):                                                   # for S^j_ab
            wb = np.zeros(nc)
            for r in np.nonzero(a_r)[0]:
                row = self.chi.getrow(r)
                idx = row.indices
                wb[idx] += a_r[r] * row.data * (Xf[idx, b] - self.R_img[r, b])
            self.Wb.append(wb.reshape(self.shape))

    # -- operator pieces -------------------------------------------------------------------
    def d2(self, t, a):
        """Second-difference stencil along axis a (times h_a^2), restricted."""
        w = self.prob.w
        out = w[0] * t
        for p in range(1, self.prob.n_o + 1):
            out = out + w[p] * (_shift(t, p, a) + _shift(t, -p, a))
        return out

    def grad(self, t, a):
        """Restricted first-derivative matrix grad_a,q applied to t."""
        g = self.prob.g
        out = np.zeros_like(t)
        for p in range(1, self.prob.n_o + 1):
            out = out + g[p] * (_shift(t, p, a) - _shift(t, -p, a))
        return out / self.prob.h[a]

    def apply_nl(self, t):
        """V_nl,q t = sum_I sum_lm gamma_Jl h^3 chi_Ilm (chi_Ilm^T t)."""
        if self.chi.shape[0] == 0:
            return np.zeros_like(t)
        p = self.prob.dV * (self.chi @ t.reshape(-1))
        return np.asarray(self.chi.T @ (self.gamma * p)).reshape(t.shape)

    def apply_H(self, t):
        """H_q t = -1/2 sum_a (D2_a / h_a^2) t + V t + V_nl t on the region (zero extension)."""
        out = self.V * t
        for a in range(3):
            out = out - 0.5 / self.prob.h[a] ** 2 * self.d2(t, a)
        return out + self.apply_nl(t)

    def dense_H(self):
        """H_q as a dense matrix, assembled from Kronecker products of 1-D matrices (an
        independent construction of the same operator, used by the exact-polynomial pin)."""
        prob = self.prob
        eye = [np.eye(s) for s in self.shape]                                # (z, y, x)
        H = np.diag(self.V.reshape(-1)).astype(np.float64)
        for a in range(3):
            nax = self.shape[2 - a]
            D = prob.w[0] * np.eye(nax)
            for p in range(1, prob.n_o + 1):
                D += prob.w[p] * (np.eye(nax, k=p) + np.eye(nax, k=-p))
            mats = [eye[0], eye[1], eye[2]]
            mats[2 - a] = D
            H -= 0.5 / prob.h[a] ** 2 * np.kron(np.kron(mats[0], mats[1]), mats[2])
        if self.chi.shape[0]:
            C = self.chi.toarray()
            H += C.T @ np.diag(self.gamma * prob.dV) @ C
        return H

    def dense_grad(self, a):
        prob = self.prob
        eye = [np.eye(s) for s in self.shape]
        nax = self.shape[2 - a]
        G = np.zeros((nax, nax))
        for p in range(1, prob.n_o + 1):
            G += prob.g[p] * (np.eye(nax, k=p) - np.eye(nax, k=-p))
        mats = [eye[0], eye[1], eye[2]]
        mats[2 - a] = G / prob.h[a]
        return np.kron(np.kron(mats[0], mats[1]), mats[2])

    def unit(self):
        e = np.zeros(self.shape)
        e[self.center] = 1.0
        return e

    # -- moments of one Chebyshev column ---------------------------------------------------
    def moments(self, t):
        """The 17 moments of t = t_q^j (layout in the module docstring)."""
        c = self.center
        out = np.zeros(N_MOM)
        out[0] = t[c]
        g = [self.grad(t, a) for a in range(3)]
        for slot, (a, b) in enumerate(K_PAIRS):
            out[1 + slot] = self.grad(g[b], a)[c]
        out[7] = float(np.sum(self.W0 * t))
        for a in range(3):
            for b in range(3):
                out[8 + 3 * a + b] = float(np.sum(self.Wb[b] * g[a]))
        return out

    def d2_at_center(self, t):
        """L_a = [D2_a t]_q / h_a^2 (the second-difference form of the diagonal kinetic term)."""
        c = self.center
        return np.array([self.d2(t, a)[c] / self.prob.h[a] ** 2 for a in range(3)])


def chebyshev_columns(region: NodeRegion, chi_q: float, zeta_q: float, n_pl: int):
    """t^0 = w_q, t^1 = Hhat w_q, t^{i+1} = 2 Hhat t^i - t^{i-1}  (Sec. 4), i.e. the q-th
    columns of T_j(Hhat_q) for j = 0..n_pl."""
    def hhat(t):
        return (region.apply_H(t) - chi_q * t) / zeta_q
    cols = [region.unit()]
    if n_pl >= 1:
        cols.append(hhat(cols[0]))
    for _ in range(1, n_pl):
        cols.append(2.0 * hhat(cols[-1]) - cols[-2])
    return cols


def node_moments(prob: Problem, q, lam_lo: float, lam_hi: float, with_d2: bool = False):
    """Moment table rows (n_pl + 1, 17) of node q (integer lattice coordinates)."""
    region = NodeRegion(prob, q)
    chi_q = 0.5 * (lam_hi + lam_lo)
    zeta_q = 0.5 * (lam_hi - lam_lo)
    cols = chebyshev_columns(region, chi_q, zeta_q, prob.n_pl)
    mom = np.array([region.moments(t) for t in cols])
    if with_d2:
        return mom, np.array([region.d2_at_center(t) for t in cols])
    return mom


# ----------------------------------------------------------------------------------------
# Clenshaw-Curtis coefficients (Sec. 4): c^j = (2/pi) int_{-1}^{1} f(r) T_j(r) / sqrt(1-r^2) dr,
# evaluated by M-point Chebyshev-Gauss quadrature (exact for polynomial f of degree < 2M - j).
# ----------------------------------------------------------------------------------------
def cheb_coeffs(f, n_pl: int, M: int) -> np.ndarray:
    theta = math.pi * (np.arange(M) + 0.5) / M
    fv = f(np.cos(theta))
    j = np.arange(n_pl + 1)
    return (2.0 / M) * (np.cos(np.outer(j, theta)) @ fv)


def fermi(x):
    """g = 1 / (1 + exp(x)), evaluated without overflow."""
    x = np.asarray(x, dtype=np.float64)
    ex = np.exp(-np.abs(x))
    return np.where(x > 0, ex / (1.0 + ex), 1.0 / (1.0 + ex))


def entropy_fn(x):
    """s = g ln g + (1-g) ln(1-g) at g = fermi(x), in the stable form
    -[ln(1 + e^-|x|) + |x| e^-|x| / (1 + e^-|x|)]  (always <= 0)."""
    x = np.abs(np.asarray(x, dtype=np.float64))
    ex = np.exp(-x)
    return -(np.log1p(ex) + x * ex / (1.0 + ex))


def fd_coefficients(mu, kT, chi_q, zeta_q, n_pl, M):
    """(c, d, s): coefficients of g(r), r g(r) and the entropy function in the scaled
    variable r = (lambda - chi_q) / zeta_q, with g the Fermi-Dirac function at (mu, kT)."""
    def xr(r):
        return (chi_q + zeta_q * r - mu) / kT
    c = cheb_coeffs(lambda r: fermi(xr(r)), n_pl, M)
    d = cheb_coeffs(lambda r: r * fermi(xr(r)), n_pl, M)
    s = cheb_coeffs(lambda r: entropy_fn(xr(r)), n_pl, M)
    return c, d, s


def primed(n_pl: int) -> np.ndarray:
    """Weights of the primed sum: the j = 0 term is halved."""
    wp = np.ones(n_pl + 1)
    wp[0] = 0.5
    return wp


# ----------------------------------------------------------------------------------------
# Fermi level: bisection on N(mu) = 2 sum_q sum'_j c^j(mu) rho_q^j = N_e (the paper does not
# say how mu is found; this rule is shared with the library).
# ----------------------------------------------------------------------------------------
class NoBracket(RuntimeError):
    pass


def electron_count(R, mu, kT, chi_q, zeta_q, M):
    n_pl = len(R) - 1
    c = cheb_coeffs(lambda r: fermi((chi_q + zeta_q * r - mu) / kT), n_pl, M)
    return 2.0 * float(np.sum(primed(n_pl) * c * R))


def fermi_bisect(R, n_e, kT, lam_lo, lam_hi, M, max_iter=200, rtol=1e-13):
    chi_q = 0.5 * (lam_hi + lam_lo)
    zeta_q = 0.5 * (lam_hi - lam_lo)
    lo = lam_lo - 40.0 * kT
    hi = lam_hi + 40.0 * kT
    if not (electron_count(R, lo, kT, chi_q, zeta_q, M) < n_e < electron_count(R, hi, kT, chi_q, zeta_q, M)):
        raise NoBracket("N(mu) - N_e has no sign change on the bracket")
    for _ in range(max_iter):
        mid = 0.5 * (lo + hi)
        if electron_count(R, mid, kT, chi_q, zeta_q, M) < n_e:
            lo = mid
        else:
            hi = mid
        if hi - lo < rtol * max(1.0, abs(mid)):
            break
    return 0.5 * (lo + hi)


# ----------------------------------------------------------------------------------------
# Contraction (Sec. 4 density, stress sums; App. A band-energy form).
# ----------------------------------------------------------------------------------------
def contract(prob: Problem, mom: np.ndarray, mu: float, lam_lo: float, lam_hi: float):
    """mom: (N_d, n_pl+1, 17). Returns rho (N_d), energies and sigma (3x3, Ha/bohr^3)."""
    chi_q = 0.5 * (lam_hi + lam_lo)
    zeta_q = 0.5 * (lam_hi - lam_lo)
    c, d, s = fd_coefficients(mu, prob.kT, chi_q, zeta_q, prob.n_pl, prob.M)
    wp = primed(prob.n_pl)
    cw, dw, sw = wp * c, wp * d, wp * s
    rho_j = mom[:, :, 0]
    rho = 2.0 / prob.dV * (rho_j @ cw)
    E_band = 2.0 * float(np.sum(rho_j @ (chi_q * cw + zeta_q * dw)))
    E_s = 2.0 * prob.kT * float(np.sum(rho_j @ sw))
    E_nl = 2.0 * float(np.sum(mom[:, :, 7] @ cw))
    sig_I = np.zeros((3, 3))
    for slot, (a, b) in enumerate(K_PAIRS):
        v = 2.0 * float(np.sum(mom[:, :, 1 + slot] @ cw))
        sig_I[a, b] = v
        sig_I[b, a] = v
    sig_III = np.zeros((3, 3))
    for a in range(3):
        for b in range(3):
            S_ab = float(np.sum(mom[:, :, 8 + 3 * a + b] @ cw))
            sig_III[a, b] = -2.0 * ((E_nl / 2.0 if a == b else 0.0) + 2.0 * S_ab)
    sigma = (sig_I + sig_III) / prob.vol
    # App. A (Eq. ON:Pressure and its SQ form), restricted to the kinetic and nonlocal terms:
    # the first term -4 sum_q sum' (chi c^j + zeta d^j) rho^j_q is -4 tr(D H) = -2 E_band; its
    # V_eff part -2 |dOmega| sum_q V_q rho_q belongs with the exchange-correlation and
    # electrostatic terms (outside this path) and is taken out, leaving -4 tr(D (H - V_eff));
    # the nonlocal term -2 sum_q w_q^T V_nl,q (sum' c^j t^j + 2 (X - R) . grad sum' c^j t^j)
    # is -E_nl - 4 sum_q sum' c^j (S^j_xx + S^j_yy + S^j_zz).
    E_pot = prob.dV * float(np.sum(prob.v.reshape(-1) * rho))
    trS = float(np.sum((mom[:, :, 8] + mom[:, :, 12] + mom[:, :, 16]) @ cw))
    bracket = -2.0 * (E_band - E_pot) - E_nl - 4.0 * trS
    pressure_A = -bracket / (3.0 * prob.vol)
    return {
        "rho": rho,
        "E_band": E_band,
        "E_s": E_s,
        "E_nl": E_nl,
        "F": E_band + E_s,
        "N_check": prob.dV * float(np.sum(rho)),
        "sigma": sigma,
        "sigma_I": sig_I / prob.vol,
        "sigma_III": sig_III / prob.vol,
        "pressure": -float(np.trace(sigma)) / 3.0,
        "E_pot": E_pot,
        "pressure_A": pressure_A,
    }


# ----------------------------------------------------------------------------------------
# Spectral bounds (the paper uses the extreme eigenvalues of H_q without saying how they
# are found). Reading: k-step Lanczos with full reorthogonalisation on the regions of a few
# sample nodes, Ritz extremes widened by their residual norms, then by 1 % of the width.
# ----------------------------------------------------------------------------------------
def lanczos_start(nc: int, node_index: int) -> np.ndarray:
    i = np.arange(nc, dtype=np.uint64)
    hsh = (i * np.uint64(2654435761) + np.uint64(node_index) * np.uint64(40503)) & np.uint64(0xFFFFFFFF)
    v = 1.0 + (hsh % np.uint64(1009)).astype(np.float64) / 1009.0
    return v / np.linalg.norm(v)


def lanczos_extremes(apply, v0: np.ndarray, k: int):
    """k-step Lanczos with full reorthogonalisation by classical Gram-Schmidt applied twice:
    w = H v_i, c = V^T w, w -= V c, c' = V^T w, w -= V c', alpha_i = c_i + c'_i,
    beta_i = ||w||, v_{i+1} = w / beta_i (stop early when beta_i <= 1e-12 max(1, |alpha_i|)).
    Returns (theta_min - res_min, theta_max + res_max) of the tridiagonal (alpha, beta),
    res = beta_last |last component of the Ritz vector|."""
    V = [v0]
    alpha, beta = [], []
    for i in range(k):
        w = apply(V[i])
        Vm = np.array(V)
        c1 = Vm @ w
        w = w - Vm.T @ c1
        c2 = Vm @ w
        w = w - Vm.T @ c2
        a = float(c1[i] + c2[i])
        b = float(np.linalg.norm(w))
        alpha.append(a)
        beta.append(b)
        if i == k - 1 or b <= 1e-12 * max(1.0, abs(a)):
            break
        V.append(w / b)
    kk = len(alpha)
    theta, S = scipy.linalg.eigh_tridiagonal(np.array(alpha), np.array(beta[:kk - 1]))
    res = abs(beta[kk - 1]) * np.abs(S[-1, :])
    return float(theta[0] - res[0]), float(theta[-1] + res[-1])


def lanczos_sample_nodes(prob: Problem):
    """Seeds argmin V, argmax V and a stride-n/2 node grid; every node of the 2 x 2 x 2 node
    block (origin at even lattice coordinates) holding a seed is sampled, blocks in order of
    first appearance, nodes within a block x fastest."""
    v = prob.v.reshape(-1)
    seeds = [int(np.argmin(v)), int(np.argmax(v))]
    steps = [max(1, int(prob.n[a]) // 2) for a in range(3)]
    for iz in range(0, int(prob.n[2]), steps[2]):
        for iy in range(0, int(prob.n[1]), steps[1]):
            for ix in range(0, int(prob.n[0]), steps[0]):
                seeds.append(int(ix + prob.n[0] * (iy + prob.n[1] * iz)))
    blocks = []
    for q in seeds:
        blk = tuple(int(c) // 2 for c in prob.node_coords(q))
        if blk not in blocks:
            blocks.append(blk)
    nodes = []
    for blk in blocks:
        for dz in range(2):
            for dy in range(2):
                for dx in range(2):
                    c = (2 * blk[0] + dx, 2 * blk[1] + dy, 2 * blk[2] + dz)
                    if all(c[a] < prob.n[a] for a in range(3)):
                        nodes.append(int(c[0] + prob.n[0] * (c[1] + prob.n[1] * c[2])))
    return nodes


def lanczos_bounds(prob: Problem, k: int = 40):
    lo, hi = math.inf, -math.inf
    for qi in lanczos_sample_nodes(prob):
        region = NodeRegion(prob, prob.node_coords(qi))
        shape = region.shape
        v0 = lanczos_start(region.chi.shape[1], qi)
        l, h = lanczos_extremes(lambda x: region.apply_H(x.reshape(shape)).reshape(-1), v0,
                                min(k, region.chi.shape[1]))
        lo, hi = min(lo, l), max(hi, h)
    wdt = hi - lo
    return lo - 0.01 * wdt, hi + 0.01 * wdt


# ----------------------------------------------------------------------------------------
# Whole sweep
# ----------------------------------------------------------------------------------------
def _moments_worker(args):
    inst, nodes, lo, hi = args
    prob = Problem(inst)
    return np.array([node_moments(prob, prob.node_coords(q), lo, hi) for q in nodes])


def all_moments(prob: Problem, lam_lo: float, lam_hi: float, nodes=None, workers: int = 1):
    nodes = list(range(prob.Nd)) if nodes is None else list(nodes)
    if workers <= 1 or len(nodes) < 2 * workers:
        return np.array([node_moments(prob, prob.node_coords(q), lam_lo, lam_hi) for q in nodes])
    import multiprocessing as mp
    chunks = [nodes[i::workers] for i in range(workers)]
    with mp.get_context("spawn").Pool(workers) as pool:
        parts = pool.map(_moments_worker, [(prob.inst, ch, lam_lo, lam_hi) for ch in chunks])
    out = np.zeros((len(nodes), prob.n_pl + 1, N_MOM))
    for i, ch in enumerate(chunks):
        out[i::workers] = parts[i]
    return out


def run(inst: dict, bounds=None, workers: int = 1, lanczos_k: int = 40):
    """Full oracle: bounds -> moments of every node -> Fermi level -> rho, energies, sigma."""
    prob = Problem(inst)
    lo, hi = bounds if bounds is not None else lanczos_bounds(prob, lanczos_k)
    mom = all_moments(prob, lo, hi, workers=workers)
    R = mom[:, :, 0].sum(axis=0)
    mu = fermi_bisect(R, prob.n_e, prob.kT, lo, hi, prob.M)
    out = contract(prob, mom, mu, lo, hi)
    out.update({"mu": mu, "lambda_lo": lo, "lambda_hi": hi, "moments": mom, "R": R})
    return out
