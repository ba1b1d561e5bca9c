"""k-integrated dense diagonalisation of the periodic grid Hamiltonian (FP64, CPU).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py). Independent of the SQ sweep: it uses
Bloch-phase matrices on the unit cell and a uniform grid of Bloch phases theta in
[-pi, pi)^3, so as the grid is refined it gives the infinite-crystal density matrix that
the infinite-cell SQ method approximates without Brillouin-zone integration (Sec. 4).

It provides
  * rho, N, E_band, E_s (= -TS), E_nl and the density-matrix stress of Eq. (ON:Stress)
    restricted to its kinetic and nonlocal terms (Eqs. stressIRe / stressIIIRe), in the
    paper's discrete form (first-derivative products grad_a grad_b, (x - R)_b grad_a),
  * the "strain-consistent" stress 2 tr(D dH/dF_ab) / |Omega| of the same discrete
    Hamiltonian (second-difference stencil on the diagonal, analytic projector gradient),
  * the Mermin free energy of the homogeneously strained cell F = I + e E_ab, so that the
    stress definition of Eq. (stressdefinition) can be checked by finite differences.
"""
from __future__ import annotations

import math

import numpy as np

from .sq_oracle import Problem, entropy_fn, fermi, projector_gradient, projector_value


def theta_grid(nk):
    """Uniform, Gamma-free grid of Bloch phases per axis: theta_i = 2 pi (i + 1/2) / nk - pi."""
    nk = [int(x) for x in np.broadcast_to(nk, (3,))]
    axes = [2.0 * math.pi * (np.arange(k) + 0.5) / k - math.pi for k in nk]
    tz, ty, tx = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    return np.stack([tx.ravel(), ty.ravel(), tz.ravel()], axis=1)


def bloch_1d(n: int, coefs, theta: float, odd: bool, center: float = 0.0) -> np.ndarray:
    """(M f)_i = center f_i + sum_p c_p (f_{i+p} +- f_{i-p}) on n periodic points with the
    Bloch condition f_{i+n} = exp(i theta) f_i (odd selects the minus sign)."""
    M = np.zeros((n, n), dtype=np.complex128)
    for i in range(n):
        M[i, i] += center
        for p in range(1, len(coefs)):
            for sgn, fac in ((1, 1.0), (-1, -1.0 if odd else 1.0)):
                j = i + sgn * p
                wraps = j // n
                M[i, j % n] += fac * coefs[p] * np.exp(1j * theta * wraps)
    return M


def _kron3(mx, my, mz):
    return np.kron(mz, np.kron(my, mx))


class BlochOps:
    """Grid operators of one Problem at one Bloch phase theta (3,)."""

    def __init__(self, prob: Problem, theta):
        self.prob = prob
        n = prob.n
        self.I = [np.eye(int(n[a]), dtype=np.complex128) for a in range(3)]
        self.D2 = []        # second-difference stencils / h^2, embedded in 3-D
        self.G = []         # first-derivative matrices / h, embedded in 3-D
        for a in range(3):
            d2 = bloch_1d(int(n[a]), prob.w, theta[a], odd=False, center=prob.w[0]) / prob.h[a] ** 2
            g1 = bloch_1d(int(n[a]), prob.g, theta[a], odd=True) / prob.h[a]
            mats = list(self.I)
            mats[a] = d2
            self.D2.append(_kron3(*mats))
            mats = list(self.I)
            mats[a] = g1
            self.G.append(_kron3(*mats))
        self.theta = np.asarray(theta, dtype=np.float64)
        # reference node positions X (N_d, 3), x fastest
        iz, iy, ix = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
        self.X = np.stack([ix.ravel() * prob.h[0], iy.ravel() * prob.h[1], iz.ravel() * prob.h[2]], axis=1)

    def projector_blochs(self, F=None, with_grad=False):
        """For every projector row r: b_r(y) = sum_s chi_r(F (X_y + s L - R_J)) exp(i theta.s),
        and (optionally) phi_rab(y) = sum_s chi_r(u) u_b e^{i theta.s} with u = X_y + s L - R_J,
        and db_rab(y) = sum_s (d_a chi_r)(u) u_b e^{i theta.s}."""
        prob = self.prob
        F = np.eye(3) if F is None else np.asarray(F, dtype=np.float64)
        rows = []
        for (J, l, ch, width, gamma, rc) in prob.rows:
            R = prob.pos[J]
            # images: any s with some node within reach (generous, sqrt(3) for shear)
            reach = 1.5 * rc
            rng = [range(int(math.floor((-reach - R[a]) / prob.L[a])) - 1,
                         int(math.ceil((prob.L[a] + reach - R[a]) / prob.L[a])) + 2) for a in range(3)]
            b = np.zeros(prob.Nd, dtype=np.complex128)
            phi = np.zeros((3, prob.Nd), dtype=np.complex128) if with_grad else None
            db = np.zeros((3, 3, prob.Nd), dtype=np.complex128) if with_grad else None
            for sz in rng[2]:
                for sy in rng[1]:
                    for sx in rng[0]:
                        s = np.array([sx, sy, sz], dtype=np.float64)
                        u = self.X + s * prob.L - R
                        Fu = u @ F.T
                        if np.min(np.einsum("ij,ij->i", Fu, Fu)) > rc * rc:
                            continue
                        ph = np.exp(1j * float(np.dot(self.theta, s)))
                        v = projector_value(l, ch, width, rc, Fu)
                        b += ph * v
                        if with_grad:
                            gr = projector_gradient(l, ch, width, rc, u)
                            v0 = projector_value(l, ch, width, rc, u)
                            for bb in range(3):
                                phi[bb] += ph * v0 * u[:, bb]
                                for a in range(3):
                                    db[a, bb] += ph * gr[:, a] * u[:, bb]
            rows.append((gamma, b, phi, db))
        return rows

    def hamiltonian(self, F=None, rows=None):
        prob = self.prob
        F = np.eye(3) if F is None else np.asarray(F, dtype=np.float64)
        Finv = np.linalg.inv(F)
        A = Finv @ Finv.T
        H = np.diag(prob.v.reshape(-1)).astype(np.complex128)
        for c in range(3):
            for d in range(3):
                if abs(A[c, d]) < 1e-300:
                    continue
                Kcd = self.D2[c] if c == d else self.G[c] @ self.G[d]
                H += -0.5 * A[c, d] * Kcd
        if rows is None:
            rows = self.projector_blochs(F)
        detF = float(np.linalg.det(F))
        for (gamma, b, _, _) in rows:
            H += gamma * prob.dV * detF * np.outer(np.conj(b), b)
        return H


def _solve_mu(eigs, n_e, kT, weights, lo, hi, iters=200):
    def count(mu):
        return 2.0 * sum(wk * float(np.sum(fermi((e - mu) / kT))) for e, wk in zip(eigs, weights))
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if count(mid) < n_e:
            lo = mid
        else:
            hi = mid
        if hi - lo < 1e-14 * max(1.0, abs(mid)):
            break
    return 0.5 * (lo + hi)


def observables(prob: Problem, nk=4, mu=None):
    """Infinite-crystal (k-integrated) rho, energies and both stress forms at fixed N_e
    (mu from bisection) or at a given mu."""
    thetas = theta_grid(nk)
    wk = 1.0 / len(thetas)
    data = []
    for th in thetas:
        ops = BlochOps(prob, th)
        rows = ops.projector_blochs(with_grad=True)
        H = ops.hamiltonian(rows=rows)
        e, U = np.linalg.eigh(H)
        data.append((ops, rows, H, e, U))
    if mu is None:
        emin = min(float(d[3][0]) for d in data)
        emax = max(float(d[3][-1]) for d in data)
        mu = _solve_mu([d[3] for d in data], prob.n_e, prob.kT, [wk] * len(data),
                       emin - 40 * prob.kT, emax + 40 * prob.kT)
    N = 0.0
    E_band = 0.0
    E_s = 0.0
    E_nl = 0.0
    rho = np.zeros(prob.Nd)
    sig_I = np.zeros((3, 3))
    sig_S = np.zeros((3, 3))          # the -4 sum gamma ... (X_b - R_b) grad_a term
    sig_kin_strain = np.zeros((3, 3))
    sig_nl_strain = np.zeros((3, 3))
    for (ops, rows, H, e, U) in data:
        gn = fermi((e - mu) / prob.kT)
        D = (U * gn) @ U.conj().T                      # D_ij = sum_n g_n psi_n(i) psi_n(j)^*
        N += 2.0 * wk * float(np.sum(gn))
        E_band += 2.0 * wk * float(np.sum(gn * e))
        E_s += 2.0 * prob.kT * wk * float(np.sum(entropy_fn((e - mu) / prob.kT)))
        rho += 2.0 / prob.dV * wk * np.real(np.diag(D))
        enl = 0.0
        for (gamma, b, phi, db) in rows:
            # psi^H V psi summed: tr(D conj(b) b^T) = b^T D conj(b)
            enl += gamma * prob.dV * float(np.real(b @ D @ np.conj(b)))
        E_nl += 2.0 * wk * enl
        for a in range(3):
            for bb in range(3):
                sig_I[a, bb] += 2.0 * wk * float(np.real(np.trace(D @ (ops.G[a] @ ops.G[bb]))))
                K = ops.D2[a] if a == bb else ops.G[a] @ ops.G[bb]
                sig_kin_strain[a, bb] += 2.0 * wk * float(np.real(np.trace(D @ K)))
                sacc = 0.0
                nacc = 0.0
                for (gamma, b, phi, db) in rows:
                    # sum_n g (phi_b^T grad_a psi_n) conj(b^T psi_n) = phi_b^T grad_a D conj(b)
                    sacc += gamma * prob.dV * float(np.real(phi[bb] @ (ops.G[a] @ (D @ np.conj(b)))))
                    # tr(D [conj(db) b^T + conj(b) db^T]) = b^T D conj(db) + db^T D conj(b)
                    nacc += gamma * prob.dV * float(np.real(b @ D @ np.conj(db[a, bb])
                                                            + db[a, bb] @ D @ np.conj(b)))
                sig_S[a, bb] += -4.0 * wk * sacc
                sig_nl_strain[a, bb] += 2.0 * wk * nacc
    eye = np.eye(3)
    sigma_paper = (sig_I - E_nl * eye + sig_S) / prob.vol
    sigma_strain = (sig_kin_strain + E_nl * eye + sig_nl_strain) / prob.vol
    return {
        "mu": mu, "N": N, "E_band": E_band, "E_s": E_s, "E_nl": E_nl, "F": E_band + E_s,
        "rho": rho, "sigma": sigma_paper, "sigma_strain": sigma_strain,
        "sigma_I": sig_I / prob.vol,
        "sigma_III": (sig_S - E_nl * eye) / prob.vol,
        "sigma_III_strain": (sig_nl_strain + E_nl * eye) / prob.vol,
    }


def free_energy(prob: Problem, F, nk=4):
    """Mermin free energy Omega(mu) + mu N_e = E_band - TS of the cell strained by F, at
    fixed N_e. V_eff is held fixed in index space; nonlocal projectors move affinely."""
    thetas = theta_grid(nk)
    wk = 1.0 / len(thetas)
    eigs = []
    for th in thetas:
        ops = BlochOps(prob, th)
        eigs.append(np.linalg.eigvalsh(ops.hamiltonian(F=F)))
    emin = min(float(e[0]) for e in eigs)
    emax = max(float(e[-1]) for e in eigs)
    mu = _solve_mu(eigs, prob.n_e, prob.kT, [wk] * len(eigs), emin - 40 * prob.kT, emax + 40 * prob.kT)
    omega = 0.0
    for e in eigs:
        x = (e - mu) / prob.kT
        omega += -2.0 * prob.kT * wk * float(np.sum(np.logaddexp(0.0, -x)))
    return omega + mu * prob.n_e


def strain_fd_stress(prob: Problem, a: int, b: int, nk=4, eps=1e-3):
    """(1/|Omega|) dF/dF_ab by central differences at eps and 2 eps, Richardson-combined."""
    def deriv(e):
        E = np.zeros((3, 3))
        E[a, b] = 1.0
        fp = free_energy(prob, np.eye(3) + e * E, nk)
        fm = free_energy(prob, np.eye(3) - e * E, nk)
        return (fp - fm) / (2.0 * e)
    return (4.0 * deriv(eps) - deriv(2.0 * eps)) / 3.0 / prob.vol
