"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics
(closed forms, exact diagonalisation, invariants, finite differences) - no GPU.

Each test names what a plausible mistake in the oracle would break."""
import json
import math
import os

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg

from oracle import dense_k, free_electron, gauss_sq, green_kubo, per_node
from oracle.sq_oracle import (K_PAIRS, NodeRegion, Problem, cheb_coeffs, chebyshev_columns, contract,
                              entropy_fn, fd_coefficients, fd_weights, fermi, fermi_bisect, lanczos_bounds,
                              node_moments, primed, run)
from workloads import make_instance, tiny_instance

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- finite differences
@pytest.mark.parametrize("n_o", [1, 2, 3, 4, 5, 6])
def test_fd_weights_match_vandermonde_solve(n_o):
    """Closed-form central weights == the unique weights exact on polynomials of degree
    <= 2 n_o (Taylor / Vandermonde conditions solved independently)."""
    w, g = fd_weights(n_o)
    p = np.arange(1, n_o + 1, dtype=np.float64)
    # second derivative: sum_p w_p 2 p^(2k) = 2 delta_{k,1} (k = 1..n_o) with symmetric taps
    A = np.array([2.0 * p ** (2 * k) for k in range(1, n_o + 1)])
    rhs = np.zeros(n_o)
    rhs[0] = 2.0
    np.testing.assert_allclose(w[1:], np.linalg.solve(A, rhs), rtol=1e-10, atol=1e-13)
    assert abs(w[0] + 2.0 * w[1:].sum()) < 1e-13
    # first derivative: sum_p g_p 2 p^(2k-1) = delta_{k,1}
    A1 = np.array([2.0 * p ** (2 * k - 1) for k in range(1, n_o + 1)])
    rhs1 = np.zeros(n_o)
    rhs1[0] = 1.0
    np.testing.assert_allclose(g[1:], np.linalg.solve(A1, rhs1), rtol=1e-10, atol=1e-13)


def test_fd_weights_n_o_3_values():
    w, g = fd_weights(3)
    np.testing.assert_allclose(w, [-49.0 / 18.0, 1.5, -0.15, 1.0 / 90.0], rtol=1e-14)
    np.testing.assert_allclose(g, [0.0, 0.75, -0.15, 1.0 / 60.0], rtol=1e-14)


def test_fd_spectral_sup():
    """sup of the 1-D second-difference symbol -w0 - 2 sum w_p cos(p t): 6.044 (n_o=3), 7.073 (n_o=6)."""
    t = np.linspace(0, math.pi, 20001)
    for n_o, want in ((3, 6.044), (6, 7.073)):
        w, _ = fd_weights(n_o)
        s = -w[0] - 2.0 * sum(w[p] * np.cos(p * t) for p in range(1, n_o + 1))
        assert abs(s.max() - want) < 2e-3
        assert s.min() > -1e-12           # the discrete -Laplacian is positive semidefinite


# ---------------------------------------------------------------- coefficients
def test_cheb_coeffs_match_adaptive_quadrature():
    """c^j = (2/pi) int g(r) T_j(r)/sqrt(1-r^2) dr (Sec. 4) against adaptive quadrature
    in theta (r = cos theta) - catches a wrong node set, weight or primed-sum convention."""
    mu_hat, sig_hat = 0.13, 0.07

    def g(r):
        return fermi((r - mu_hat) / sig_hat)
    c = cheb_coeffs(g, 40, 2048)
    for j in (0, 1, 2, 7, 25, 40):
        ref, _ = scipy.integrate.quad(lambda th: g(math.cos(th)) * math.cos(j * th), 0.0, math.pi,
                                      limit=400, epsabs=1e-15, epsrel=1e-13)
        assert abs(c[j] - 2.0 / math.pi * ref) < 1e-12
    # the primed series of enough terms reproduces g inside [-1, 1]
    c = cheb_coeffs(g, 400, 4096)
    r = np.linspace(-0.99, 0.99, 37)
    T = np.cos(np.outer(np.arange(401), np.arccos(r)))
    approx = (primed(400) * c) @ T
    assert np.abs(approx - g(r)).max() < 1e-12


def test_entropy_stable_form_matches_direct():
    x = np.linspace(-30, 30, 601)
    g = 1.0 / (1.0 + np.exp(x))
    direct = g * np.log(g) + (1 - g) * np.log1p(-g)
    ok = (g > 1e-12) & (g < 1 - 1e-12)
    np.testing.assert_allclose(entropy_fn(x)[ok], direct[ok], rtol=1e-9, atol=1e-14)
    assert entropy_fn(np.array([0.0]))[0] == pytest.approx(-math.log(2.0), rel=1e-15)


# ---------------------------------------------------------------- P1: exact polynomial identity
def _tiny_region(seed=3, n_o=2, half=(3, 3, 3)):
    inst = tiny_instance(seed=seed, n=(5, 5, 5), h=(0.7, 0.7, 0.7), n_atoms=3, n_o=n_o, r_cut=2.1, n_pl=12,
                         proj=[{"l": 0, "width": 0.6, "gamma": 1.0, "rcut": 3.0},
                               {"l": 1, "width": 0.6, "gamma": -0.4, "rcut": 3.0}])
    prob = Problem(inst)
    return prob, NodeRegion(prob, np.array([1, 2, 3]), half=np.array(half))


def test_p1_recurrence_equals_exact_chebyshev_columns():
    """t^j from the three-term recurrence == U cos(j arccos Lambda_hat) U^T e_q from eigh of the
    Kronecker-assembled dense H_q (independent operator construction)."""
    prob, reg = _tiny_region()
    H = reg.dense_H()
    lam, U = np.linalg.eigh(H)
    lo, hi = lam[0] - 0.3, lam[-1] + 0.2
    chi_q, zeta_q = 0.5 * (hi + lo), 0.5 * (hi - lo)
    cols = chebyshev_columns(reg, chi_q, zeta_q, 12)
    e = reg.unit().reshape(-1)
    th = np.arccos((lam - chi_q) / zeta_q)
    for j, t in enumerate(cols):
        exact = U @ (np.cos(j * th) * (U.T @ e))
        assert np.abs(t.reshape(-1) - exact).max() < 1e-12 * max(1.0, np.abs(exact).max())


def test_p1_moments_equal_dense_matrix_forms():
    """K, N, S of the oracle == the paper's matrix expressions built densely:
    K_ab = w^T grad_a grad_b t, N = w^T V_nl t, S_ab = sum_I w^T V^I (X_b - R_Ib) grad_a t (Sec. 4)."""
    prob, reg = _tiny_region()
    H = reg.dense_H()
    lam = np.linalg.eigvalsh(H)
    lo, hi = lam[0] - 0.3, lam[-1] + 0.2
    cols = chebyshev_columns(reg, 0.5 * (hi + lo), 0.5 * (hi - lo), 12)
    G = [reg.dense_grad(a) for a in range(3)]
    C = reg.chi.toarray()
    Vnl = C.T @ np.diag(reg.gamma * prob.dV) @ C
    e = reg.unit().reshape(-1)
    X = reg.X.reshape(-1, 3)
    # group projector rows by atom image (identical image position)
    imgs = {}
    for r, R in enumerate(reg.R_img):
        imgs.setdefault(tuple(np.round(R, 12)), []).append(r)
    for t in cols:
        tv = t.reshape(-1)
        mom = reg.moments(t)
        assert mom[0] == pytest.approx(tv[e.argmax()], abs=1e-15)
        for slot, (a, b) in enumerate(K_PAIRS):
            assert abs(mom[1 + slot] - e @ G[a] @ G[b] @ tv) < 1e-10 * (1 + abs(mom[1 + slot]))
        assert abs(mom[7] - e @ Vnl @ tv) < 1e-12
        for a in range(3):
            for b in range(3):
                s = 0.0
                for R, rows in imgs.items():
                    VI = C[rows].T @ np.diag(reg.gamma[rows] * prob.dV) @ C[rows]
                    s += e @ VI @ ((X[:, b] - R[b]) * (G[a] @ tv))
                assert abs(mom[8 + 3 * a + b] - s) < 1e-12 * (1 + abs(s))


# ---------------------------------------------------------------- P2: Chebyshev vs exact g(H_q)
def test_p2_density_matrix_column_within_chebyshev_tail():
    prob, reg = _tiny_region()
    H = reg.dense_H()
    lam, U = np.linalg.eigh(H)
    lo, hi = lam[0] - 0.3, lam[-1] + 0.2
    chi_q, zeta_q = 0.5 * (hi + lo), 0.5 * (hi - lo)
    mu, kT = 0.3 * lam[0] + 0.7 * lam[-1], 2.0
    n_pl = 40
    cols = chebyshev_columns(reg, chi_q, zeta_q, n_pl)
    c, _, _ = fd_coefficients(mu, kT, chi_q, zeta_q, n_pl, 2048)
    approx = sum(wp * cj * t.reshape(-1) for wp, cj, t in zip(primed(n_pl), c, cols))
    e = reg.unit().reshape(-1)
    exact = U @ (fermi((lam - mu) / kT) * (U.T @ e))
    c_long, _, _ = fd_coefficients(mu, kT, chi_q, zeta_q, 400, 4096)
    tail = np.abs(c_long[n_pl + 1:]).sum()
    assert np.abs(approx - exact).max() <= tail + 1e-13


# ---------------------------------------------------------------- P3: infinite-cell limit
def test_p3_sq_converges_to_k_integrated_dense_result():
    """Infinite-cell SQ -> infinite crystal (k-integrated dense diagonalisation, stored by
    tests/golden/make_golden.py from the oracle only) as R_cut and n_pl grow."""
    with open(os.path.join(GOLDEN, "p3_dense_k.json")) as f:
        ref = json.load(f)
    case = dict(ref["case"])
    bounds = lanczos_bounds(Problem(tiny_instance(**{**case, "r_cut": 4.5})))
    errs = []
    for rc, npl in ((1.8, 20), (2.7, 30), (4.5, 50)):
        o = run(tiny_instance(**{**case, "r_cut": rc, "n_pl": npl}), bounds=bounds)
        errs.append(max(abs(o["mu"] - ref["mu"]), abs(o["E_band"] - ref["E_band"]), abs(o["E_s"] - ref["E_s"]),
                        abs(o["E_nl"] - ref["E_nl"]), np.abs(o["rho"] - np.array(ref["rho"])).max(),
                        np.abs(o["sigma"] - np.array(ref["sigma"])).max()))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-8


# ---------------------------------------------------------------- P4: free electrons
def test_p4_free_electron_bz_closed_form_and_separable_region():
    """V = 0, no projectors: SQ density and kinetic stress == Brillouin-zone integrals
    (paper form uses G(theta)^2 of the first-derivative symbol), and the truncated region ==
    the exactly separable Kronecker-sum result."""
    h = 1.0
    inst = tiny_instance(seed=5, n=(3, 3, 3), h=(h, h, h), n_atoms=0, n_o=2, kT=3.17, r_cut=6.0,
                         n_pl=40, proj=[], vdepth=0.0, n_e=10.0)
    inst["proj"] = [[]]
    prob = Problem(inst)
    lo, hi = -0.05, 8.2
    mom = node_moments(prob, np.array([0, 0, 0]), lo, hi)
    mom_all = np.repeat(mom[None], prob.Nd, axis=0)     # translation invariance
    mu = fermi_bisect(mom_all[:, :, 0].sum(0), prob.n_e, prob.kT, lo, hi, prob.M)
    out = contract(prob, mom_all, mu, lo, hi)
    bz = free_electron.bz_values(mu, prob.kT, prob.h, prob.n_o)
    assert abs(out["rho"][0] - bz["rho"]) < 1e-9
    np.testing.assert_allclose(np.diag(out["sigma"]), bz["sigma_paper_diag"], atol=1e-9)
    assert np.abs(out["sigma"] - np.diag(np.diag(out["sigma"]))).max() < 1e-13
    assert abs(out["E_band"] / prob.vol - bz["E_band_density"]) < 1e-9
    assert abs(out["E_s"] / prob.vol - bz["E_s_density"]) < 1e-9
    # truncated region, exact by separability, against the same Chebyshev sums
    diag, kin = free_electron.separable_region(lambda e: fermi((e - mu) / prob.kT), prob.h, prob.n_o, prob.m)
    c, _, _ = fd_coefficients(mu, prob.kT, 0.5 * (hi + lo), 0.5 * (hi - lo), prob.n_pl, prob.M)
    cw = primed(prob.n_pl) * c
    assert abs(cw @ mom[:, 0] - diag) < 1e-12
    np.testing.assert_allclose([cw @ mom[:, 1], cw @ mom[:, 2], cw @ mom[:, 3]], kin, atol=1e-11)


# ---------------------------------------------------------------- P5: strain derivative
def _p5_problem(n=4, n_o=2):
    L = 3.6
    return Problem(tiny_instance(seed=1, n=(n, n, n), h=(L / n,) * 3, n_o=n_o, kT=3.17, n_e=2,
                                 pos=np.array([[0.7, 1.3, 2.2], [2.5, 2.9, 0.4]]),
                                 proj=[{"l": 0, "width": 0.8, "gamma": 1.0, "rcut": 8.0},
                                       {"l": 1, "width": 0.8, "gamma": 0.5, "rcut": 8.0}]))


def test_p5_strain_finite_difference_equals_density_matrix_stress():
    """(1/|Omega|) dF/dF_ab of the Mermin free energy under homogeneous strain (Eq.
    stressdefinition) == 2 tr(D dH/dF_ab)/|Omega| of the same grid Hamiltonian."""
    prob = _p5_problem()
    obs = dense_k.observables(prob, nk=2)
    scale = np.abs(obs["sigma_strain"]).max()
    for (a, b) in ((0, 0), (0, 1), (2, 1)):
        fd = dense_k.strain_fd_stress(prob, a, b, nk=2)
        assert abs(fd - obs["sigma_strain"][a, b]) < 1e-7 * scale


def test_p5_paper_nonlocal_stress_converges_to_strain_form():
    """The paper's discrete sigma^III (summation by parts, (X_b - R_b) grad_a) differs from the
    strain-consistent form only by discretisation error, which shrinks with h."""
    diffs = []
    for n in (4, 6, 8):
        obs = dense_k.observables(_p5_problem(n=n, n_o=4), nk=2)
        diffs.append(np.abs(obs["sigma_III"] - obs["sigma_III_strain"]).max())
    assert diffs[0] > diffs[1] > diffs[2]
    assert diffs[2] < 0.02 * diffs[0]


# ---------------------------------------------------------------- P6-P9 on a small cell
@pytest.fixture(scope="module")
def small_run():
    inst = tiny_instance(seed=11, n=(5, 5, 5), h=(0.8, 0.8, 0.8), n_atoms=3, n_o=3, r_cut=2.4, n_pl=24)
    prob = Problem(inst)
    bounds = lanczos_bounds(prob)
    return inst, bounds, run(inst, bounds=bounds)


def test_p6_electron_count(small_run):
    inst, _, out = small_run
    assert abs(out["N_check"] - inst["n_e"]) < 1e-12 * inst["n_e"]


def _rotate_z(inst):
    """90 degree rotation about z through the origin: (x, y, z) -> (-y, x, z) on a cubic grid."""
    n = int(inst["n"][0])
    L = float(inst["L"][0])
    v = np.asarray(inst["v_eff"]).reshape(n, n, n)          # [iz, iy, ix]
    vr = np.empty_like(v)
    for iy in range(n):
        for ix in range(n):
            vr[:, ix, (-iy) % n] = v[:, iy, ix]
    out = dict(inst)
    out["v_eff"] = vr.reshape(-1)
    p = np.asarray(inst["pos"])
    out["pos"] = np.mod(np.stack([-p[:, 1], p[:, 0], p[:, 2]], axis=1), L)
    return out


def test_p7_rotation_translation_permutation(small_run):
    inst, bounds, out = small_run
    Q = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    rot = run(_rotate_z(inst), bounds=bounds)
    np.testing.assert_allclose(rot["sigma"], Q @ out["sigma"] @ Q.T, atol=1e-12)
    assert rot["E_band"] == pytest.approx(out["E_band"], abs=1e-11)
    # translation by one grid vector along y
    n = int(inst["n"][0])
    tr = dict(inst)
    tr["v_eff"] = np.roll(np.asarray(inst["v_eff"]).reshape(n, n, n), 1, axis=1).reshape(-1)
    tr["pos"] = np.asarray(inst["pos"]) + np.array([0.0, float(inst["L"][1]) / n, 0.0])
    o2 = run(tr, bounds=bounds)
    np.testing.assert_allclose(o2["sigma"], out["sigma"], atol=1e-12)
    np.testing.assert_allclose(np.roll(out["rho"].reshape(n, n, n), 1, axis=1).reshape(-1), o2["rho"], atol=1e-12)
    # atom permutation
    pm = dict(inst)
    pm["pos"] = np.asarray(inst["pos"])[::-1].copy()
    o3 = run(pm, bounds=bounds)
    np.testing.assert_allclose(o3["sigma"], out["sigma"], atol=1e-13)
    # grid asymmetry of sigma^III is small (the continuum form is symmetric)
    s3 = out["sigma_III"]
    assert np.abs(s3 - s3.T).max() < 0.05 * np.abs(s3).max() + 1e-12


def test_p8_moment_identity(small_run):
    """-1/2 sum_a [D2_a t^j]_q / h_a^2 = w^T H t^j - V_q rho^j - N^j with
    w^T H t^j = chi rho^j + zeta (rho^{j+1} + rho^{j-1}) / 2 (Chebyshev identity)."""
    inst, (lo, hi), _ = small_run
    prob = Problem(inst)
    chi_q, zeta_q = 0.5 * (hi + lo), 0.5 * (hi - lo)
    q = np.array([2, 1, 3])
    mom, L2 = node_moments(prob, q, lo, hi, with_d2=True)
    Vq = prob.v[q[2], q[1], q[0]]
    rho = mom[:, 0]
    for j in range(0, prob.n_pl):
        wHt = chi_q * rho[j] + zeta_q * (rho[j + 1] + (rho[j - 1] if j > 0 else rho[1])) / 2.0
        lhs = -0.5 * L2[j].sum()
        assert abs(lhs - (wHt - Vq * rho[j] - mom[j, 7])) < 1e-10 * (1 + abs(lhs))


def test_p9_no_projectors_gives_zero_nonlocal_stress(small_run):
    inst, bounds, _ = small_run
    z = dict(inst)
    z["proj"] = [[{"l": 0, "width": 0.5, "gamma": 0.0, "rcut": 3.5}]]
    o = run(z, bounds=bounds)
    assert abs(o["E_nl"]) < 1e-15
    assert np.abs(o["sigma_III"]).max() < 1e-15


def test_lanczos_bounds_contain_region_spectra():
    inst = tiny_instance(seed=2, n=(4, 4, 4), h=(0.8, 0.8, 0.8), n_atoms=2, n_o=2, r_cut=1.6, n_pl=10)
    prob = Problem(inst)
    lo, hi = lanczos_bounds(prob)
    for idx in range(prob.Nd):
        lam = np.linalg.eigvalsh(NodeRegion(prob, prob.node_coords(idx)).dense_H())
        assert lo <= lam[0] and lam[-1] <= hi


def test_config1_instance_shape():
    inst = make_instance(1)
    prob = Problem(inst)
    assert list(prob.m) == [6, 6, 6] and prob.Nc == 13 ** 3 and prob.Nd == 1728
    assert Problem(make_instance(2)).Nc == 27 ** 3


# ---------------------------------------------------------------- P10: App. A pressure
def test_p10_pressure_free_electrons_is_grand_potential_volume_derivative():
    """V = 0, no projectors: the App. A pressure (kinetic part 2 E_kin / (3 |Omega|)) equals
    -d(Omega_grand)/d|Omega| at fixed mu under isotropic scaling of the grid, from the
    Brillouin-zone closed forms: P = -(omega + (h/3) d omega/dh), omega = e + e_s - mu rho."""
    h = 1.0
    inst = tiny_instance(seed=5, n=(3, 3, 3), h=(h, h, h), n_atoms=0, n_o=2, kT=3.17, r_cut=6.0,
                         n_pl=40, proj=[], vdepth=0.0, n_e=10.0)
    inst["proj"] = [[]]
    prob = Problem(inst)
    lo, hi = -0.05, 8.2
    mom = node_moments(prob, np.array([0, 0, 0]), lo, hi)
    mom_all = np.repeat(mom[None], prob.Nd, axis=0)
    mu = fermi_bisect(mom_all[:, :, 0].sum(0), prob.n_e, prob.kT, lo, hi, prob.M)
    out = contract(prob, mom_all, mu, lo, hi)

    def omega(hh):
        b = free_electron.bz_values(mu, prob.kT, (hh, hh, hh), prob.n_o)
        return b["E_band_density"] + b["E_s_density"] - mu * b["rho"]

    def dcentral(dh):
        return (omega(h + dh) - omega(h - dh)) / (2.0 * dh)

    dh = 1e-3 * h
    domega = (4.0 * dcentral(dh / 2) - dcentral(dh)) / 3.0      # Richardson: O(dh^4)
    p_bz = -(omega(h) + h / 3.0 * domega)
    assert abs(out["pressure_A"] - p_bz) < 1e-9 * abs(p_bz)
    # a dropped 2/3 (or a sign) in the kinetic part would miss by O(1)
    assert abs(out["pressure_A"] - out["E_band"] / prob.vol) > 0.1 * abs(p_bz)
    assert abs(out["E_pot"]) == 0.0


def test_p10_pressure_equals_trace_stress_with_second_difference_kinetic_term():
    """With nonlocal projectors and a potential: the App. A pressure equals -tr(sigma)/3 when
    the kinetic moments grad_a grad_a are replaced by the second-difference stencil D2_a (the
    operator in H), up to the Chebyshev truncation of the band-energy form (reading: the
    V_eff part of tr(DH) is left to the terms outside this path). The truncation part
    vanishes as n_pl grows; the paper-form trace differs by the restricted-gradient kinetic
    moments (m < 2 n_o here)."""
    diffs = []
    for n_pl in (12, 24):
        inst = tiny_instance(seed=11, n=(4, 4, 4), h=(0.8, 0.8, 0.8), n_atoms=3, n_o=3, r_cut=2.4, n_pl=n_pl)
        prob = Problem(inst)
        lo, hi = lanczos_bounds(prob)
        moms, l2s = [], []
        for q in range(prob.Nd):
            m, l2 = node_moments(prob, np.array([q % 4, (q // 4) % 4, q // 16]), lo, hi, with_d2=True)
            moms.append(m)
            l2s.append(l2)
        mom, l2 = np.array(moms), np.array(l2s)
        mu = fermi_bisect(mom[:, :, 0].sum(0), prob.n_e, prob.kT, lo, hi, prob.M)
        out = contract(prob, mom, mu, lo, hi)
        c, _, _ = fd_coefficients(mu, prob.kT, 0.5 * (hi + lo), 0.5 * (hi - lo), prob.n_pl, prob.M)
        cw = primed(prob.n_pl) * c
        sig_d2 = out["sigma"].copy() * prob.vol
        for a in range(3):
            sig_d2[a, a] += 2.0 * float(np.sum(l2[:, :, a] @ cw)) - 2.0 * float(np.sum(mom[:, :, 1 + a] @ cw))
        p_trace = -float(np.trace(sig_d2)) / (3.0 * prob.vol)
        diffs.append(abs(out["pressure_A"] - p_trace))
    assert diffs[1] < 1e-12 * abs(out["pressure_A"])
    assert diffs[0] > diffs[1]


# ---------------------------------------------------------------- P11: Green-Kubo viscosity
def _sigma_series(s12):
    """(n_traj, n_steps, 3, 3) stress tensors with only sigma_12 = sigma_21 non-zero."""
    sig = np.zeros(s12.shape + (3, 3))
    sig[..., 0, 1] = s12
    sig[..., 1, 0] = s12
    return sig


def test_p11_green_kubo_cosine_closed_form():
    """s_12(t) = A cos(w t): the origin-averaged autocorrelation has the closed form
    (A^2/5) [cos(w k)/2 + sin(w K) cos(w (k + K - 1)) / (2 K sin w)], K = n - k origins
    (product-to-sum and the geometric sum of cosines); eta is |Omega|/kT times its trapezoid."""
    n, A, w, dt, vol, kT = 400, 0.03, 0.173, 2.5, 1728.0, 3.17
    t = np.arange(n)
    sig = _sigma_series((A * np.cos(w * t))[None, :])
    eta, c = green_kubo.viscosity(sig, dt, vol, kT, 60)
    k = np.arange(61)
    K = n - k
    closed = A * A / 5.0 * (0.5 * np.cos(w * k) + np.sin(w * K) * np.cos(w * (k + K - 1)) / (2.0 * K * np.sin(w)))
    np.testing.assert_allclose(c, closed, rtol=0, atol=1e-15)
    trap = np.concatenate([[0.0], np.cumsum(0.5 * dt * (closed[:-1] + closed[1:]))])
    np.testing.assert_allclose(eta, vol / kT * trap, rtol=1e-12, atol=0)


def test_p11_green_kubo_deviatoric_invariance_and_component_weights():
    """An isotropic pressure p(t) I added to sigma leaves the viscosity unchanged (only the
    traceless part enters); sigma_11 = -sigma_22 = x(t) enters through (s_11 - s_22)/2 and
    (s_22 - s_33)/2 with weights 1 and 1/4 of x, against 1 for x in sigma_12."""
    rng = np.random.Generator(np.random.PCG64(11))
    sig = rng.normal(size=(2, 300, 3, 3)) * 0.01
    sig = 0.5 * (sig + np.swapaxes(sig, -1, -2))
    eta0, _ = green_kubo.viscosity(sig, 1.0, 1000.0, 2.0, 40)
    p = rng.normal(size=(2, 300)) * 5.0
    eta1, _ = green_kubo.viscosity(sig + p[..., None, None] * np.eye(3), 1.0, 1000.0, 2.0, 40)
    np.testing.assert_allclose(eta1, eta0, rtol=1e-9, atol=1e-12)
    x = rng.normal(size=(1, 500))
    s_shear = _sigma_series(x)
    s_normal = np.zeros_like(s_shear)
    s_normal[..., 0, 0] = x
    s_normal[..., 1, 1] = -x
    c_shear = green_kubo.stress_acf(s_shear, 5)
    c_normal = green_kubo.stress_acf(s_normal, 5)
    np.testing.assert_allclose(c_normal, c_shear * (1.0 + 0.25), rtol=1e-12)


def test_p11_green_kubo_exponential_correlation():
    """An Ornstein-Uhlenbeck sigma_12 with unit variance and correlation time tau (steps):
    C(k) -> exp(-k / tau) / 5 and eta(inf) -> (|Omega|/kT) dt (1/5) (1 + e^{-1/tau}) / (2 (1 - e^{-1/tau}))
    (the trapezoid sum of the exponential), within the statistical error of 4 x 200k steps."""
    tau, n, ntr = 8.0, 200_000, 4
    a = math.exp(-1.0 / tau)
    rng = np.random.Generator(np.random.PCG64(5))
    x = np.empty((ntr, n))
    x[:, 0] = rng.normal(size=ntr)
    noise = rng.normal(size=(ntr, n)) * math.sqrt(1.0 - a * a)
    for i in range(1, n):
        x[:, i] = a * x[:, i - 1] + noise[:, i]
    dt, vol, kT = 0.5, 100.0, 1.0
    eta, c = green_kubo.viscosity(_sigma_series(x), dt, vol, kT, 80)
    np.testing.assert_allclose(c[:4], np.exp(-np.arange(4) / tau) / 5.0, atol=0.01)
    expect = vol / kT * dt / 5.0 * 0.5 * (1.0 + a) / (1.0 - a)
    assert abs(eta[-1] - expect) < 0.1 * expect


# ---------------------------------------------------------------- P12: per-node spectral bounds
@pytest.fixture(scope="module")
def per_node_case():
    inst = tiny_instance(seed=11, n=(4, 4, 4), h=(0.8, 0.8, 0.8), n_atoms=3, n_o=3, r_cut=2.4, n_pl=24)
    return inst, per_node.run(inst)


def test_p12_per_node_intervals_contain_each_spectrum(per_node_case):
    """Each node's interval (Lanczos extremes with residual widening, then 1 %) contains the
    whole spectrum of its H_q, from a dense symmetric eigensolver of the Kronecker-assembled
    matrix; and it is no wider than needed by more than the 1 % margins plus the residuals."""
    inst, out = per_node_case
    prob = Problem(inst)
    for q in (0, 21, 42, 63):
        ev = np.linalg.eigvalsh(NodeRegion(prob, prob.node_coords(q)).dense_H())
        lo, hi = out["bounds"][q]
        assert lo <= ev[0] and ev[-1] <= hi
        assert (hi - lo) <= 1.05 * (ev[-1] - ev[0])


def test_p12_per_node_mode_reduces_to_shared_mode(per_node_case):
    """Per-node code with every node given the shared interval reproduces the shared mode
    exactly (moments, Fermi level, contraction); with its own intervals it converges to the
    same density matrix (n_pl = 24 here: free energy and stress agree to 1e-12)."""
    inst, out = per_node_case
    prob = Problem(inst)
    gb = lanczos_bounds(prob)
    ref = run(inst, bounds=gb)
    B = np.tile(np.array(gb), (prob.Nd, 1))
    mom = per_node.moments(prob, B)
    mu = per_node.fermi_bisect(prob, mom, B)
    same = per_node.contract(prob, mom, B, mu)
    assert mu == ref["mu"]
    assert abs(same["F"] - ref["F"]) <= 1e-14 * abs(ref["F"])
    np.testing.assert_allclose(same["sigma"], ref["sigma"], rtol=0, atol=1e-15)
    assert abs(out["F"] - ref["F"]) <= 1e-12 * abs(ref["F"])
    np.testing.assert_allclose(out["sigma"], ref["sigma"], rtol=0, atol=1e-12)
    assert abs(out["N_check"] - inst["n_e"]) < 1e-10 * inst["n_e"]


# ---------------------------------------------------------------- P13: Gauss SQ density
def test_p13_gauss_quadrature_is_exact_to_degree_2k_minus_1():
    """k-point Gauss quadrature of e_q's spectral measure integrates lambda^p exactly for
    p <= 2k - 1: sum_i w_i theta_i^p = e_q^T H_q^p e_q (repeated applications of the region
    operator), and not for p = 2k."""
    inst = tiny_instance(seed=11, n=(4, 4, 4), h=(0.8, 0.8, 0.8), n_atoms=3, n_o=3, r_cut=2.4, n_pl=12)
    prob = Problem(inst)
    region = NodeRegion(prob, prob.node_coords(21))
    k = 3
    theta, w = gauss_sq.node_quadrature(prob, 21, k)
    t = region.unit()
    e = t.copy()
    for p in range(0, 2 * k + 1):
        exact = float(np.sum(e * t))
        quad = float(np.sum(w * theta ** p))
        if p <= 2 * k - 1:
            assert abs(quad - exact) <= 1e-11 * max(1.0, abs(exact)), p
        else:
            assert abs(quad - exact) > 1e-6 * abs(exact)
        t = region.apply_H(t)


def test_p13_gauss_full_krylov_equals_dense_and_matches_clenshaw_curtis():
    """With k = the region dimension the quadrature is [g(H_q)]_qq from a dense eigensolver; on a
    4^3 cell the Gauss SQ density, electron count and band energy equal the Clenshaw-Curtis SQ
    ones once both have converged (k = n_pl = 40)."""
    inst = tiny_instance(seed=2, n=(4, 4, 4), h=(0.8, 0.8, 0.8), n_atoms=2, n_o=1, r_cut=0.9, n_pl=10)
    prob = Problem(inst)
    region = NodeRegion(prob, prob.node_coords(5))
    Hd = region.dense_H()
    ev, U = np.linalg.eigh(Hd)
    c = np.ravel_multi_index(region.center, region.shape)
    theta, w = gauss_sq.node_quadrature(prob, 5, Hd.shape[0])
    mu = 2.0
    dense = float(np.sum(U[c, :] ** 2 * fermi((ev - mu) / prob.kT)))
    assert abs(float(np.sum(w * fermi((theta - mu) / prob.kT))) - dense) <= 1e-12
    inst = tiny_instance(seed=11, n=(4, 4, 4), h=(0.8, 0.8, 0.8), n_atoms=3, n_o=3, r_cut=2.4, n_pl=40)
    g = gauss_sq.run(inst, k=40)
    cc = run(inst, bounds=lanczos_bounds(Problem(inst)))
    assert abs(g["mu"] - cc["mu"]) <= 1e-11 * abs(cc["mu"])
    assert np.abs(g["rho"] - cc["rho"]).max() <= 1e-11 * np.abs(cc["rho"]).max()
    assert abs(g["E_band"] - cc["E_band"]) <= 1e-11 * abs(cc["E_band"])
    assert abs(g["N_check"] - inst["n_e"]) <= 1e-11 * inst["n_e"]


def test_p11_green_kubo_autocorrelation_equals_wiener_khinchin():
    """The origin-averaged autocorrelation equals the Wiener-Khinchin form computed by FFT with
    zero padding (inverse transform of the power spectrum, divided by the origin count) - an
    independent route to the same estimator."""
    rng = np.random.Generator(np.random.PCG64(21))
    sig = rng.normal(size=(3, 700, 3, 3))
    sig = 0.5 * (sig + np.swapaxes(sig, -1, -2))
    max_lag = 90
    c = green_kubo.stress_acf(sig, max_lag)
    s = green_kubo.deviatoric_components(sig)                # (n_traj, n, 5)
    n = s.shape[1]
    spec = np.fft.rfft(s, n=2 * n, axis=1)
    raw = np.fft.irfft(spec * np.conj(spec), n=2 * n, axis=1)[:, : max_lag + 1, :]   # sum over origins
    wk = raw.sum(axis=(0, 2)) / (5.0 * s.shape[0] * (n - np.arange(max_lag + 1)))
    np.testing.assert_allclose(c, wk, rtol=1e-10, atol=1e-13)


def test_p13_gauss_plain_lanczos_matches_reorthogonalised():
    """The plain three-term Lanczos recurrence (no reorthogonalisation) gives the same Gauss
    rule to rounding: exact to degree 2k - 1 at small k and the same density, Fermi level and
    band energy as the reorthogonalised run once converged (k = 40)."""
    inst = tiny_instance(seed=11, n=(4, 4, 4), h=(0.8, 0.8, 0.8), n_atoms=3, n_o=3, r_cut=2.4, n_pl=40)
    prob = Problem(inst)
    theta, w = gauss_sq.node_quadrature(prob, 21, 3, reorth=False)
    region = NodeRegion(prob, prob.node_coords(21))
    t = region.unit()
    e = t.copy()
    for p in range(0, 6):
        exact = float(np.sum(e * t))
        assert abs(float(np.sum(w * theta ** p)) - exact) <= 1e-11 * max(1.0, abs(exact)), p
        t = region.apply_H(t)
    a = gauss_sq.run(inst, k=40)
    b = gauss_sq.run(inst, k=40, reorth=False)
    assert abs(a["mu"] - b["mu"]) <= 1e-12 * abs(a["mu"])
    assert np.abs(a["rho"] - b["rho"]).max() <= 1e-12 * np.abs(a["rho"]).max()
    assert abs(a["E_band"] - b["E_band"]) <= 1e-12 * abs(a["E_band"])
