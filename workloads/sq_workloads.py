"""Synthetic hot-hydrogen-like instances for the SQ stress sweep.

An *instance* is a plain dict (the same keys the C-ABI descriptor carries):

  L        (3,) float   orthorhombic cell sides (bohr)
  n        (3,) int     grid nodes per side; h_a = L_a / n_a, node i sits at i*h
  n_o      int          finite-difference half order (stencil reach)
  v_eff    (N_d,) f64   effective potential on the nodes, x fastest:
                        i = ix + n0*(iy + n1*iz)
  pos      (N_a, 3)     atom positions (bohr)
  species  (N_a,) int   species index of each atom
  proj     list         per species, a list of Kleinman-Bylander projector
                        specs {"l": 0|1, "width": w, "gamma": g, "rcut": rc}
  kT, n_e, r_cut, n_pl  smearing (Ha), electron count, truncation radius
                        (bohr), Chebyshev degree
  M        int          Chebyshev-Gauss points used for the coefficients

The paper's workload is hydrogen at 10^6 K (kT = 3.17 Ha); its pseudopotential
is not available, so V_eff is a periodic sum of Gaussian wells centred on the
atoms and the projectors are Gaussian s / p functions. Seeds follow
seed = 1000 * config + instance (NumPy PCG64).
"""
from __future__ import annotations

import math

import numpy as np

KT_1E6_K = 3.17          # k_B * 10^6 K in Ha (3.1668), rounded as the configs state
DENSITY_BATCH = 0.0375   # atoms / bohr^3 for the batched / served snapshots


def _rng(config: int, instance: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(1000 * config + instance))


def random_positions(rng: np.random.Generator, n_atoms: int, L, min_sep: float = 0.0,
                     max_tries: int = 200000) -> np.ndarray:
    """Uniform positions in the cell; with min_sep > 0, random sequential addition
    under the periodic minimum-image distance."""
    L = np.asarray(L, dtype=np.float64)
    if min_sep <= 0.0:
        return rng.uniform(0.0, 1.0, size=(n_atoms, 3)) * L
    out = np.zeros((0, 3))
    tries = 0
    while out.shape[0] < n_atoms:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("random sequential addition did not place all atoms")
        x = rng.uniform(0.0, 1.0, size=3) * L
        if out.shape[0]:
            d = out - x
            d -= L * np.round(d / L)
            if np.min(np.einsum("ij,ij->i", d, d)) < min_sep * min_sep:
                continue
        out = np.vstack([out, x])
    return out


def perturb_positions(rng: np.random.Generator, pos: np.ndarray, sigma: float, L) -> np.ndarray:
    """One trajectory step of a served snapshot stream: Gaussian displacements,
    wrapped back into the cell."""
    L = np.asarray(L, dtype=np.float64)
    return np.mod(pos + rng.normal(0.0, sigma, size=pos.shape), L)


def gaussian_veff(L, n, pos, depth: float = -2.0, width: float = 0.6,
                  tol: float = 1e-20) -> np.ndarray:
    """V_eff(x) = sum over atoms and their periodic images of depth*exp(-r^2/(2 w^2)),
    sampled at the nodes i*h; images are summed while the term exceeds tol*|depth|."""
    L = np.asarray(L, dtype=np.float64)
    n = np.asarray(n, dtype=np.int64)
    h = L / n
    rmax = width * math.sqrt(2.0 * math.log(1.0 / tol))
    axes = [np.arange(n[a]) * h[a] for a in range(3)]
    v = np.zeros((n[2], n[1], n[0]))
    inv2w2 = 1.0 / (2.0 * width * width)
    for R in np.asarray(pos, dtype=np.float64).reshape(-1, 3):
        # per-axis Gaussian factors summed over images (the Gaussian is separable)
        fac = []
        for a in range(3):
            s_lo = int(math.floor((-rmax - R[a]) / L[a])) - 1
            s_hi = int(math.ceil((L[a] + rmax - R[a]) / L[a])) + 1
            f = np.zeros(n[a])
            for s in range(s_lo, s_hi + 1):
                d = axes[a] - (R[a] + s * L[a])
                f += np.exp(-d * d * inv2w2)
            fac.append(f)
        v += depth * fac[2][:, None, None] * fac[1][None, :, None] * fac[0][None, None, :]
    return v.reshape(-1).copy()


def _instance(name, L, n, n_o, pos, proj, kT, n_e, r_cut, n_pl, vdepth=-2.0, vwidth=0.6,
              M=2048):
    L = np.asarray(L, dtype=np.float64).reshape(3)
    n = np.asarray(n, dtype=np.int64).reshape(3)
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    return {
        "name": name,
        "L": L,
        "n": n,
        "n_o": int(n_o),
        "v_eff": gaussian_veff(L, n, pos, vdepth, vwidth) if vdepth != 0.0
        else np.zeros(int(np.prod(n))),
        "pos": pos,
        "species": np.zeros(pos.shape[0], dtype=np.int64),
        "proj": [list(proj)],
        "kT": float(kT),
        "n_e": float(n_e),
        "r_cut": float(r_cut),
        "n_pl": int(n_pl),
        "M": int(M),
    }


def s_proj(width=0.5, gamma=1.0):
    return {"l": 0, "width": width, "gamma": gamma, "rcut": 7.0 * width}


def p_proj(width=0.5, gamma=0.5):
    return {"l": 1, "width": width, "gamma": gamma, "rcut": 7.0 * width}


CONFIGS = {
    1: "8 H, cube 6 bohr, h=0.5 (12^3), n_o=3, s projectors, kT=3.17, R_cut=3 (13^3), n_pl=30",
    2: "64 H, cube 12 bohr, h=0.3 (40^3), n_o=6, s+p projectors, kT=3.17, R_cut=4 (27^3), n_pl=60",
    3: "216 H, cube 18 bohr, h=0.3 (60^3), n_o=6, s+p projectors, kT=3.17, R_cut=4, n_pl=60",
}


def make_instance(config: int, instance: int = 0) -> dict:
    """The single-instance workloads (configs 1-3)."""
    rng = _rng(config, instance)
    if config == 1:
        pos = random_positions(rng, 8, [6.0] * 3)
        return _instance("c1_8H_12cube", [6.0] * 3, [12] * 3, 3, pos, [s_proj(0.5, 1.0)],
                         KT_1E6_K, 8, 3.0, 30)
    if config == 2:
        pos = random_positions(rng, 64, [12.0] * 3)
        return _instance("c2_64H_40cube", [12.0] * 3, [40] * 3, 6, pos,
                         [s_proj(0.5, 1.0), p_proj(0.5, 0.5)], KT_1E6_K, 64, 4.0, 60)
    if config == 3:
        pos = random_positions(rng, 216, [18.0] * 3)
        return _instance("c3_216H_60cube", [18.0] * 3, [60] * 3, 6, pos,
                         [s_proj(0.5, 1.0), p_proj(0.5, 0.5)], KT_1E6_K, 216, 4.0, 60)
    raise ValueError(f"no single-instance config {config}")


def make_profile_case(instance: int = 0) -> dict:
    """The 40^3 / 64 H workload's parameters (h = 0.3, n_o = 6, s+p, R_cut = 4, kT, atom
    density 0.037 / bohr^3) on a 16^3-node cell with 4 atoms and n_pl = 4: the same per-tile
    work in a case small enough (about 2.5 GB on the device) for a profiler capture."""
    rng = _rng(9, instance)
    pos = random_positions(rng, 4, [4.8] * 3)
    return _instance("profile_4H_16cube", [4.8] * 3, [16] * 3, 6, pos,
                     [s_proj(0.5, 1.0), p_proj(0.5, 0.5)], KT_1E6_K, 4, 4.0, 4)


def make_batch(config: int = 4, count: int = 32, h: float = 0.3, start: int = 0,
               atom_choices=(32, 64, 128, 256, 512), p_large: float | None = None) -> list:
    """Uneven quantum-MD-like snapshots: atom count from atom_choices (or 512 with
    probability p_large), cubic side L = (N/0.0375)^(1/3) snapped to n = round(L/h),
    0.8 bohr minimum separation, kT ~ U[1.6, 6.3], n_pl ~ U{30..80}, R_cut ~ U[3, 5]."""
    out = []
    for i in range(start, start + count):
        rng = _rng(config, i)
        if p_large is not None and rng.uniform() < p_large:
            na = 512
        else:
            na = int(rng.choice(np.asarray(atom_choices)))
        n = int(round((na / DENSITY_BATCH) ** (1.0 / 3.0) / h))
        L = n * h
        kT = float(rng.uniform(1.6, 6.3))
        n_pl = int(rng.integers(30, 81))
        r_cut = float(rng.uniform(3.0, 5.0))
        pos = random_positions(rng, na, [L] * 3, min_sep=0.8)
        out.append(_instance(f"c{config}_{i}_{na}H_{n}cube", [L] * 3, [n] * 3, 6, pos,
                             [s_proj(0.5, 1.0), p_proj(0.5, 0.5)], kT, na, r_cut, n_pl))
    return out


def tiny_instance(seed: int = 0, n=(6, 6, 6), h=(0.8, 0.8, 0.8), n_atoms: int = 2, n_o: int = 2,
                  kT: float = KT_1E6_K, r_cut: float = 2.4, n_pl: int = 20, n_e=None,
                  proj=None, vdepth: float = -2.0, vwidth: float = 0.6, M: int = 2048,
                  pos=None) -> dict:
    """Small periodic cells for pins and parity tests (sizes the oracle finishes in
    seconds); everything is a keyword so tests can sweep one knob at a time."""
    rng = np.random.Generator(np.random.PCG64(777000 + seed))
    n = np.asarray(n, dtype=np.int64)
    L = n * np.asarray(h, dtype=np.float64)
    if pos is None:
        pos = random_positions(rng, n_atoms, L)
    if proj is None:
        proj = [s_proj(0.5, 1.0), p_proj(0.5, 0.5)]
    if n_e is None:
        n_e = float(max(1, len(pos)))
    return _instance(f"tiny{seed}", L, n, n_o, pos, proj, kT, n_e, r_cut, n_pl,
                     vdepth=vdepth, vwidth=vwidth, M=M)
