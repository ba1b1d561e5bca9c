"""Thin ctypes binding of the C ABI in include/sq_api.h (argument marshalling only).

Every function keeps the C name and returns what the C call writes; a non-zero status
raises SQError with the library's error text. The CUDA library must have been built
(paper_2006_03697_gb300.build); there is no fallback of any kind.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

LIB_PATH = Path(__file__).resolve().parent / "_lib" / "libsq_gb300.so"

SQ_OK = 0
SQ_ERR_INVALID_ARG = 1
SQ_ERR_OOM = 2
SQ_ERR_CUDA = 3
SQ_ERR_NO_BRACKET = 4
SQ_ERR_TIMEOUT = 5
SQ_ERR_STATE = 6
SQ_FP64 = 0
SQ_MIXED = 1
SQ_BOUNDS_LANCZOS = 0
SQ_BOUNDS_GIVEN = 1
SQ_BOUNDS_PER_NODE = 2
SQ_N_MOMENTS = 17

EXPORTED = [
    "sq_setup", "sq_moments", "sq_fermi_level", "sq_node_sums", "sq_fermi_level_sums",
    "sq_density_energy_stress",
    "sq_density_energy_stress_dev", "sq_pressure", "sq_get_bounds", "sq_node_bounds", "sq_moments_copy", "sq_footprint_bytes",
    "sq_kernel_launches", "sq_keep_lists", "sq_step_launch_counts", "sq_tune_step", "sq_kernel_timing", "sq_kernel_timing_read", "sq_fermi_level_noalloc", "sq_batch_evaluate",
    "sq_batch_create", "sq_batch_set_chains", "sq_batch_run", "sq_batch_last_error", "sq_batch_destroy", "sq_server_create", "sq_server_submit", "sq_server_submit_traj", "sq_server_resident",
    "sq_update_atoms",
    "sq_server_poll", "sq_server_pending", "sq_server_destroy", "sq_gauss_density", "sq_green_kubo", "sq_destroy",
    "sq_last_error",
]
SQ_K_STENCIL = 0
SQ_K_PROJECT = 1
SQ_K_MOMENTS = 2


class sq_proj(C.Structure):
    _fields_ = [("l", C.c_int), ("width", C.c_double), ("gamma", C.c_double), ("rcut", C.c_double)]


class sq_instance_desc(C.Structure):
    _fields_ = [
        ("L", C.c_double * 3), ("n", C.c_int * 3), ("n_o", C.c_int),
        ("v_eff", C.POINTER(C.c_double)),
        ("n_atoms", C.c_int), ("pos", C.POINTER(C.c_double)), ("species", C.POINTER(C.c_int)),
        ("n_species", C.c_int), ("proj_offset", C.POINTER(C.c_int)), ("proj", C.POINTER(sq_proj)),
        ("kT", C.c_double), ("n_e", C.c_double), ("r_cut", C.c_double), ("n_pl", C.c_int),
        ("precision", C.c_int), ("bounds_mode", C.c_int),
        ("lambda_lo", C.c_double), ("lambda_hi", C.c_double),
        ("cheb_quad_M", C.c_int), ("lanczos_k", C.c_int), ("stream", C.c_void_p),
        ("part_rank", C.c_int), ("part_count", C.c_int),
    ]


class sq_energies(C.Structure):
    _fields_ = [("E_band", C.c_double), ("E_s", C.c_double), ("E_nl", C.c_double),
                ("F", C.c_double), ("N_check", C.c_double), ("mu", C.c_double)]


class sq_result(C.Structure):
    _fields_ = [("tag", C.c_longlong), ("status", C.c_int), ("mu", C.c_double), ("energies", sq_energies),
                ("sigma", C.c_double * 9), ("latency_ms", C.c_double), ("error", C.c_char * 128)]


class SQError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


_lib = None


def lib():
    """Loads the in-tree CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2006_03697_gb300.build")
        L = C.CDLL(str(LIB_PATH))
        H = C.c_void_p
        L.sq_setup.argtypes = [C.POINTER(sq_instance_desc), C.POINTER(H)]
        L.sq_moments.argtypes = [H]
        L.sq_fermi_level.argtypes = [H, C.POINTER(C.c_double)]
        L.sq_node_sums.argtypes = [H, C.c_void_p]
        L.sq_node_sums.restype = C.c_int
        L.sq_fermi_level_sums.argtypes = [H, C.c_void_p, C.POINTER(C.c_double)]
        L.sq_fermi_level_sums.restype = C.c_int
        L.sq_density_energy_stress.argtypes = [H, C.c_double, C.c_void_p, C.POINTER(sq_energies), C.c_void_p]
        L.sq_density_energy_stress_dev.argtypes = [H, C.c_double, C.c_void_p, C.POINTER(sq_energies), C.c_void_p]
        L.sq_pressure.argtypes = [H, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.sq_get_bounds.argtypes = [H, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.sq_node_bounds.argtypes = [H, C.c_void_p, C.c_void_p]
        L.sq_node_bounds.restype = C.c_int
        L.sq_moments_copy.argtypes = [H, C.c_void_p]
        L.sq_footprint_bytes.argtypes = [C.POINTER(sq_instance_desc)]
        L.sq_footprint_bytes.restype = C.c_size_t
        L.sq_kernel_launches.argtypes = [H]
        L.sq_kernel_launches.restype = C.c_longlong
        L.sq_tune_step.argtypes = [H, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double)]
        L.sq_tune_step.restype = C.c_int
        L.sq_keep_lists.argtypes = [H, C.c_int]
        L.sq_keep_lists.restype = C.c_int
        L.sq_step_launch_counts.argtypes = [H, C.POINTER(C.c_longlong)]
        L.sq_step_launch_counts.restype = C.c_int
        L.sq_kernel_timing.argtypes = [H, C.c_int]
        L.sq_kernel_timing.restype = C.c_int
        L.sq_kernel_timing_read.argtypes = [H, C.c_int, C.POINTER(C.c_longlong), C.POINTER(C.c_double),
                                            C.POINTER(C.c_double)]
        L.sq_kernel_timing_read.restype = C.c_int
        L.sq_fermi_level_noalloc.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                             C.c_double, C.c_int, C.c_void_p, C.c_void_p]
        L.sq_fermi_level_noalloc.restype = C.c_int
        L.sq_batch_evaluate.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
        L.sq_batch_evaluate.restype = C.c_int
        L.sq_batch_create.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_void_p)]
        L.sq_batch_create.restype = C.c_int
        L.sq_batch_set_chains.argtypes = [C.c_void_p, C.c_int]
        L.sq_batch_set_chains.restype = C.c_int
        L.sq_batch_run.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.sq_batch_run.restype = C.c_int
        L.sq_batch_last_error.argtypes = [C.c_void_p]
        L.sq_batch_last_error.restype = C.c_char_p
        L.sq_batch_destroy.argtypes = [C.c_void_p]
        L.sq_batch_destroy.restype = None
        L.sq_server_create.argtypes = [C.c_size_t, C.c_int, C.POINTER(C.c_void_p)]
        L.sq_server_create.restype = C.c_int
        L.sq_server_submit.argtypes = [C.c_void_p, C.POINTER(sq_instance_desc), C.c_longlong]
        L.sq_server_submit.restype = C.c_int
        L.sq_server_submit_traj.argtypes = [C.c_void_p, C.POINTER(sq_instance_desc), C.c_longlong, C.c_longlong]
        L.sq_server_submit_traj.restype = C.c_int
        L.sq_server_resident.argtypes = [C.c_void_p]
        L.sq_server_resident.restype = C.c_int
        L.sq_update_atoms.argtypes = [H, C.c_void_p, C.c_void_p]
        L.sq_update_atoms.restype = C.c_int
        L.sq_server_poll.argtypes = [C.c_void_p, C.POINTER(sq_result), C.c_int, C.c_int, C.POINTER(C.c_int)]
        L.sq_server_poll.restype = C.c_int
        L.sq_server_pending.argtypes = [C.c_void_p]
        L.sq_server_pending.restype = C.c_int
        L.sq_server_destroy.argtypes = [C.c_void_p]
        L.sq_server_destroy.restype = None
        L.sq_gauss_density.argtypes = [H, C.c_int, C.POINTER(C.c_double), C.c_void_p, C.POINTER(C.c_double)]
        L.sq_gauss_density.restype = C.c_int
        L.sq_green_kubo.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_int,
                                    C.c_void_p, C.c_void_p, C.c_void_p]
        L.sq_green_kubo.restype = C.c_int
        L.sq_destroy.argtypes = [H]
        L.sq_destroy.restype = None
        L.sq_last_error.argtypes = [H]
        L.sq_last_error.restype = C.c_char_p
        for name in ("sq_setup", "sq_moments", "sq_fermi_level", "sq_density_energy_stress",
                     "sq_density_energy_stress_dev", "sq_pressure", "sq_get_bounds", "sq_node_bounds", "sq_moments_copy"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


class Desc:
    """Owns the host arrays a sq_instance_desc points to (built from a workloads dict)."""

    def __init__(self, inst: dict, precision=SQ_FP64, bounds=None, stream=None, lanczos_k=0, partition=None):
        self.v = np.ascontiguousarray(inst["v_eff"], dtype=np.float64)
        self.pos = np.ascontiguousarray(np.asarray(inst["pos"], dtype=np.float64).reshape(-1, 3))
        self.species = np.ascontiguousarray(inst["species"], dtype=np.int32)
        offs = [0]
        plist = []
        for sp in inst["proj"]:
            for pj in sp:
                plist.append(sq_proj(int(pj["l"]), float(pj["width"]), float(pj["gamma"]),
                                     float(pj.get("rcut", 0.0) or 0.0)))
            offs.append(len(plist))
        self.offs = np.ascontiguousarray(offs, dtype=np.int32)
        self.proj = (sq_proj * max(1, len(plist)))(*plist)
        d = sq_instance_desc()
        for a in range(3):
            d.L[a] = float(inst["L"][a])
            d.n[a] = int(inst["n"][a])
        d.n_o = int(inst["n_o"])
        d.v_eff = self.v.ctypes.data_as(C.POINTER(C.c_double))
        d.n_atoms = int(self.pos.shape[0])
        d.pos = self.pos.ctypes.data_as(C.POINTER(C.c_double))
        d.species = self.species.ctypes.data_as(C.POINTER(C.c_int))
        d.n_species = len(inst["proj"])
        d.proj_offset = self.offs.ctypes.data_as(C.POINTER(C.c_int))
        d.proj = C.cast(self.proj, C.POINTER(sq_proj))
        d.kT = float(inst["kT"])
        d.n_e = float(inst["n_e"])
        d.r_cut = float(inst["r_cut"])
        d.n_pl = int(inst["n_pl"])
        d.precision = int(precision)
        if bounds is None:
            d.bounds_mode = SQ_BOUNDS_LANCZOS
        elif isinstance(bounds, str):
            if bounds != "per_node":
                raise ValueError(f"unknown bounds mode {bounds!r}")
            d.bounds_mode = SQ_BOUNDS_PER_NODE
        else:
            d.bounds_mode = SQ_BOUNDS_GIVEN
            d.lambda_lo, d.lambda_hi = float(bounds[0]), float(bounds[1])
        d.cheb_quad_M = int(inst.get("M", 2048))
        d.lanczos_k = int(lanczos_k)
        d.stream = stream
        if partition is not None:
            d.part_rank, d.part_count = int(partition[0]), int(partition[1])
        self.c = d


def _check(rc, h=None):
    if rc != SQ_OK:
        msg = lib().sq_last_error(h).decode(errors="replace")
        raise SQError(rc, msg)


def sq_setup(desc: Desc):
    h = C.c_void_p()
    _check(lib().sq_setup(C.byref(desc.c), C.byref(h)), None)
    return h


def sq_moments(h):
    _check(lib().sq_moments(h), h)


def sq_fermi_level(h) -> float:
    mu = C.c_double()
    _check(lib().sq_fermi_level(h, C.byref(mu)), h)
    return mu.value


def sq_update_atoms(h, pos, v_eff):
    """New atom positions [n_atoms][3] and V_eff [N_d] for a live handle (same cell and species)."""
    pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, 3))
    v = np.ascontiguousarray(v_eff, dtype=np.float64)
    _check(lib().sq_update_atoms(h, pos.ctypes.data if pos.size else None, v.ctypes.data), h)


def sq_node_sums(h, n_pl: int) -> np.ndarray:
    """R^j = this handle's (or partition part's) node sums of rho_q^j, j = 0..n_pl."""
    R = np.zeros(n_pl + 1)
    _check(lib().sq_node_sums(h, R.ctypes.data), h)
    return R


def sq_fermi_level_sums(h, R) -> float:
    """Fermi level from whole-cell node sums R (e.g. the allreduce of every part's sq_node_sums)."""
    R = np.ascontiguousarray(R, dtype=np.float64)
    mu = C.c_double()
    _check(lib().sq_fermi_level_sums(h, R.ctypes.data, C.byref(mu)), h)
    return mu.value


def partition_tiles(n, rank: int, count: int, b: int = 2):
    """The tile range [begin, end) of part `rank` of `count` (the library's rule: equal
    contiguous ranges of the b x b x b-node tiles, t = tx + T0 (ty + T1 tz))."""
    tiles = [(int(x) + b - 1) // b for x in n]
    nt = tiles[0] * tiles[1] * tiles[2]
    return nt * rank // count, nt * (rank + 1) // count


def partition_nodes(n, rank: int, count: int, b: int = 2) -> np.ndarray:
    """Node indices (x fastest) that part `rank` of `count` sweeps."""
    n = [int(x) for x in n]
    tiles = [(x + b - 1) // b for x in n]
    t0, t1 = partition_tiles(n, rank, count, b)
    out = []
    for t in range(t0, t1):
        ox, oy, oz = (t % tiles[0]) * b, ((t // tiles[0]) % tiles[1]) * b, (t // (tiles[0] * tiles[1])) * b
        for qz in range(b):
            for qy in range(b):
                for qx in range(b):
                    x, y, z = ox + qx, oy + qy, oz + qz
                    if x < n[0] and y < n[1] and z < n[2]:
                        out.append(x + n[0] * (y + n[1] * z))
    return np.asarray(sorted(out), dtype=np.int64)


# contraction outputs that add up over the parts of a node partition
PART_SUM_KEYS = ("E_band", "E_s", "E_nl", "N_check", "E_pot", "pressure_A")


def run_partitioned(inst: dict, precision, rank: int, count: int, allreduce, bounds=None, stream=None):
    """One evaluation of part `rank` of `count` of the cell: the sweep over the part's tiles,
    allreduce(R^j) (the exchange step before the Fermi search), the Fermi level, the part's
    contraction and allreduce of the partial energies, pressure and sigma. `allreduce` maps a
    float64 numpy vector to its sum over the parts (torch.distributed, or any callable)."""
    d = Desc(inst, precision, bounds, stream, partition=(rank, count))
    h = sq_setup(d)
    try:
        sq_moments(h)
        n_pl = int(inst["n_pl"])
        R = allreduce(sq_node_sums(h, n_pl))
        mu = sq_fermi_level_sums(h, R)
        nd = int(np.prod(inst["n"]))
        rho, en, sig = sq_density_energy_stress(h, mu, nd)
        p_a, e_pot = sq_pressure(h, mu)
        part = dict(en)
        part["pressure_A"], part["E_pot"] = p_a, e_pot
        vec = np.concatenate([[part[k] for k in PART_SUM_KEYS], np.asarray(sig).reshape(9)])
        tot = allreduce(vec)
        out = {k: float(tot[i]) for i, k in enumerate(PART_SUM_KEYS)}
        out["F"] = out["E_band"] + out["E_s"]
        out["sigma"] = np.asarray(tot[len(PART_SUM_KEYS):]).reshape(3, 3)
        out["mu"] = mu
        out["rho_part"] = rho
        out["R"] = R
        out["bounds"] = sq_get_bounds(h)
        return out
    finally:
        sq_destroy(h)


def sq_density_energy_stress(h, mu: float, nd: int | None = None):
    """Host outputs: (rho (N_d,) or None, energies dict, sigma (3, 3))."""
    e = sq_energies()
    sig = np.zeros(9)
    rho = np.zeros(nd) if nd else None
    _check(lib().sq_density_energy_stress(h, C.c_double(mu), rho.ctypes.data if rho is not None else None,
                                          C.byref(e), sig.ctypes.data), h)
    en = {k: getattr(e, k) for k, _ in sq_energies._fields_}
    return rho, en, sig.reshape(3, 3)


def sq_density_energy_stress_dev(h, mu: float, rho_dev_ptr: int | None, sigma_dev_ptr: int | None, energies=True):
    e = sq_energies()
    _check(lib().sq_density_energy_stress_dev(h, C.c_double(mu), rho_dev_ptr, C.byref(e) if energies else None,
                                              sigma_dev_ptr), h)
    return {k: getattr(e, k) for k, _ in sq_energies._fields_} if energies else None


def sq_pressure(h, mu: float):
    """App. A pressure (kinetic + nonlocal terms), Ha/bohr^3, and E_pot (Ha)."""
    p, ep = C.c_double(), C.c_double()
    _check(lib().sq_pressure(h, C.c_double(mu), C.byref(p), C.byref(ep)), h)
    return p.value, ep.value


def sq_get_bounds(h):
    lo, hi = C.c_double(), C.c_double()
    _check(lib().sq_get_bounds(h, C.byref(lo), C.byref(hi)), h)
    return lo.value, hi.value


def sq_node_bounds(h, nd: int):
    """Per-node effective intervals (lo, hi), each (N_d,), in SQ_BOUNDS_PER_NODE mode."""
    lo, hi = np.zeros(nd), np.zeros(nd)
    _check(lib().sq_node_bounds(h, lo.ctypes.data, hi.ctypes.data), h)
    return lo, hi


def sq_moments_copy(h, nd: int, n_pl: int):
    out = np.zeros((nd, n_pl + 1, SQ_N_MOMENTS))
    _check(lib().sq_moments_copy(h, out.ctypes.data), h)
    return out


def sq_footprint_bytes(desc: Desc) -> int:
    return int(lib().sq_footprint_bytes(C.byref(desc.c)))


def sq_kernel_launches(h) -> int:
    return int(lib().sq_kernel_launches(h))


def sq_keep_lists(h, enable: bool = True):
    """Keeps the sweep's lists and W table of unchanged atom positions across sq_moments calls
    (SCF iterations with fixed atoms); off by default."""
    _check(lib().sq_keep_lists(h, 1 if enable else 0), h)


def sq_step_launch_counts(h):
    """Step-kernel launches by variant: (shared memory + tensor cores, shared memory + scalar,
    global-memory projections, TMA-staged step)."""
    c = (C.c_longlong * 4)()
    _check(lib().sq_step_launch_counts(h, c), h)
    return tuple(int(x) for x in c)


def sq_tune_step(h, n_warps: int = 0, wave_tiles: int = 0, reps: int = 0):
    """Sets the step kernel's warps per block and tiles per wave; with reps > 0 returns the
    timed milliseconds per tile and step, else None."""
    ms = C.c_double(0.0)
    _check(lib().sq_tune_step(h, int(n_warps), int(wave_tiles), int(reps), C.byref(ms) if reps > 0 else None), h)
    return ms.value if reps > 0 else None


TUNE_CACHE = Path(__file__).resolve().parent / "_lib" / "step_tune.json"


def autotune_step(h, inst: dict, precision, candidates_warps=(4, 5, 6, 7, 8), wave_fractions=(1, 2, 4),
                  reps: int = 3, cache: Path | None = TUNE_CACHE, partition=None):
    """Chooses warps per step block and tiles per wave for this handle's geometry by timing the
    candidates (sq_tune_step) and keeps the fastest; the choice is cached per geometry key
    (precision, n_o, region half-widths m, tiles) in a JSON file beside the built library, so the
    next handle of the same shape takes it without timing. Returns (key, choice, timings)."""
    import json
    n = np.asarray(inst["n"], dtype=np.int64)
    h_ = np.asarray(inst["L"], dtype=np.float64) / n
    m = np.floor(float(inst["r_cut"]) / h_ + 1e-9).astype(int)
    tiles = int(np.prod((n + 1) // 2))
    if partition is not None:                                # this part's tile range only
        r, c = int(partition[0]), int(partition[1])
        tiles = tiles * (r + 1) // c - tiles * r // c
    key = f"p{int(precision)}_no{int(inst['n_o'])}_m{'x'.join(str(x) for x in m)}_t{tiles}"
    table = {}
    if cache is not None and cache.exists():
        try:
            table = json.loads(cache.read_text())
        except ValueError:
            table = {}
    if key in table:
        w, wt = table[key]["warps"], table[key]["wave_tiles"]
        sq_tune_step(h, w, wt, 0)
        return key, table[key], None
    times = {}
    base = sq_tune_step(h, 0, 0, reps)                       # the default settings first
    times[(0, 0)] = base
    for frac in wave_fractions:
        wt = 0 if frac == 1 else max(1, tiles // frac)
        for w in candidates_warps:
            times[(w, wt)] = sq_tune_step(h, w, wt, reps)
    (w, wt), best = min(times.items(), key=lambda kv: kv[1])
    sq_tune_step(h, w, wt, 0)
    choice = {"warps": w, "wave_tiles": wt, "ms_per_tile": best, "default_ms_per_tile": base}
    if cache is not None:
        import os
        import tempfile
        table[key] = choice
        cache.parent.mkdir(exist_ok=True)
        fd, tmp = tempfile.mkstemp(dir=str(cache.parent), suffix=".json")   # atomic: ranks may share the file
        with os.fdopen(fd, "w") as f:
            f.write(json.dumps(table, indent=1))
        os.replace(tmp, cache)
    return key, choice, {f"{k[0]}w_{k[1]}t": v for k, v in times.items()}


def sq_kernel_timing(h, enable: bool):
    _check(lib().sq_kernel_timing(h, 1 if enable else 0), h)


def sq_kernel_timing_read(h, kid: int):
    """(launches, total_ms, algorithmic_bytes) of kernel class kid since timing was enabled."""
    n, ms, b = C.c_longlong(), C.c_double(), C.c_double()
    _check(lib().sq_kernel_timing_read(h, kid, C.byref(n), C.byref(ms), C.byref(b)), h)
    return n.value, ms.value, b.value


def sq_fermi_level_noalloc(mom_dev_ptr: int, n_nodes: int, n_pl: int, lambda_lo: float, lambda_hi: float,
                           kT: float, n_e: float, cheb_quad_M: int, stream, mu_dev_ptr: int):
    """Asynchronous; mu lands in the caller's device double at mu_dev_ptr."""
    rc = lib().sq_fermi_level_noalloc(mom_dev_ptr, n_nodes, n_pl, lambda_lo, lambda_hi, kT, n_e, cheb_quad_M,
                                      stream, mu_dev_ptr)
    if rc != SQ_OK:
        raise SQError(rc, "sq_fermi_level_noalloc rejected its arguments" if rc == SQ_ERR_INVALID_ARG
                      else "CUDA error in sq_fermi_level_noalloc")


def sq_destroy(h):
    if h:
        lib().sq_destroy(h)


def sq_last_error(h=None) -> str:
    return lib().sq_last_error(h).decode(errors="replace")


def run(inst: dict, precision=SQ_FP64, bounds=None, want_moments=False, stream=None):
    """setup -> moments -> Fermi level -> contraction -> destroy; returns a result dict."""
    d = Desc(inst, precision, bounds, stream)
    h = sq_setup(d)
    try:
        sq_moments(h)
        mu = sq_fermi_level(h)
        nd = int(np.prod(inst["n"]))
        rho, en, sig = sq_density_energy_stress(h, mu, nd)
        p_a, e_pot = sq_pressure(h, mu)
        out = {"mu": mu, "rho": rho, "sigma": sig, "bounds": sq_get_bounds(h),
               "launches": sq_kernel_launches(h), "pressure_A": p_a, "E_pot": e_pot,
               "step_variants": sq_step_launch_counts(h)}
        out.update(en)
        if want_moments:
            out["moments"] = sq_moments_copy(h, nd, int(inst["n_pl"]))
        if isinstance(bounds, str):
            out["node_bounds"] = sq_node_bounds(h, nd)
        return out
    finally:
        sq_destroy(h)


def sq_batch_evaluate(handles, max_concurrent: int = 0):
    """Evaluates every handle concurrently; returns (mu (n,), energies list, sigma (n, 3, 3))."""
    n = len(handles)
    arr = (C.c_void_p * max(1, n))(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    mu = np.zeros(n)
    en = (sq_energies * max(1, n))()
    sig = np.zeros((n, 9))
    rc = lib().sq_batch_evaluate(arr, n, max_concurrent, mu.ctypes.data, C.cast(en, C.c_void_p), sig.ctypes.data)
    if rc != SQ_OK:
        raise SQError(rc, "sq_batch_evaluate failed (see the handles' sq_last_error)")
    energies = [{k: getattr(en[i], k) for k, _ in sq_energies._fields_} for i in range(n)]
    return mu, energies, sig.reshape(n, 3, 3)


def sq_gauss_density(h, k: int, nd: int):
    """Gauss SQ density: (mu, rho (N_d,), E_band)."""
    mu, eb = C.c_double(), C.c_double()
    rho = np.zeros(nd)
    _check(lib().sq_gauss_density(h, int(k), C.byref(mu), rho.ctypes.data, C.byref(eb)), h)
    return mu.value, rho, eb.value


def sq_green_kubo(sigma, dt: float, volume: float, kT: float, max_lag: int, stream=None):
    """sigma: (n_traj, n_steps, 3, 3) stresses (Ha/bohr^3). Returns (eta (max_lag + 1,), acf)."""
    sig = np.ascontiguousarray(np.asarray(sigma, dtype=np.float64))
    if sig.ndim != 4 or sig.shape[2:] != (3, 3):
        raise ValueError("sigma must have shape (n_traj, n_steps, 3, 3)")
    eta = np.zeros(max_lag + 1)
    acf = np.zeros(max_lag + 1)
    rc = lib().sq_green_kubo(sig.ctypes.data, sig.shape[0], sig.shape[1], C.c_double(dt), C.c_double(volume),
                             C.c_double(kT), int(max_lag), stream, eta.ctypes.data, acf.ctypes.data)
    if rc != SQ_OK:
        raise SQError(rc, sq_last_error(None))
    return eta, acf


class Batch:
    """sq_batch_* : one CUDA graph evaluating a batch of handles (argument marshalling only)."""

    def __init__(self, handles):
        self.n = len(handles)
        arr = (C.c_void_p * self.n)(*[h.value for h in handles])
        self.b = C.c_void_p()
        rc = lib().sq_batch_create(arr, self.n, C.byref(self.b))
        if rc != SQ_OK:
            raise SQError(rc, "sq_batch_create failed: " + " / ".join(sq_last_error(h) for h in handles))

    def set_chains(self, chains: int):
        """Graph schedule: `chains` parallel chains of members (0 = all concurrent, 1 = serial)."""
        rc = lib().sq_batch_set_chains(self.b, int(chains))
        if rc != SQ_OK:
            raise SQError(rc, lib().sq_batch_last_error(self.b).decode(errors="replace"))

    def run(self):
        mu = np.zeros(self.n)
        en = (sq_energies * self.n)()
        sig = np.zeros((self.n, 9))
        rc = lib().sq_batch_run(self.b, mu.ctypes.data, en, sig.ctypes.data)
        if rc != SQ_OK:
            raise SQError(rc, lib().sq_batch_last_error(self.b).decode(errors="replace"))
        out = [{k: getattr(en[i], k) for k, _ in sq_energies._fields_} for i in range(self.n)]
        return mu, out, sig.reshape(self.n, 3, 3)

    def close(self):
        if self.b:
            lib().sq_batch_destroy(self.b)
            self.b = C.c_void_p()


class Server:
    """sq_server_* request loop (argument marshalling only)."""

    def __init__(self, hbm_budget_bytes: int, max_inflight: int):
        self.h = C.c_void_p()
        _check(lib().sq_server_create(int(hbm_budget_bytes), int(max_inflight), C.byref(self.h)))

    def submit(self, desc: Desc, tag: int, traj: int | None = None):
        if traj is None:
            rc = lib().sq_server_submit(self.h, C.byref(desc.c), int(tag))
        else:
            rc = lib().sq_server_submit_traj(self.h, C.byref(desc.c), int(tag), int(traj))
        if rc != SQ_OK:
            raise SQError(rc, "sq_server_submit rejected the request")

    def resident(self) -> int:
        return int(lib().sq_server_resident(self.h))

    def poll(self, max_results: int = 64, timeout_ms: int = 100):
        buf = (sq_result * max_results)()
        n = C.c_int()
        _check(lib().sq_server_poll(self.h, buf, max_results, timeout_ms, C.byref(n)))
        out = []
        for i in range(n.value):
            r = buf[i]
            out.append({"tag": r.tag, "status": r.status, "mu": r.mu, "latency_ms": r.latency_ms,
                        "error": r.error.decode(errors="replace"),
                        "sigma": np.array(list(r.sigma)).reshape(3, 3),
                        **{k: getattr(r.energies, k) for k, _ in sq_energies._fields_}})
        return out

    def pending(self) -> int:
        return int(lib().sq_server_pending(self.h))

    def close(self):
        if self.h:
            lib().sq_server_destroy(self.h)
            self.h = C.c_void_p()
