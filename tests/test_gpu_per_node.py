"""Per-node spectral bounds (SQ_BOUNDS_PER_NODE): the literal reading of Sec. 4, where chi_q and
zeta_q come from the extreme eigenvalues of each node's own H_q, against the FP64 oracle of that
mode (oracle/per_node.py, pinned by P12) through the C ABI.

The device's per-node Lanczos intervals are compared with the oracle's (1e-9 of each node's
width in FP64, the agreement of the shared-interval Lanczos; 1e-5 with the FP32 Krylov vectors
of SQ_MIXED). The oracle then runs its per-node moments, Fermi search and contraction with the
device's effective intervals (the ones the recurrence realises), so that the sweep, the
per-node coefficient tables of the Fermi search and the contraction are compared at 1e-10 in
FP64 and at the mixed tolerances (1e-6 relative in energy, 1e-5 Ha/bohr^3 in sigma)."""
import numpy as np
import pytest

from oracle import per_node
from oracle import sq_oracle as orc
from workloads import make_instance, tiny_instance

pytestmark = pytest.mark.gpu

CASES = {
    "ragged_sp": dict(seed=1, n=(5, 6, 7), h=(0.7, 0.65, 0.6), n_atoms=3, n_o=2, r_cut=2.0, n_pl=16,
                      proj=[{"l": 0, "width": 0.5, "gamma": 1.0, "rcut": 3.5},
                            {"l": 1, "width": 0.5, "gamma": -0.5, "rcut": 3.5}]),
    "m1_no1": dict(seed=2, n=(4, 4, 4), h=(0.8, 0.8, 0.8), n_atoms=2, n_o=1, r_cut=0.9, n_pl=10),
    "no_atoms": dict(seed=3, n=(6, 5, 4), h=(0.7, 0.7, 0.7), n_atoms=0, n_o=3, r_cut=2.2, n_pl=14),
    "thin_cell": dict(seed=5, n=(1, 3, 2), h=(0.9, 0.8, 0.7), n_atoms=1, n_o=2, r_cut=2.0, n_pl=8),
}
_CACHE = {}


@pytest.fixture(scope="module")
def sq():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2006_03697_gb300 import build
    build.build()
    from paper_2006_03697_gb300 import sq as mod
    return mod


def _oracle_bounds(name, inst):
    if name not in _CACHE:
        prob = orc.Problem(inst)
        _CACHE[name] = np.array([per_node.node_bounds(prob, q) for q in range(prob.Nd)])
    return _CACHE[name]


def _device(sq, inst, precision):
    nd = int(np.prod(inst["n"]))
    h = sq.sq_setup(sq.Desc(inst, precision, bounds="per_node"))
    try:
        sq.sq_moments(h)
        lo, hi = sq.sq_node_bounds(h, nd)
        mom = sq.sq_moments_copy(h, nd, int(inst["n_pl"]))
        mu = sq.sq_fermi_level(h)
        rho, en, sig = sq.sq_density_energy_stress(h, mu, nd)
        glo, ghi = sq.sq_get_bounds(h)
        launches = sq.sq_step_launch_counts(h)
    finally:
        sq.sq_destroy(h)
    return dict(en, lo=lo, hi=hi, moments=mom, mu=mu, rho=rho, sigma=sig, glo=glo, ghi=ghi, launches=launches)


@pytest.mark.parametrize("name", sorted(CASES))
def test_per_node_fp64_parity(sq, name):
    inst = tiny_instance(**CASES[name])
    prob = orc.Problem(inst)
    g = _device(sq, inst, sq.SQ_FP64)
    ob = _oracle_bounds(name, inst)
    wdt = ob[:, 1] - ob[:, 0]
    assert np.all(np.abs(g["lo"] - ob[:, 0]) <= 1e-9 * wdt)
    assert np.all(np.abs(g["hi"] - ob[:, 1]) <= 1e-9 * wdt)
    assert g["glo"] == g["lo"].min() and g["ghi"] == g["hi"].max()
    # with atoms the intervals really differ from node to node (not one shared interval)
    if len(inst["pos"]) > 0 and prob.Nd > 1:
        assert np.ptp(g["hi"] - g["lo"]) > 1e-6
    B = np.stack([g["lo"], g["hi"]], axis=1)
    mom = per_node.moments(prob, B)
    for k in range(mom.shape[2]):
        scale = max(np.abs(mom[:, :, k]).max(), 1e-3)
        assert np.abs(g["moments"][:, :, k] - mom[:, :, k]).max() <= 1e-10 * scale, k
    mu = per_node.fermi_bisect(prob, mom, B)
    o = per_node.contract(prob, mom, B, mu)
    assert abs(g["mu"] - mu) <= 1e-10 * max(1.0, abs(mu))
    for key in ("E_band", "E_s", "E_nl", "N_check"):
        assert abs(g[key] - o[key]) <= 1e-10 * max(1.0, abs(o[key])), key
    assert np.abs(g["rho"] - o["rho"]).max() <= 1e-10 * np.abs(o["rho"]).max()
    assert np.abs(g["sigma"] - o["sigma"]).max() <= 1e-10 * max(np.abs(o["sigma"]).max(), 1e-3)


@pytest.mark.parametrize("name", ["ragged_sp", "m1_no1", "thin_cell"])
def test_per_node_mixed(sq, name):
    inst = tiny_instance(**CASES[name])
    prob = orc.Problem(inst)
    g = _device(sq, inst, sq.SQ_MIXED)
    assert g["launches"][0] > 0                       # the tensor-core step variant ran
    ob = _oracle_bounds(name, inst)
    wdt = ob[:, 1] - ob[:, 0]
    assert np.all(np.abs(g["lo"] - ob[:, 0]) <= 1e-5 * wdt)
    assert np.all(np.abs(g["hi"] - ob[:, 1]) <= 1e-5 * wdt)
    B = np.stack([g["lo"], g["hi"]], axis=1)
    mom = per_node.moments(prob, B)
    mu = per_node.fermi_bisect(prob, mom, B)
    o = per_node.contract(prob, mom, B, mu)
    for key in ("E_band", "E_s", "F"):
        assert abs(g[key] - o[key]) <= 1e-6 * abs(o[key]), key
    assert abs(g["E_nl"] - o["E_nl"]) <= 1e-6 * abs(o["E_nl"]) + 1e-10
    assert np.abs(g["sigma"] - o["sigma"]).max() <= 1e-5
    assert abs(g["N_check"] - inst["n_e"]) <= 1e-9 * inst["n_e"]


def test_per_node_config1_converges_to_shared_mode(sq):
    """8 H / 12^3: the per-node and the shared-interval evaluations describe the same density
    matrix up to the Chebyshev truncation (P2 tail of each scaling)."""
    inst = make_instance(1)
    pn = _device(sq, inst, sq.SQ_FP64)
    sh = sq.run(inst, sq.SQ_FP64, bounds=None)
    assert abs(pn["N_check"] - inst["n_e"]) <= 1e-9 * inst["n_e"]
    assert abs(pn["F"] - sh["F"]) <= 1e-6 * abs(sh["F"])
    assert np.abs(pn["sigma"] - sh["sigma"]).max() <= 1e-6


def test_per_node_rejects_partition(sq):
    inst = tiny_instance(**CASES["m1_no1"])
    with pytest.raises(sq.SQError) as ei:
        sq.sq_setup(sq.Desc(inst, sq.SQ_FP64, bounds="per_node", partition=(0, 2)))
    assert ei.value.code == sq.SQ_ERR_INVALID_ARG
