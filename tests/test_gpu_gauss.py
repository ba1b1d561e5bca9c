"""Gauss SQ density through the C ABI against the oracle (oracle/gauss_sq.py, pinned by P13):
Fermi level, density and band energy on the edge cases, FP64 at 1e-10 relative, mixed
precision (FP32 Lanczos vectors) at 1e-6 on the energy and 1e-5 on the density."""
import numpy as np
import pytest

from oracle import gauss_sq
from workloads import tiny_instance

pytestmark = pytest.mark.gpu

CASES = {
    "ragged_sp": dict(seed=1, n=(5, 6, 7), h=(0.7, 0.65, 0.6), n_atoms=3, n_o=2, r_cut=2.0, n_pl=16,
                      proj=[{"l": 0, "width": 0.5, "gamma": 1.0, "rcut": 3.5},
                            {"l": 1, "width": 0.5, "gamma": -0.5, "rcut": 3.5}]),
    "m1_no1": dict(seed=2, n=(4, 4, 4), h=(0.8, 0.8, 0.8), n_atoms=2, n_o=1, r_cut=0.9, n_pl=10),
    "no_atoms": dict(seed=3, n=(6, 5, 4), h=(0.7, 0.7, 0.7), n_atoms=0, n_o=3, r_cut=2.2, n_pl=14),
    "thin_cell": dict(seed=5, n=(1, 3, 2), h=(0.9, 0.8, 0.7), n_atoms=1, n_o=2, r_cut=2.0, n_pl=8),
}


@pytest.fixture(scope="module")
def sq():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2006_03697_gb300 import build
    build.build()
    from paper_2006_03697_gb300 import sq as mod
    return mod


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gauss_density_matches_oracle(sq, name, precision):
    inst = tiny_instance(**CASES[name])
    k = 20
    ref = gauss_sq.run(inst, k=k)
    nd = int(np.prod(inst["n"]))
    mode = sq.SQ_FP64 if precision == "fp64" else sq.SQ_MIXED
    h = sq.sq_setup(sq.Desc(inst, mode, bounds=(-5.0, 60.0)))
    try:
        mu, rho, eb = sq.sq_gauss_density(h, k, nd)
    finally:
        sq.sq_destroy(h)
    if precision == "fp64":
        assert abs(mu - ref["mu"]) <= 1e-10 * max(1.0, abs(ref["mu"]))
        assert np.abs(rho - ref["rho"]).max() <= 1e-10 * np.abs(ref["rho"]).max()
        assert abs(eb - ref["E_band"]) <= 1e-10 * max(1.0, abs(ref["E_band"]))
    else:
        assert abs(mu - ref["mu"]) <= 1e-5 * max(1.0, abs(ref["mu"]))
        assert np.abs(rho - ref["rho"]).max() <= 1e-5 * np.abs(ref["rho"]).max()
        assert abs(eb - ref["E_band"]) <= 1e-6 * max(1.0, abs(ref["E_band"]))
    assert abs(rho.sum() * float(np.prod(np.asarray(inst["L"]) / np.asarray(inst["n"]))) - inst["n_e"]) <= 1e-9 * inst["n_e"]
