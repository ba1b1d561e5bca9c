"""Error table of the mixed-precision path (FP32 recurrence and projectors, FP64 sums,
bounds, coefficients, bisection and contraction) for the precision workload:

  * config 1 (8 H, 12^3 nodes) against the FP64 CPU oracle,
  * the 216 H, 18 bohr, 60^3-node instance against the FP64 GPU path (which matches the
    oracle to 1e-10 on sampled nodes), same spectral bounds on both sides.

Targets: energy within 1e-6 relative, each sigma_ab within 1e-5 Ha/bohr^3; the density
error is reported. The table is printed (pytest -s)."""
import numpy as np
import pytest

from oracle import sq_oracle as orc
from workloads import make_instance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sq():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2006_03697_gb300 import build
    build.build()
    from paper_2006_03697_gb300 import sq as mod
    return mod


def _table(name, mixed, ref):
    rows = [f"precision {name}: mixed vs reference"]
    for key in ("E_band", "E_s", "E_nl", "F", "mu", "E_pot"):
        rel = abs(mixed[key] - ref[key]) / max(1e-300, abs(ref[key]))
        rows.append(f"  {key:7s} {ref[key]: .12e}  rel err {rel:.2e}")
    rows.append(f"  P (App. A) {ref['pressure_A']: .12e}  abs err {abs(mixed['pressure_A'] - ref['pressure_A']):.2e}")
    drho = np.abs(mixed["rho"] - ref["rho"]).max() / np.abs(ref["rho"]).max()
    rows.append(f"  rho     max rel err {drho:.2e}")
    ds = np.abs(np.asarray(mixed["sigma"]) - np.asarray(ref["sigma"]))
    for a in range(3):
        rows.append("  sigma   " + "  ".join(f"{ds[a, b]:.2e}" for b in range(3)) + "  (Ha/bohr^3, abs)")
    print("\n".join(rows))
    return ds


def _check(mixed, ref, ds):
    # every energy within 1e-6 of its own magnitude, each sigma_ab within 1e-5 Ha/bohr^3
    for key in ("E_band", "E_s", "E_nl", "F"):
        assert abs(mixed[key] - ref[key]) <= 1e-6 * abs(ref[key]), key
    assert ds.max() <= 1e-5
    assert abs(mixed["pressure_A"] - ref["pressure_A"]) <= 1e-5


def test_precision_config1_vs_oracle(sq):
    inst = make_instance(1)
    bounds = orc.lanczos_bounds(orc.Problem(inst))
    ref = orc.run(inst, bounds=bounds, workers=8)
    mixed = sq.run(inst, sq.SQ_MIXED, bounds=bounds)
    _check(mixed, ref, _table("config 1 (8 H, 12^3) vs FP64 oracle", mixed, ref))


def test_precision_216_atoms_vs_fp64_gpu(sq):
    inst = make_instance(3)
    ref = sq.run(inst, sq.SQ_FP64, bounds=None)            # device Lanczos bounds
    mixed = sq.run(inst, sq.SQ_MIXED, bounds=ref["bounds"])
    _check(mixed, ref, _table("216 H, 60^3 vs FP64 GPU path", mixed, ref))
    assert abs(mixed["N_check"] - inst["n_e"]) <= 1e-9 * inst["n_e"]


def test_precision_bench_workload_vs_fp64_gpu(sq):
    """The benchmarked configuration (64 H, 40^3 nodes, 27^3 regions, n_pl = 60) in the launch
    configuration bench.py times: mixed precision against the plain FP64 GPU path (which matches
    the oracle to 1e-10 on sampled nodes), same spectral bounds, on E_band, E_s, E_nl, F, the
    App. A pressure and every sigma_ab."""
    inst = make_instance(2)
    ref = sq.run(inst, sq.SQ_FP64, bounds=None)            # device Lanczos bounds
    mixed = sq.run(inst, sq.SQ_MIXED, bounds=ref["bounds"])
    _check(mixed, ref, _table("64 H, 40^3 (bench workload) vs FP64 GPU path", mixed, ref))
    assert abs(mixed["N_check"] - inst["n_e"]) <= 1e-9 * inst["n_e"]
