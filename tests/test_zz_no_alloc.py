"""The allocation-free Fermi-level entry point against the regular one, through the C ABI.

sq_fermi_level_noalloc serves callers that cannot call cudaMalloc; its scratch is a fixed
device array inside the library. It must give the same mu as sq_fermi_level on the same
moment table, on two calls in a row (the second call reuses the scratch the first left)."""
import numpy as np
import pytest

from workloads import tiny_instance

pytestmark = pytest.mark.gpu


def test_noalloc_fermi_level_matches_regular_entry_point():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2006_03697_gb300 import build
    build.build()
    from paper_2006_03697_gb300 import sq

    results = []
    for seed, n_pl in ((11, 14), (12, 22)):
        inst = tiny_instance(seed=seed, n=(5, 6, 4), h=(0.7, 0.7, 0.7), n_atoms=2, n_o=2, r_cut=1.5, n_pl=n_pl)
        nd = int(np.prod(inst["n"]))
        h = sq.sq_setup(sq.Desc(inst, sq.SQ_FP64))
        try:
            sq.sq_moments(h)
            mu_ref = sq.sq_fermi_level(h)
            lo, hi = sq.sq_get_bounds(h)
            mom = sq.sq_moments_copy(h, nd, n_pl)
        finally:
            sq.sq_destroy(h)
        mom_dev = torch.from_numpy(mom).cuda()
        mu_dev = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        sq.sq_fermi_level_noalloc(mom_dev.data_ptr(), nd, n_pl, lo, hi, inst["kT"], inst["n_e"], 2048, stream,
                                  mu_dev.data_ptr())
        torch.cuda.synchronize()
        mu = float(mu_dev.item())
        assert abs(mu - mu_ref) <= 1e-12 * max(1.0, abs(mu_ref)), (mu, mu_ref)
        results.append(mu)
    assert results[0] != results[1]

    # a moment table that cannot bracket N_e (all zero: N(mu) = 0 everywhere) gives NaN, and
    # the next regular call is unaffected by the scratch this one left
    zeros = torch.zeros((nd, n_pl + 1, sq.SQ_N_MOMENTS), dtype=torch.float64, device="cuda")
    sq.sq_fermi_level_noalloc(zeros.data_ptr(), nd, n_pl, lo, hi, inst["kT"], inst["n_e"], 2048, stream,
                              mu_dev.data_ptr())
    torch.cuda.synchronize()
    assert np.isnan(float(mu_dev.item()))
    sq.sq_fermi_level_noalloc(mom_dev.data_ptr(), nd, n_pl, lo, hi, inst["kT"], inst["n_e"], 2048, stream,
                              mu_dev.data_ptr())
    torch.cuda.synchronize()
    assert abs(float(mu_dev.item()) - results[1]) <= 1e-12 * max(1.0, abs(results[1]))

    # sizes beyond the fixed scratch are rejected before any launch
    with pytest.raises(sq.SQError) as ei:
        sq.sq_fermi_level_noalloc(mom_dev.data_ptr(), nd, 5000, lo, hi, 1.0, 1.0, 2048, None, mu_dev.data_ptr())
    assert ei.value.code == sq.SQ_ERR_INVALID_ARG
