"""The C-ABI library builds, loads and exports every symbol include/sq_api.h declares;
host-side validation and footprint logic (no GPU compute calls)."""
import re
from pathlib import Path

import numpy as np
import pytest

from workloads import make_instance, tiny_instance

ROOT = Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module")
def sq():
    from paper_2006_03697_gb300 import build
    build.build()
    from paper_2006_03697_gb300 import sq as mod
    return mod


def test_header_symbols_exported(sq):
    hdr = (ROOT / "include" / "sq_api.h").read_text()
    names = set(re.findall(r"\b(sq_[a-z_]+)\s*\(", hdr))
    assert names, "no declarations parsed"
    L = sq.lib()
    for n in sorted(names):
        assert hasattr(L, n), n
    assert names == set(sq.EXPORTED)


def test_footprint_scales_with_problem(sq):
    f1 = sq.sq_footprint_bytes(sq.Desc(make_instance(1), sq.SQ_FP64, bounds=(-1.0, 40.0)))
    f1m = sq.sq_footprint_bytes(sq.Desc(make_instance(1), sq.SQ_MIXED, bounds=(-1.0, 40.0)))
    f2 = sq.sq_footprint_bytes(sq.Desc(make_instance(2), sq.SQ_FP64, bounds=(-1.0, 130.0)))
    f2m = sq.sq_footprint_bytes(sq.Desc(make_instance(2), sq.SQ_MIXED, bounds=(-1.0, 130.0)))
    assert 0 < f1 < f2
    assert 0 < f1m < f1            # one wave: FP32 vectors and tables take less room
    # per-tile buffers that fit in 64 GiB form one wave (config 2 in mixed precision, about
    # 50 GB); larger ones run in waves of at most 24 GiB (config 2 in FP64)
    assert 32 << 30 < f2m < 66 << 30
    assert f2 < 32 << 30


@pytest.mark.parametrize("field,value", [
    ("n_o", 0), ("n_o", 7), ("kT", 0.0), ("n_e", 0.0), ("n_e", 1e9), ("r_cut", 0.01), ("n_pl", 0),
    ("precision", 5), ("bounds_mode", 9),
])
def test_setup_rejects_invalid_descriptor(sq, field, value):
    d = sq.Desc(tiny_instance(seed=0), sq.SQ_FP64, bounds=(-1.0, 20.0))
    setattr(d.c, field, value)
    with pytest.raises(sq.SQError) as ei:
        sq.sq_setup(d)
    assert ei.value.code == sq.SQ_ERR_INVALID_ARG
    assert sq.sq_last_error(None) != "no error"


def test_setup_rejects_nan_potential_and_bad_bounds(sq):
    inst = tiny_instance(seed=0)
    inst["v_eff"] = np.asarray(inst["v_eff"]).copy()
    inst["v_eff"][3] = np.nan
    with pytest.raises(sq.SQError) as ei:
        sq.sq_setup(sq.Desc(inst, sq.SQ_FP64, bounds=(-1.0, 20.0)))
    assert ei.value.code == sq.SQ_ERR_INVALID_ARG
    with pytest.raises(sq.SQError) as ei:
        sq.sq_setup(sq.Desc(tiny_instance(seed=0), sq.SQ_FP64, bounds=(5.0, 5.0)))
    assert ei.value.code == sq.SQ_ERR_INVALID_ARG


def test_null_handle_calls_are_rejected(sq):
    L = sq.lib()
    assert L.sq_moments(None) == sq.SQ_ERR_INVALID_ARG
    assert L.sq_fermi_level(None, None) == sq.SQ_ERR_INVALID_ARG
    assert L.sq_pressure(None, 0.0, None, None) == sq.SQ_ERR_INVALID_ARG
    assert L.sq_gauss_density(None, 20, None, None, None) == sq.SQ_ERR_INVALID_ARG
    assert L.sq_kernel_launches(None) == 0
    L.sq_destroy(None)


def test_server_refuses_request_larger_than_budget(sq):
    """Admission by device footprint: a request that can never fit completes with SQ_ERR_OOM
    without touching a GPU."""
    srv = sq.Server(hbm_budget_bytes=1024, max_inflight=2)
    try:
        d = sq.Desc(tiny_instance(seed=0), sq.SQ_FP64, bounds=(-1.0, 20.0))
        srv.submit(d, tag=7)
        got = []
        for _ in range(50):
            got += srv.poll(timeout_ms=100)
            if got:
                break
        assert len(got) == 1 and got[0]["tag"] == 7 and got[0]["status"] == sq.SQ_ERR_OOM
        assert srv.pending() == 0
    finally:
        srv.close()


def test_server_rejects_invalid_descriptor(sq):
    srv = sq.Server(hbm_budget_bytes=1 << 30, max_inflight=1)
    try:
        d = sq.Desc(tiny_instance(seed=0), sq.SQ_FP64, bounds=(-1.0, 20.0))
        d.c.n_o = 0
        with pytest.raises(sq.SQError):
            srv.submit(d, tag=1)
    finally:
        srv.close()


def test_green_kubo_rejects_bad_arguments_before_any_device_work(sq):
    import numpy as np
    sig = np.zeros((1, 10, 3, 3))
    for kw in (dict(max_lag=10), dict(max_lag=-1), dict(dt=0.0), dict(volume=-1.0), dict(kT=0.0)):
        args = dict(dt=1.0, volume=1.0, kT=1.0, max_lag=3)
        args.update(kw)
        with pytest.raises(sq.SQError) as ei:
            sq.sq_green_kubo(sig, **args)
        assert ei.value.code == sq.SQ_ERR_INVALID_ARG
    with pytest.raises(sq.SQError):
        sq.sq_green_kubo(np.zeros((1, 1, 3, 3)), 1.0, 1.0, 1.0, 0)
