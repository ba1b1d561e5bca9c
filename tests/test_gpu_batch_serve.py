"""Batched and served evaluation: every instance gives the same result in a concurrent batch
or in the request loop's mix as when evaluated alone (FP64: 1e-10 relative; the projector
sums use atomics, so agreement is to rounding, not bitwise)."""
import numpy as np
import pytest

from oracle import sq_oracle as orc
from workloads import tiny_instance

pytestmark = pytest.mark.gpu

CASES = [
    dict(seed=21, n=(5, 6, 7), h=(0.7, 0.7, 0.7), n_atoms=3, n_o=2, r_cut=2.0, n_pl=16),
    dict(seed=22, n=(8, 8, 8), h=(0.6, 0.6, 0.6), n_atoms=4, n_o=3, r_cut=2.4, n_pl=24),
    dict(seed=23, n=(4, 4, 4), h=(0.8, 0.8, 0.8), n_atoms=1, n_o=1, r_cut=1.6, n_pl=12),
    dict(seed=24, n=(6, 6, 6), h=(0.7, 0.7, 0.7), n_atoms=2, n_o=4, r_cut=3.0, n_pl=30),
]


@pytest.fixture(scope="module")
def sq():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2006_03697_gb300 import build
    build.build()
    from paper_2006_03697_gb300 import sq as mod
    return mod


@pytest.fixture(scope="module")
def alone(sq):
    out = []
    for c in CASES:
        inst = tiny_instance(**c)
        b = orc.lanczos_bounds(orc.Problem(inst))
        out.append((inst, b, sq.run(inst, sq.SQ_FP64, bounds=b)))
    return out


def _same(a, b):
    assert abs(a["mu"] - b["mu"]) <= 1e-10 * max(1.0, abs(b["mu"]))
    for k in ("E_band", "E_s", "E_nl", "F"):
        assert abs(a[k] - b[k]) <= 1e-10 * max(1.0, abs(b[k])), k
    assert np.abs(np.asarray(a["sigma"]) - np.asarray(b["sigma"])).max() <= 1e-10 * max(1e-3, np.abs(b["sigma"]).max())


def test_batch_equals_alone(sq, alone):
    import torch
    streams = [torch.cuda.Stream() for _ in alone]
    descs = [sq.Desc(inst, sq.SQ_FP64, bounds=b, stream=s.cuda_stream) for (inst, b, _), s in zip(alone, streams)]
    hs = [sq.sq_setup(d) for d in descs]
    try:
        mu, en, sig = sq.sq_batch_evaluate(hs, max_concurrent=4)
    finally:
        for h in hs:
            sq.sq_destroy(h)
    for i, (_, _, ref) in enumerate(alone):
        _same({"mu": mu[i], "sigma": sig[i], **en[i]}, ref)


def test_server_mix_equals_alone(sq, alone):
    srv = sq.Server(hbm_budget_bytes=4 << 30, max_inflight=3)
    try:
        descs = []
        for rep in range(3):
            for i, (inst, b, _) in enumerate(alone):
                d = sq.Desc(inst, sq.SQ_FP64, bounds=b)
                descs.append(d)
                srv.submit(d, tag=100 * rep + i)
        got = []
        for _ in range(600):
            got += srv.poll(timeout_ms=100)
            if len(got) == len(descs):
                break
        assert len(got) == len(descs)
        lat = np.array([r["latency_ms"] for r in got])
        assert np.all(lat > 0)
        for r in got:
            assert r["status"] == sq.SQ_OK
            _same(r, alone[r["tag"] % 100][2])
        assert srv.pending() == 0
    finally:
        srv.close()


def test_served_trajectory_green_kubo(sq):
    """A synthetic trajectory (successively perturbed positions of one cell) served through the
    request loop, its stress stream fed to sq_green_kubo: every request succeeds, results come
    back for every step, the autocorrelation at lag 0 is the mean squared deviatoric stress of
    the stream and the running viscosity starts at 0."""
    from workloads import gaussian_veff, perturb_positions
    base = tiny_instance(seed=31, n=(6, 6, 6), h=(0.7, 0.7, 0.7), n_atoms=3, n_o=2, r_cut=2.0, n_pl=16)
    rng = np.random.Generator(np.random.PCG64(31))
    steps = 8
    srv = sq.Server(hbm_budget_bytes=4 << 30, max_inflight=4)
    descs, pos = [], np.asarray(base["pos"])
    try:
        for k in range(steps):
            pos = perturb_positions(rng, pos, 0.05, base["L"])
            inst = dict(base)
            inst["pos"] = pos
            inst["v_eff"] = gaussian_veff(base["L"], base["n"], pos)
            d = sq.Desc(inst, sq.SQ_FP64, bounds=(-1.0, 20.0))   # contains [0.64, 15.1] with margin
            descs.append(d)
            srv.submit(d, tag=k)
        got = []
        for _ in range(600):
            got += srv.poll(timeout_ms=100)
            if len(got) == steps:
                break
    finally:
        srv.close()
    assert len(got) == steps and all(r["status"] == sq.SQ_OK for r in got)
    sig = np.array([r["sigma"] for r in sorted(got, key=lambda r: r["tag"])]).reshape(1, steps, 3, 3)
    eta, acf = sq.sq_green_kubo(sig, 16.5, float(np.prod(base["L"])), float(base["kT"]), steps // 2)
    s = np.stack([sig[0, :, 0, 1], sig[0, :, 1, 2], sig[0, :, 2, 0], 0.5 * (sig[0, :, 0, 0] - sig[0, :, 1, 1]),
                  0.5 * (sig[0, :, 1, 1] - sig[0, :, 2, 2])], axis=1)
    assert acf[0] == pytest.approx(float(np.mean(s * s)), rel=1e-12)
    assert eta[0] == 0.0 and np.all(np.isfinite(eta))
