"""A batch of uneven instances evaluated by one CUDA graph (sq_batch_create / sq_batch_run)
through the C ABI: every member's result equals its alone evaluation; launching the graph again
repeats them; after sq_update_atoms on a member (the next quantum-MD snapshot) the same graph
evaluates the new snapshot."""
import numpy as np
import pytest

from workloads import gaussian_veff, make_batch, perturb_positions, tiny_instance

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


def _members(sq):
    return [
        (tiny_instance(seed=1, n=(5, 6, 7), h=(0.7, 0.65, 0.6), n_atoms=3, n_o=2, r_cut=2.0, n_pl=16), sq.SQ_FP64, None),
        (tiny_instance(seed=2, n=(6, 6, 6), h=(0.6, 0.6, 0.6), n_atoms=2, n_o=3, r_cut=1.8, n_pl=22), sq.SQ_MIXED, None),
        (tiny_instance(seed=3, n=(4, 5, 4), h=(0.8, 0.8, 0.8), n_atoms=1, n_o=1, r_cut=0.9, n_pl=9), sq.SQ_FP64,
         (-4.0, 30.0)),
        (make_batch(config=4, count=1, atom_choices=(32,))[0], sq.SQ_MIXED, None),
    ]


def _check(r_mu, r_en, r_sig, ref, rtol):
    assert abs(r_mu - ref["mu"]) <= rtol * max(1.0, abs(ref["mu"]))
    for k in ("E_band", "E_s", "E_nl", "F", "N_check"):
        assert abs(r_en[k] - ref[k]) <= rtol * max(1.0, abs(ref[k])), k
    assert np.abs(r_sig - ref["sigma"]).max() <= rtol * max(1.0, np.abs(ref["sigma"]).max())


def test_graph_batch_equals_alone_and_relaunches(sq):
    import torch
    members = _members(sq)
    streams = [torch.cuda.Stream() for _ in members]
    hs = [sq.sq_setup(sq.Desc(inst, prec, bounds=b, stream=st.cuda_stream)) for (inst, prec, b), st in zip(members, streams)]
    batch = None
    try:
        batch = sq.Batch(hs)
        refs = [sq.run(inst, prec, bounds=b) for inst, prec, b in members]
        for rep in range(2):                          # the second launch repeats the first
            mu, en, sig = batch.run()
            for i, ((inst, prec, b), ref) in enumerate(zip(members, refs)):
                _check(mu[i], en[i], sig[i], ref, 1e-10 if prec == sq.SQ_FP64 else 1e-7)
        # after the launch the members hold their moments: another contraction works on them
        rho, e2, s2 = sq.sq_density_energy_stress(hs[0], mu[0], int(np.prod(members[0][0]["n"])))
        assert abs(e2["F"] - refs[0]["F"]) <= 1e-10 * abs(refs[0]["F"])
        # any schedule of the graph (serial chain, two chains) gives the same results
        for chains in (1, 2):
            batch.set_chains(chains)
            mu_c, en_c, sig_c = batch.run()
            for i, ((inst, prec, b), ref) in enumerate(zip(members, refs)):
                _check(mu_c[i], en_c[i], sig_c[i], ref, 1e-10 if prec == sq.SQ_FP64 else 1e-7)
        batch.set_chains(0)
        # the next snapshot of member 1 through the same graph
        rng = np.random.Generator(np.random.PCG64(77))
        nxt = dict(members[1][0])
        nxt["pos"] = perturb_positions(rng, np.asarray(nxt["pos"]), 0.3, nxt["L"])
        nxt["v_eff"] = gaussian_veff(nxt["L"], nxt["n"], nxt["pos"])
        sq.sq_update_atoms(hs[1], nxt["pos"], nxt["v_eff"])
        mu, en, sig = batch.run()
        _check(mu[1], en[1], sig[1], sq.run(nxt, sq.SQ_MIXED, bounds=None), 1e-7)
        _check(mu[0], en[0], sig[0], refs[0], 1e-10)
    finally:
        if batch is not None:
            batch.close()
        for h in hs:
            sq.sq_destroy(h)


def test_graph_batch_rejects_shared_streams(sq):
    import torch
    st = torch.cuda.Stream()
    insts = [tiny_instance(seed=s, n=(4, 4, 4), h=(0.8, 0.8, 0.8), n_atoms=1, n_o=1, r_cut=0.9, n_pl=8) for s in (4, 5)]
    hs = [sq.sq_setup(sq.Desc(i, sq.SQ_FP64, bounds=(-4.0, 30.0), stream=st.cuda_stream)) for i in insts]
    try:
        with pytest.raises(sq.SQError) as ei:
            sq.Batch(hs)
        assert ei.value.code == sq.SQ_ERR_INVALID_ARG
    finally:
        for h in hs:
            sq.sq_destroy(h)


def test_tuned_step_settings_keep_parity(sq):
    """Every setting the autotuner may pick (warps per step block, tiles per wave) gives the
    default's result: FP64 to 1e-10, mixed to the projector atomics' rounding."""
    inst = tiny_instance(seed=1, n=(5, 6, 7), h=(0.7, 0.65, 0.6), n_atoms=3, n_o=2, r_cut=2.0, n_pl=16)
    nd = int(np.prod(inst["n"]))
    for prec, rtol in ((sq.SQ_FP64, 1e-10), (sq.SQ_MIXED, 1e-7)):
        ref = sq.run(inst, prec, bounds=(-4.0, 40.0))
        h = sq.sq_setup(sq.Desc(inst, prec, bounds=(-4.0, 40.0)))
        try:
            sq.sq_moments(h)
            for warps, wave_tiles in ((4, 0), (8, 0), (5, 7), (0, 3)):
                ms = sq.sq_tune_step(h, warps, wave_tiles, reps=1)
                assert ms > 0.0
                sq.sq_moments(h)
                mu = sq.sq_fermi_level(h)
                rho, en, sig = sq.sq_density_energy_stress(h, mu, nd)
                _check(mu, en, sig, ref, rtol)
        finally:
            sq.sq_destroy(h)
    with pytest.raises(sq.SQError):
        h = sq.sq_setup(sq.Desc(inst, sq.SQ_FP64, bounds=(-4.0, 40.0)))
        try:
            sq.sq_tune_step(h, 9, 0, 0)
        finally:
            sq.sq_destroy(h)
