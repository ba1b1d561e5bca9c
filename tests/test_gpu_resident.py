"""Resident state across the snapshots of a trajectory (quantum MD: the atoms move a little
between consecutive stress evaluations), through the C ABI.

sq_update_atoms moves the atoms and V_eff of a live handle in place: its results must equal a
fresh sq_setup of the new snapshot (FP64 to 1e-10 relative, the repeat-call agreement of the
projector sums' atomics). The request loop keeps one handle per trajectory resident and gives
each served snapshot its fresh, alone result."""
import numpy as np
import pytest

from workloads import gaussian_veff, perturb_positions, tiny_instance

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


def _trajectory(n_snap=3, seed=5):
    base = tiny_instance(seed=seed, n=(6, 5, 6), h=(0.6, 0.6, 0.6), n_atoms=3, n_o=3, r_cut=1.8, n_pl=14)
    rng = np.random.Generator(np.random.PCG64(424242))
    snaps = [base]
    for _ in range(n_snap - 1):
        s = dict(snaps[-1])
        # big enough moves to shift support boxes by lattice points and change argmin / argmax V
        s["pos"] = perturb_positions(rng, np.asarray(s["pos"]), 0.35, s["L"])
        s["v_eff"] = gaussian_veff(s["L"], s["n"], s["pos"])
        snaps.append(s)
    return snaps


def _close(a, b, rtol):
    for k in ("mu", "E_band", "E_s", "E_nl", "N_check", "E_pot", "pressure_A"):
        assert abs(a[k] - b[k]) <= rtol * max(1.0, abs(b[k])), k
    assert np.abs(a["sigma"] - b["sigma"]).max() <= rtol * max(1.0, np.abs(b["sigma"]).max())
    assert np.abs(a["rho"] - b["rho"]).max() <= rtol * np.abs(b["rho"]).max()


def _evaluate(sq, h, nd):
    sq.sq_moments(h)
    mu = sq.sq_fermi_level(h)
    rho, en, sig = sq.sq_density_energy_stress(h, mu, nd)
    p_a, e_pot = sq.sq_pressure(h, mu)
    return dict(en, mu=mu, rho=rho, sigma=sig, pressure_A=p_a, E_pot=e_pot, bounds=sq.sq_get_bounds(h))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("lanczos", [False, True])
def test_update_atoms_equals_fresh_setup(sq, precision, lanczos):
    mode = sq.SQ_FP64 if precision == "fp64" else sq.SQ_MIXED
    snaps = _trajectory()
    nd = int(np.prod(snaps[0]["n"]))
    bounds = None if lanczos else (-4.0, 40.0)
    h = sq.sq_setup(sq.Desc(snaps[0], mode, bounds=bounds))
    try:
        for s in snaps:
            if s is not snaps[0]:
                sq.sq_update_atoms(h, s["pos"], s["v_eff"])
                with pytest.raises(sq.SQError) as ei:       # the old moments are gone
                    sq.sq_fermi_level(h)
                assert ei.value.code == sq.SQ_ERR_STATE
            got = _evaluate(sq, h, nd)
            ref = sq.run(s, mode, bounds=bounds)
            if lanczos:
                assert got["bounds"] == pytest.approx(ref["bounds"], rel=1e-12, abs=1e-12)
            _close(got, ref, 1e-10 if precision == "fp64" else 1e-7)
    finally:
        sq.sq_destroy(h)


def test_served_trajectory_keeps_its_handle_resident(sq):
    snaps = _trajectory(n_snap=4, seed=9)
    refs = [sq.run(s, sq.SQ_MIXED, bounds=None) for s in snaps]
    srv = sq.Server(hbm_budget_bytes=8 << 30, max_inflight=2)
    try:
        descs = [sq.Desc(s, sq.SQ_MIXED, bounds=None) for s in snaps]
        for i, d in enumerate(descs):
            srv.submit(d, tag=i, traj=7)
        # a request without a trajectory in the mix
        extra = tiny_instance(seed=2, n=(4, 4, 4), h=(0.8, 0.8, 0.8), n_atoms=2, n_o=1, r_cut=0.9, n_pl=10)
        srv.submit(sq.Desc(extra, sq.SQ_MIXED, bounds=None), tag=100)
        got = []
        while len(got) < len(snaps) + 1:
            got += srv.poll(timeout_ms=500)
        assert srv.resident() == 1
    finally:
        srv.close()
    by_tag = {r["tag"]: r for r in got}
    assert all(r["status"] == 0 for r in got), [r["error"] for r in got]
    order = [r["tag"] for r in got if r["tag"] < 100]
    assert order == sorted(order)                     # a trajectory runs in submission order
    for i, ref in enumerate(refs):
        r = by_tag[i]
        for k in ("E_band", "E_s", "E_nl", "F", "N_check"):
            assert abs(r[k] - ref[k]) <= 1e-7 * max(1.0, abs(ref[k])), (i, k)
        assert np.abs(r["sigma"] - ref["sigma"]).max() <= 1e-7
    e = sq.run(extra, sq.SQ_MIXED, bounds=None)
    assert abs(by_tag[100]["F"] - e["F"]) <= 1e-7 * abs(e["F"])


def test_resident_handles_are_evicted_for_memory(sq):
    """A budget that holds one handle: a second trajectory evicts the idle first one."""
    a = tiny_instance(seed=3, n=(5, 5, 5), h=(0.7, 0.7, 0.7), n_atoms=2, n_o=2, r_cut=1.5, n_pl=10)
    b = tiny_instance(seed=4, n=(5, 5, 5), h=(0.7, 0.7, 0.7), n_atoms=2, n_o=2, r_cut=1.5, n_pl=10)
    da, db = sq.Desc(a, sq.SQ_FP64, bounds=(-4.0, 30.0)), sq.Desc(b, sq.SQ_FP64, bounds=(-4.0, 30.0))
    need = max(sq.sq_footprint_bytes(da), sq.sq_footprint_bytes(db))
    srv = sq.Server(hbm_budget_bytes=int(1.5 * need), max_inflight=1)
    try:
        srv.submit(da, tag=0, traj=1)
        got = []
        while len(got) < 1:
            got += srv.poll(timeout_ms=200)
        assert srv.resident() == 1
        srv.submit(db, tag=1, traj=2)
        while len(got) < 2:
            got += srv.poll(timeout_ms=200)
        assert srv.resident() == 1
    finally:
        srv.close()
    assert all(r["status"] == 0 for r in got)
    ra, rb = sq.run(a, sq.SQ_FP64, bounds=(-4.0, 30.0)), sq.run(b, sq.SQ_FP64, bounds=(-4.0, 30.0))
    got = {r["tag"]: r for r in got}
    assert abs(got[0]["F"] - ra["F"]) <= 1e-10 * abs(ra["F"])
    assert abs(got[1]["F"] - rb["F"]) <= 1e-10 * abs(rb["F"])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_keep_lists_for_fixed_atoms(sq, precision):
    """SCF-like use (Sec. 5): the atoms stay, V_eff changes between evaluations. With
    sq_keep_lists the sweep keeps the atom-image lists, brick records and W table of the
    positions (and the Lanczos bounds the lists of their sample tiles): a repeated evaluation,
    an evaluation after a new V_eff at the same positions, and one after the atoms move (which
    discards them) must each equal a fresh setup of that snapshot (FP64 1e-10, mixed 1e-7)."""
    mode = sq.SQ_FP64 if precision == "fp64" else sq.SQ_MIXED
    base = _trajectory(n_snap=2, seed=11)
    scf = dict(base[0])
    scf["v_eff"] = 1.2 * np.asarray(base[0]["v_eff"]) - 0.05      # same atoms, new potential
    nd = int(np.prod(base[0]["n"]))
    rtol = 1e-10 if precision == "fp64" else 1e-7
    h = sq.sq_setup(sq.Desc(base[0], mode, bounds=None))
    try:
        sq.sq_keep_lists(h, True)
        first = _evaluate(sq, h, nd)
        again = _evaluate(sq, h, nd)                                  # lists and W reused
        ref0 = sq.run(base[0], mode, bounds=None)
        _close(first, ref0, rtol)
        _close(again, ref0, rtol)
        sq.sq_update_atoms(h, scf["pos"], scf["v_eff"])
        _close(_evaluate(sq, h, nd), sq.run(scf, mode, bounds=None), rtol)
        sq.sq_update_atoms(h, base[1]["pos"], base[1]["v_eff"])      # moved: rebuilt
        _close(_evaluate(sq, h, nd), sq.run(base[1], mode, bounds=None), rtol)
    finally:
        sq.sq_destroy(h)
