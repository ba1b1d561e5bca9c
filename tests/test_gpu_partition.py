"""The node partition of one instance (Sec. 4: the nodes are divided among processors and every
SQ sum is a sum over them) through the C ABI on one GPU: handles that own complementary tile
ranges, with their node sums R^j added (the allreduce of a multi-GPU run) and the Fermi level
taken from the sum, reproduce the whole instance; and the Fermi search reports
SQ_ERR_NO_BRACKET for node sums that cannot bracket N_e."""
import numpy as np
import pytest

from oracle import sq_oracle as orc
from workloads import make_instance, tiny_instance

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


def _parts(sq, inst, precision, bounds, count):
    nd = int(np.prod(inst["n"]))
    hs = [sq.sq_setup(sq.Desc(inst, precision, bounds=bounds, partition=(r, count))) for r in range(count)]
    try:
        for h in hs:
            sq.sq_moments(h)
        Rs = [sq.sq_node_sums(h, int(inst["n_pl"])) for h in hs]
        R = np.sum(Rs, axis=0)
        mus = [sq.sq_fermi_level_sums(h, R) for h in hs]
        tot = {k: 0.0 for k in sq.PART_SUM_KEYS}
        sig = np.zeros((3, 3))
        rho = np.zeros(nd)
        for h, mu in zip(hs, mus):
            r, en, s = sq.sq_density_energy_stress(h, mu, nd)
            p_a, e_pot = sq.sq_pressure(h, mu)
            en = dict(en, pressure_A=p_a, E_pot=e_pot)
            for k in tot:
                tot[k] += en[k]
            sig += s
            rho += r
        return mus, tot, sig, rho, Rs
    finally:
        for h in hs:
            sq.sq_destroy(h)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("count", [2, 3])
def test_parts_add_up_to_the_whole_instance(sq, precision, count):
    inst = make_instance(1)                     # 8 H, 12^3 nodes: 216 tiles
    mode = sq.SQ_FP64 if precision == "fp64" else sq.SQ_MIXED
    bounds = orc.lanczos_bounds(orc.Problem(inst))
    whole = sq.run(inst, mode, bounds=bounds)
    mus, tot, sig, rho, Rs = _parts(sq, inst, mode, bounds, count)
    # every part owns nodes, and the parts' node sums add up to the whole cell's
    assert all(R[0] > 0.0 for R in Rs)
    assert sum(R[0] for R in Rs) == pytest.approx(1728.0, rel=1e-12)
    for mu in mus:
        assert mu == pytest.approx(whole["mu"], rel=1e-12, abs=1e-12)
    for k in sq.PART_SUM_KEYS:
        assert tot[k] == pytest.approx(whole[k], rel=1e-12, abs=1e-12), k
    assert np.abs(sig - whole["sigma"]).max() <= 1e-12 * max(1.0, np.abs(whole["sigma"]).max())
    assert np.abs(rho - whole["rho"]).max() <= 1e-12 * np.abs(whole["rho"]).max()


def test_default_bounds_agree_across_parts(sq):
    """Device Lanczos bounds come from the same sample tiles on every part."""
    inst = tiny_instance(seed=3, n=(6, 5, 4), h=(0.7, 0.7, 0.7), n_atoms=2, n_o=2, r_cut=1.5, n_pl=10)
    b = []
    for r in range(2):
        h = sq.sq_setup(sq.Desc(inst, sq.SQ_FP64, partition=(r, 2)))
        try:
            sq.sq_moments(h)
            b.append(sq.sq_get_bounds(h))
        finally:
            sq.sq_destroy(h)
    assert b[0] == b[1]


def test_no_bracket_from_zero_node_sums(sq):
    inst = tiny_instance(seed=3, n=(6, 5, 4), h=(0.7, 0.7, 0.7), n_atoms=2, n_o=2, r_cut=1.5, n_pl=10)
    h = sq.sq_setup(sq.Desc(inst, sq.SQ_FP64, bounds=(-4.0, 30.0)))
    try:
        sq.sq_moments(h)
        with pytest.raises(sq.SQError) as ei:
            sq.sq_fermi_level_sums(h, np.zeros(11))
        assert ei.value.code == sq.SQ_ERR_NO_BRACKET
        with pytest.raises(sq.SQError) as ei:
            sq.sq_fermi_level_sums(h, np.full(11, np.nan))
        assert ei.value.code == sq.SQ_ERR_INVALID_ARG
        # the handle stays usable: the real node sums give the regular Fermi level
        mu = sq.sq_fermi_level_sums(h, sq.sq_node_sums(h, 10))
        assert mu == pytest.approx(sq.sq_fermi_level(h), abs=0.0)
    finally:
        sq.sq_destroy(h)


def test_invalid_partition_rejected(sq):
    inst = tiny_instance(seed=3, n=(6, 5, 4), h=(0.7, 0.7, 0.7), n_atoms=2, n_o=2, r_cut=1.5, n_pl=10)
    for part in ((2, 2), (-1, 2), (0, -1)):
        with pytest.raises(sq.SQError) as ei:
            sq.sq_setup(sq.Desc(inst, sq.SQ_FP64, bounds=(-4.0, 30.0), partition=part))
        assert ei.value.code == sq.SQ_ERR_INVALID_ARG
