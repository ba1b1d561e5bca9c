"""The node partition of one instance across ranks (Sec. 4: the nodes of K_Omega are divided
among processors and every SQ sum is a sum over them), on CPU with gloo, world size 2.

Each rank takes the node set the library's tile-range rule gives it (sq.partition_nodes), forms
the FP64 oracle's moments of those nodes only, and runs the exchange steps of the partitioned
path: one allreduce of the node sums R^j before the Fermi search, one of the partial energies,
pressure and sigma after the contraction. The result must equal the whole-cell oracle."""
import datetime
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import sq_oracle as orc
from paper_2006_03697_gb300 import sq
from workloads import tiny_instance

CASE = dict(seed=21, n=(5, 4, 6), h=(0.7, 0.7, 0.7), n_atoms=2, n_o=2, r_cut=1.5, n_pl=12)
BOUNDS = (-4.0, 30.0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _allreduce(x):
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.numpy()


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    inst = tiny_instance(**CASE)
    prob = orc.Problem(inst)
    lo, hi = BOUNDS
    nodes = sq.partition_nodes(inst["n"], rank, world)
    mom = np.zeros((prob.Nd, prob.n_pl + 1, orc.N_MOM))
    if len(nodes):
        mom[nodes] = orc.all_moments(prob, lo, hi, nodes=nodes)
    R = _allreduce(mom[:, :, 0].sum(axis=0))                    # exchange 1: n_pl + 1 doubles
    mu = orc.fermi_bisect(R, prob.n_e, prob.kT, lo, hi, prob.M)
    part = orc.contract(prob, mom, mu, lo, hi)
    keys = sq.PART_SUM_KEYS
    vec = np.concatenate([[part[k] for k in keys], part["sigma"].reshape(9)])
    tot = _allreduce(vec)                                        # exchange 2: 15 doubles
    out[rank] = {"mu": mu, "tot": tot.tolist(), "nodes": nodes.tolist(), "rho": part["rho"].tolist()}
    dist.destroy_process_group()


def test_partition_rule_covers_every_node_once():
    for n in ((5, 4, 6), (1, 3, 2), (8, 8, 8), (7, 1, 1)):
        nd = int(np.prod(n))
        for count in (1, 2, 3, 5, 64):
            got = np.concatenate([sq.partition_nodes(n, r, count) for r in range(count)])
            assert np.array_equal(np.sort(got), np.arange(nd)), (n, count)
            ranges = [sq.partition_tiles(n, r, count) for r in range(count)]
            assert ranges[0][0] == 0 and all(ranges[i][1] == ranges[i + 1][0] for i in range(count - 1))


def test_partitioned_sums_equal_the_whole_cell_gloo():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(600)
        assert p.exitcode == 0
    inst = tiny_instance(**CASE)
    ref = orc.run(inst, bounds=BOUNDS)
    nodes = [set(out[r]["nodes"]) for r in range(world)]
    assert not (nodes[0] & nodes[1]) and len(nodes[0] | nodes[1]) == int(np.prod(inst["n"]))
    for r in range(world):
        assert out[r]["mu"] == pytest.approx(ref["mu"], rel=1e-12, abs=1e-12)
        tot = np.asarray(out[r]["tot"])
        for i, k in enumerate(sq.PART_SUM_KEYS):
            assert tot[i] == pytest.approx(ref[k], rel=1e-11, abs=1e-12), k
        assert np.allclose(tot[len(sq.PART_SUM_KEYS):].reshape(3, 3), ref["sigma"], rtol=1e-11, atol=1e-14)
    rho = np.asarray(out[0]["rho"]) + np.asarray(out[1]["rho"])
    assert np.allclose(rho, ref["rho"], rtol=1e-12, atol=1e-14)


def _worker_dies(rank, world, port, out):
    """Rank 1 fails before the exchange of the node sums (a sweep that raised); rank 0's
    allreduce must end with an error within the process group's timeout, not hang."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    if rank == 1:
        os._exit(3)                                   # leaves between steps, nothing in flight
    inst = tiny_instance(**CASE)
    prob = orc.Problem(inst)
    nodes = sq.partition_nodes(inst["n"], rank, world)
    mom = np.zeros((prob.Nd, prob.n_pl + 1, orc.N_MOM))
    mom[nodes] = orc.all_moments(prob, *BOUNDS, nodes=nodes)
    try:
        _allreduce(mom[:, :, 0].sum(axis=0))
        out[rank] = "no error"
    except Exception as e:                            # the failed peer is reported, not waited for
        out[rank] = "error: " + type(e).__name__
    os._exit(0)


def test_failed_rank_is_reported_to_its_peer_gloo():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker_dies, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert procs[1].exitcode == 3
    assert procs[0].exitcode == 0
    assert out[0].startswith("error"), out[0]
