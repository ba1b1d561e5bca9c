"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the timed region is the
slowest rank's, and the whole-job rate counts every rank's evaluations (independent
instances per rank, no data-path collective)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 1000.0 * (rank + 1)                      # rank 1 is the slow one
    m = bench.max_over_ranks(ms, dist, "cpu")
    out[rank] = (m, bench.whole_job_rate(world, 3, m))
    dist.destroy_process_group()


def test_max_over_ranks_and_rate_gloo():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        m, rate = out[r]
        assert m == pytest.approx(2000.0)
        assert rate == pytest.approx(2 * 3 / 2.0)


def test_single_process_passthrough():
    import bench
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5


def test_stencil_traffic_figure_is_tied_to_the_profiled_kernel_text():
    """bench.py reports the committed ncu DRAM traffic (per tile, times the tiles of a launch)
    only for the step-kernel source it was captured on (keyed by a hash of that text), else
    null; the committed figure is the current kernel's."""
    import json
    import os
    import bench
    path = os.path.join(os.path.dirname(os.path.abspath(bench.__file__)), "profiles", "stencil_traffic.json")
    t = json.load(open(path))
    assert bench.stencil_traffic(t["step_kernel_sha1"], 8000) == float(t["bytes_per_tile"]) * 8000
    assert bench.stencil_traffic("0" * 40, 8000) is None
    assert bench.step_kernel_hash() == t["step_kernel_sha1"]
