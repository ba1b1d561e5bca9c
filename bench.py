#!/usr/bin/env python
"""Benchmark of the infinite-cell Clenshaw-Curtis SQ density / energy / stress evaluation.

Workload: 64 H atoms in a 12 bohr periodic cube, h = 0.3 bohr (40^3 nodes), 12th-order
stencil (n_o = 6), Gaussian V_eff and s+p Kleinman-Bylander projectors, kT = 3.17 Ha,
R_cut = 4 bohr (27^3 region per node), n_pl = 60 (seeded synthetic input).

One step = one stress evaluation: Lanczos spectral bounds, the per-wave setup (atom-image
lists, projector weights), the Chebyshev sweep with all moments, the Fermi-level bisection
and the contraction into rho, energies and sigma - every row of the hot path.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
  python bench.py --impl reference    # the FP64 CPU oracle on the host cores

With N > 1 (torchrun, or --gpus N, which starts the N ranks itself) the instance is split
by the node partition: each rank sweeps an equal contiguous range of the node tiles, one NCCL
allreduce of the node sums R^j precedes the Fermi search and one of the energy / stress
partials follows the contraction. Strong scaling: value = whole-cell evaluations / max-rank time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "stress evals/s"
CONFIG_NAME = "64H_12bohr_40cube_no6_sp_rcut4_27cube_npl60_kT3.17"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--no-fp64-compare", dest="fp64_compare", action="store_false",
                    help="skip timing one FP64 evaluation (the plain FP64 GPU path) on the same input")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-nodes", type=int, default=416,
                    help="seeded node columns in the oracle sample of cpu_baseline")
    ap.add_argument("--cpu-nodes-per-step", type=int, default=64,
                    help="seeded node columns per step of --impl reference")
    ap.add_argument("--fp64-steps", type=int, default=3,
                    help="timed evaluations of the plain FP64 GPU path (after one warm-up)")
    ap.add_argument("--serve-requests", type=int, default=30,
                    help="requests in the served-stream measurement (0 disables it)")
    ap.add_argument("--serve-trajectories", type=int, default=10)
    ap.add_argument("--batch", type=int, default=8,
                    help="instances in the batched-snapshot measurement (0 disables it)")
    ap.add_argument("--no-large", dest="large", action="store_false",
                    help="skip the largest single-GPU configurations (216 H / 60^3, 512 H / 80^3)")
    ap.add_argument("--profile-case", action="store_true",
                    help="only run two sweeps of the small profiling case (16^3 cell at the 40^3 "
                         "workload's parameters and atom density) for a profiler capture; prints no bench line")
    return ap.parse_args()


def run_profile_case(args):
    """Two moment sweeps (device Lanczos bounds) of the small profiling case, nothing timed."""
    import torch
    from paper_2006_03697_gb300 import build
    build.build()
    from paper_2006_03697_gb300 import sq
    from workloads import make_profile_case
    prec = sq.SQ_MIXED if args.precision == "mixed" else sq.SQ_FP64
    h = sq.sq_setup(sq.Desc(make_profile_case(), prec, bounds=None))
    try:
        for _ in range(2):
            sq.sq_moments(h)
        mu = sq.sq_fermi_level(h)
        rho, en, sig = sq.sq_density_energy_stress(h, mu, 16 ** 3)
    finally:
        sq.sq_destroy(h)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": "profile_4H_16cube", "mu": mu, "N_check": en["N_check"]}))
    return 0


# ---------------------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def step_kernel_hash() -> str:
    """sha1 of the step kernel's source text (its device helpers and the kernel, through its
    end, plus sq_device.cuh): the committed traffic figure is valid for that text only."""
    csrc = os.path.join(ROOT, "paper_2006_03697_gb300", "csrc")
    src = open(os.path.join(csrc, "sq_sweep.cu")).read()
    start = src.index("template <typename Real> struct Coef;")
    end = src.index("__constant__ int c_kpairs", start)
    dev = open(os.path.join(csrc, "sq_device.cuh")).read()
    return hashlib.sha1((src[start:end] + dev).encode()).hexdigest()


def stencil_traffic(sweep_hash: str, tiles_per_launch: float):
    """Per-launch DRAM traffic of the stencil kernel: the committed ncu figure per tile (captured
    on a smaller case of the same per-tile footprint) times the tiles of an average launch, if it
    was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "stencil_traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
        if t.get("step_kernel_sha1") == sweep_hash:
            return float(t["bytes_per_tile"]) * tiles_per_launch
    except (OSError, KeyError, ValueError):
        pass
    return None


# ---------------------------------------------------------------------------- CPU oracle
_ORACLE = {}


def _oracle_init(inst, lo, hi):
    """Pool initializer: each worker builds the oracle's problem once (outside any timing)."""
    from oracle import sq_oracle as orc
    _ORACLE["orc"] = orc
    _ORACLE["prob"] = orc.Problem(inst)
    _ORACLE["bounds"] = (lo, hi)


def _oracle_nodes(nodes):
    orc, prob = _ORACLE["orc"], _ORACLE["prob"]
    lo, hi = _ORACLE["bounds"]
    for q in nodes:
        orc.node_moments(prob, prob.node_coords(q), lo, hi)
    return len(nodes)


class OracleTimer:
    """The FP64 CPU oracle as it stands, node column by node column on every host core.

    A spawn pool is started and each worker builds the problem before anything is timed; a
    timed sample is a fixed, seeded set of node columns (their per-node moments dominate the
    oracle's cost; the Fermi search and contraction are O(N_d n_pl) and not timed). The rate is
    extrapolated to whole evaluations: evals/s = (node columns/s) / N_d."""

    BOUNDS = (-6.0, 130.0)

    def __init__(self, inst):
        import multiprocessing as mp
        import numpy as np
        self.nd = int(np.prod(inst["n"]))
        self.n_pl = int(inst["n_pl"])
        self.cores = os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_init,
                                                 initargs=(inst,) + self.BOUNDS)
        self.pool.map(_oracle_nodes, [[] for _ in range(self.cores)])   # workers started and ready
        self.rng = np.random.Generator(np.random.PCG64(12345))

    def sample(self, n_nodes: int):
        nodes = self.rng.choice(self.nd, size=min(self.nd, n_nodes), replace=False).tolist()
        chunks = [nodes[i::self.cores] for i in range(self.cores)]
        t0 = time.perf_counter()
        self.pool.map(_oracle_nodes, [c for c in chunks if c])
        wall = time.perf_counter() - t0
        nodes_per_s = len(nodes) / wall
        return {"value": nodes_per_s / self.nd, "unit": METRIC, "cores": self.cores, "kind": "oracle",
                "sample": f"{len(nodes)} seeded node columns of {self.nd} (per-node moments, n_pl={self.n_pl}) in "
                          f"{wall:.1f} s on {self.cores} worker processes; scaled by N_d / sample = "
                          f"{self.nd / len(nodes):.0f}; Fermi search and contraction (O(N_d n_pl)) not timed",
                "nodes_per_s": nodes_per_s, "sample_nodes": len(nodes), "extrapolation": self.nd / len(nodes),
                "wall_s": wall}

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_oracle_rate(inst, n_nodes: int):
    """One bounded sample (n_nodes seeded node columns) of the oracle on all host cores."""
    timer = OracleTimer(inst)
    try:
        return timer.sample(n_nodes)
    finally:
        timer.close()


def serve_stream(sq, n_req: int, prec: int, n_traj: int = 10, max_inflight: int = 4, load: float = 0.7):
    """A served stream of quantum-MD snapshots with the size mix of the served workload: n_traj
    trajectories whose cells are drawn as the batched snapshots (32 ... 256 H at 0.0375 / bohr^3,
    kT in [1.6, 6.3], n_pl in [30, 80], R_cut in [3, 5]), 20 % of them (rounded) 512-atom,
    80^3-node cells; request i is the next snapshot of trajectory i mod n_traj (atoms moved by
    N(0, 0.05^2) bohr, V_eff with them), so 20 % of the requests are 512-atom cells, and keeps
    that trajectory's handle resident on the device (sq_server_submit_traj). Arrivals are Poisson
    at `load` x the saturated rate measured on the first round of requests. Reports p50 / p99
    latency (submit to result) and evals/s."""
    import numpy as np
    from workloads import gaussian_veff, make_batch, perturb_positions
    n_large = max(1, int(round(0.2 * n_traj)))
    base = make_batch(config=5, count=n_traj - n_large, atom_choices=(32, 64, 128, 256))
    base += make_batch(config=5, count=n_large, start=100, atom_choices=(512,))
    rng = np.random.Generator(np.random.PCG64(5000))
    state = [dict(b) for b in base]
    reqs = []
    for i in range(n_req):
        t = i % n_traj
        if i >= n_traj:
            s2 = dict(state[t])
            s2["pos"] = perturb_positions(rng, np.asarray(s2["pos"]), 0.05, s2["L"])
            s2["v_eff"] = gaussian_veff(s2["L"], s2["n"], s2["pos"])
            state[t] = s2
        reqs.append((t, sq.Desc(state[t], prec, bounds=None)))
    srv = sq.Server(hbm_budget_bytes=160 << 30, max_inflight=max_inflight)
    got = []
    try:
        # saturated rate: the first round (one request per trajectory) submitted at once
        t0 = time.perf_counter()
        for i in range(n_traj):
            srv.submit(reqs[i][1], tag=i, traj=reqs[i][0])
        while len(got) < n_traj:
            got += srv.poll(timeout_ms=200)
        sat = n_traj / (time.perf_counter() - t0)
        rate = load * sat
        gaps = rng.exponential(1.0 / rate, size=n_req)
        t1 = time.perf_counter()
        for i in range(n_traj, n_req):
            srv.submit(reqs[i][1], tag=i, traj=reqs[i][0])
            got += srv.poll(timeout_ms=0)
            time.sleep(float(gaps[i]))
        while len(got) < n_req:
            got += srv.poll(timeout_ms=200)
        wall = time.perf_counter() - t1
        resident = srv.resident()
    finally:
        srv.close()
    steady = [r for r in got if r["tag"] >= n_traj]
    lat = np.sort(np.array([r["latency_ms"] for r in steady]))
    sizes = [len(base[t]["pos"]) for t in range(n_traj)]
    return {"requests": n_req, "measured_requests": len(steady), "ok": all(r["status"] == 0 for r in got),
            "failed": [(int(r["status"]), r["error"]) for r in got if r["status"] != 0],
            "evals_per_s": len(steady) / wall, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "arrival_rate_per_s": rate, "saturated_evals_per_s": sat,
            "max_inflight": max_inflight, "trajectories": n_traj, "atoms_per_trajectory": sizes,
            "resident_handles_at_end": resident,
            "workload": f"served mix: {n_traj} trajectories of the batched snapshots (32-256 H, and {n_large} of "
                        "512-atom 80^3 cells: 20 % of the requests), "
                        "consecutive snapshots moved by N(0, 0.05^2) bohr with resident device state, Poisson "
                        f"arrivals at {load} x the saturated rate; the first round (one request per trajectory, "
                        "setup included) sets the rate and is not in the latency statistics"}


def batch_throughput(sq, prec: int, count: int = 8):
    """Uneven snapshots of the batched workload (32 ... 512-atom cells with their own grid, kT,
    n_pl and R_cut; one 256- and one 512-atom cell among them) evaluated by ONE CUDA graph
    (sq_batch_create captures every member's Lanczos bounds, sweep, Fermi level and
    contraction as a branch; sq_batch_run launches it): evaluations/s and region point-steps/s
    of the whole batch, timed on the second launch (the first one warms up)."""
    import numpy as np
    import torch
    from workloads import make_batch
    insts = make_batch(config=4, count=max(2, count - 2), atom_choices=(32, 64, 128))
    insts += make_batch(config=4, count=1, start=200, atom_choices=(256,))
    insts += make_batch(config=4, count=1, start=201, atom_choices=(512,))
    streams = [torch.cuda.Stream() for _ in insts]
    hs = [sq.sq_setup(sq.Desc(inst, prec, bounds=None, stream=st.cuda_stream)) for inst, st in zip(insts, streams)]
    point_steps = 0.0
    for inst in insts:
        m = np.floor(float(inst["r_cut"]) / (np.asarray(inst["L"]) / np.asarray(inst["n"])) + 1e-9)
        point_steps += float(np.prod(inst["n"])) * float(np.prod(2 * m + 1)) * float(inst["n_pl"])
    batch = None
    try:
        batch = sq.Batch(hs)
        batch.run()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mu, en, sig = batch.run()
        wall = time.perf_counter() - t0
    finally:
        if batch is not None:
            batch.close()
        for h in hs:
            sq.sq_destroy(h)
    return {"instances": len(insts), "graph_launches_timed": 1, "evals_per_s": len(insts) / wall, "wall_s": wall,
            "point_steps_per_s": point_steps / wall,
            "atoms": [int(len(i["pos"])) for i in insts], "n_pl": [int(i["n_pl"]) for i in insts],
            "ok": bool(all(abs(e["N_check"] - i["n_e"]) <= 1e-8 * i["n_e"] for e, i in zip(en, insts))),
            "workload": "uneven snapshots of the batched config (32-512 H at 0.0375 / bohr^3, h = 0.3, kT in "
                        "[1.6, 6.3], n_pl in [30, 80], R_cut in [3, 5]), device Lanczos bounds, one CUDA graph"}


def large_configs(sq, prec: int):
    """The largest single-GPU workloads, one warm-up and one timed evaluation each (setup outside,
    device Lanczos bounds inside the timed evaluation): 216 H in an 18 bohr cube (60^3 nodes,
    27^3 regions, n_pl = 60) and the largest batched snapshot (512 H, 80^3 nodes)."""
    import numpy as np
    import torch
    from workloads import make_batch, make_instance
    out = {}
    cases = (("216H_18bohr_60cube_no6_sp_rcut4_npl60", make_instance(3)),
             ("512H_24bohr_80cube_batched_snapshot", make_batch(4, count=1, atom_choices=(512,))[0]))
    for name, inst in cases:
        st = torch.cuda.Stream()
        h = sq.sq_setup(sq.Desc(inst, prec, bounds=None, stream=st.cuda_stream))
        nd = int(np.prod(inst["n"]))
        try:
            def ev():
                sq.sq_moments(h)
                mu = sq.sq_fermi_level(h)
                return sq.sq_density_energy_stress(h, mu, None)
            ev()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, en, _ = ev()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
        finally:
            sq.sq_destroy(h)
        m = np.floor(float(inst["r_cut"]) / (np.asarray(inst["L"]) / np.asarray(inst["n"])) + 1e-9)
        ps = float(nd) * float(np.prod(2 * m + 1)) * float(inst["n_pl"])
        out[name] = {"s_per_eval": dt, "evals_per_s": 1.0 / dt, "point_steps_per_s": ps / dt,
                     "nodes": nd, "region": [int(2 * x + 1) for x in m], "n_pl": int(inst["n_pl"]),
                     "N_check": en["N_check"], "n_e": float(inst["n_e"])}
    return out


def run_reference(args):
    """The oracle as the reference arm: W untimed samples, then K timed samples of
    --cpu-nodes-per-step seeded node columns each (the pool is started before the warm-up)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from workloads import make_instance
    inst = make_instance(args.config)
    timer = OracleTimer(inst)
    try:
        for _ in range(args.warmup):
            timer.sample(timer.cores)
        vals = []
        t0 = time.perf_counter()
        for _ in range(args.steps):
            vals.append(timer.sample(args.cpu_nodes_per_step))
        wall = time.perf_counter() - t0
    finally:
        timer.close()
    nodes = sum(x["sample_nodes"] for x in vals)
    node_s = sum(x["wall_s"] for x in vals)
    v = nodes / node_s / timer.nd
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": args.gpus,
        # a step is one timed sample (its measured duration); value extrapolates samples to evaluations
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * node_s / max(1, args.steps),
        "ms_per_evaluation_extrapolated": 1000.0 / v, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": CONFIG_NAME, "flush_l2": "working set > L2 (CPU run)"},
        "cpu_baseline": {"value": v, "unit": METRIC, "cores": timer.cores, "kind": "oracle",
                         "sample": f"{args.steps} samples of {args.cpu_nodes_per_step} seeded node columns of "
                                   f"{timer.nd} ({nodes} in {node_s:.1f} s on {timer.cores} worker processes), "
                                   f"scaled by N_d; Fermi search and contraction not timed",
                         "nodes_per_s": nodes / node_s},
        "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": wall,
    }
    print(json.dumps(line), flush=True)
    return 0


def max_over_ranks(x: float, dist, device: str) -> float:
    """The slowest rank's value (max-reduction); x itself without a process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: int, max_ms: float) -> float:
    """Units processed by all ranks per second of the slowest rank (weak scaling)."""
    return world * units_per_rank / (max_ms / 1000.0)


# ---------------------------------------------------------------------------- GPU arm
def run_ours(args):
    import numpy as np
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2006_03697_gb300 import build
    build.build()
    from paper_2006_03697_gb300 import sq
    from workloads import make_instance

    # one instance; with N ranks each sweeps its part of the node tiles (the node partition)
    inst = make_instance(args.config)
    nd = int(np.prod(inst["n"]))
    n_pl = int(inst["n_pl"])
    prec = sq.SQ_MIXED if args.precision == "mixed" else sq.SQ_FP64
    stream = torch.cuda.Stream()
    sptr = stream.cuda_stream
    part = (rank, world) if world > 1 else None
    desc = sq.Desc(inst, prec, bounds=None, stream=sptr, partition=part)
    h = sq.sq_setup(desc)
    rho_dev = torch.empty(nd, dtype=torch.float64, device="cuda")
    sig_dev = torch.empty(9, dtype=torch.float64, device="cuda")

    def allreduce(vec):
        """Sum of a float64 host vector over the ranks (NCCL)."""
        t = torch.from_numpy(np.ascontiguousarray(vec, dtype=np.float64)).cuda()
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return t.cpu().numpy()

    def finish(hh, mu, en):
        """Whole-cell results of a partitioned handle: the parts' sums (one allreduce)."""
        stream.synchronize()   # sigma_dev is written on the library stream
        keys = ("E_band", "E_s", "E_nl", "N_check")
        tot = allreduce(np.concatenate([[en[k] for k in keys], sig_dev.cpu().numpy()]))
        out = {k: float(tot[i]) for i, k in enumerate(keys)}
        out["F"] = out["E_band"] + out["E_s"]
        out["mu"] = mu
        sig_dev.copy_(torch.from_numpy(tot[len(keys):]))
        return out

    def step():
        sq.sq_moments(h)
        if dist is None:
            mu = sq.sq_fermi_level(h)
            return sq.sq_density_energy_stress_dev(h, mu, rho_dev.data_ptr(), sig_dev.data_ptr(), energies=True)
        mu = sq.sq_fermi_level_sums(h, allreduce(sq.sq_node_sums(h, n_pl)))   # exchange of R^j
        en = sq.sq_density_energy_stress_dev(h, mu, rho_dev.data_ptr(), sig_dev.data_ptr(), energies=True)
        return finish(h, mu, en)

    en = step()
    # autotuner: warps per step block and tiles per wave for this geometry (cached per shape),
    # chosen before the warm-up and the timed region
    tune_key, tune_choice, _ = sq.autotune_step(h, inst, prec, partition=part)
    for _ in range(max(0, args.warmup - 1)):
        en = step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    l0 = sq.sq_kernel_launches(h)
    sq.sq_kernel_timing(h, True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        en = step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = sq.sq_kernel_launches(h) - l0
    kern = {}
    for name, kid in (("stencil", sq.SQ_K_STENCIL), ("project", sq.SQ_K_PROJECT), ("moments", sq.SQ_K_MOMENTS)):
        n, kms, kb = sq.sq_kernel_timing_read(h, kid)
        kern[name] = {"launches": n, "ms": kms, "bytes": kb}
    sq.sq_kernel_timing(h, False)
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(ms, dist, "cuda")
    ms_per_step = ms / args.steps
    # one instance per step whatever N is (strong scaling): evaluations of the whole cell / s
    value = whole_job_rate(1, args.steps, ms)

    # e2e: the public C ABI from host buffers, setup copies and host outputs inside the region
    rho_h = np.zeros(nd)
    h2d = desc.v.nbytes + desc.pos.nbytes + desc.species.nbytes + desc.offs.nbytes
    d2h = rho_h.nbytes + 9 * 8 + 6 * 8
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        hh = sq.sq_setup(desc)
        sq.sq_moments(hh)
        if dist is None:
            mu = sq.sq_fermi_level(hh)
        else:
            mu = sq.sq_fermi_level_sums(hh, allreduce(sq.sq_node_sums(hh, n_pl)))
        rho_h, en2, sig_h = sq.sq_density_energy_stress(hh, mu, nd)
        if dist is not None:
            allreduce(np.concatenate([[en2[k] for k in ("E_band", "E_s", "E_nl", "N_check")], sig_h.reshape(9)]))
        sq.sq_destroy(hh)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dist, "cuda")
    e2e = {"value": args.steps / e2e_s, "unit": METRIC, "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h)}

    # roofline of the dominant sweep kernel
    hbm, peak_kind = peaks()
    dom = max(kern, key=lambda k: kern[k]["ms"])
    st = kern["stencil"]
    sweep_hash = step_kernel_hash()
    achieved = (st["bytes"] / st["launches"]) / (st["ms"] / st["launches"] / 1000.0) / 1e9 if st["launches"] else 0.0
    # tiles of an average step launch: this rank's tiles over the waves (n_pl + 1 launches per wave
    # and evaluation)
    tiles_part = int(np.prod((np.asarray(inst["n"], dtype=np.int64) + 1) // 2))
    if part is not None:
        tiles_part = tiles_part * (part[0] + 1) // part[1] - tiles_part * part[0] // part[1]
    nwaves = max(1, round(st["launches"] / max(1, args.steps * (n_pl + 1))))
    roof = {"kernel": "k_stencil", "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": stencil_traffic(sweep_hash, tiles_part / nwaves),
            "tiles_per_launch": tiles_part / nwaves,
            "peak_source": peak_kind, "dominant_kernel": dom,
            "algo_bytes_per_launch": st["bytes"] / max(1, st["launches"]),
            "avg_launch_ms": st["ms"] / max(1, st["launches"])}

    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f32" if prec == sq.SQ_MIXED else "f64", "data": "synthetic",
        "config": {"workload": CONFIG_NAME, "precision": args.precision, "bounds": "lanczos (device, per step)",
                   "parallelism": f"node partition over {world} GPU(s): tile ranges, allreduce of R^j and of the "
                                  "energy / stress partials" if world > 1 else "1 GPU",
                   "node_columns_per_step": nd,
                   "flush_l2": f"no flush: device working set {sq.sq_footprint_bytes(desc) / 1e9:.1f} GB > L2"},
        "node_columns_per_s": value * nd,
        "autotune": {"key": tune_key, **tune_choice},
        "clocks": clk, "gpu_launches": int(launches), "e2e": e2e, "roofline": roof,
        "kernels": kern, "energies": {k: en[k] for k in ("E_band", "E_s", "E_nl", "F", "N_check", "mu")},
        "sigma": sig_dev.cpu().numpy().reshape(3, 3).tolist(),
        "pressure_app_a": (sq.sq_pressure(h, en["mu"])[0] if dist is None
                           else float(allreduce(np.array([sq.sq_pressure(h, en["mu"])[0]]))[0])),
    }
    if args.fp64_compare and rank == 0 and world == 1:
        # the plain FP64 GPU path (same library, SQ_FP64) on the same input: one untimed warm-up
        # evaluation, then --fp64-steps timed ones
        d64 = sq.Desc(inst, sq.SQ_FP64, bounds=None, stream=sptr)
        h64 = sq.sq_setup(d64)

        def step64():
            sq.sq_moments(h64)
            mu64 = sq.sq_fermi_level(h64)
            return sq.sq_density_energy_stress_dev(h64, mu64, rho_dev.data_ptr(), sig_dev.data_ptr(), energies=True)

        step64()
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(args.fp64_steps):
            en64 = step64()
        a1.record(stream)
        torch.cuda.synchronize()
        f64ms = a0.elapsed_time(a1) / args.fp64_steps
        sig64 = sig_dev.cpu().numpy().reshape(3, 3)
        line["fp64_gpu"] = {"value": 1000.0 / f64ms, "unit": METRIC, "ms_per_step": f64ms, "steps": args.fp64_steps,
                            "warmup": 1, "F": en64["F"], "speedup_of_value": value / (1000.0 / f64ms),
                            "mixed_vs_fp64": {
                                "F_rel": abs(en["F"] - en64["F"]) / abs(en64["F"]),
                                "E_band_rel": abs(en["E_band"] - en64["E_band"]) / abs(en64["E_band"]),
                                "E_nl_rel": abs(en["E_nl"] - en64["E_nl"]) / abs(en64["E_nl"]),
                                "sigma_abs_max": float(np.abs(np.asarray(line["sigma"]) - sig64).max())}}
        sq.sq_destroy(h64)
    sq.sq_destroy(h)
    if rank == 0 and world == 1 and args.serve_requests > 0:
        line["serving"] = serve_stream(sq, args.serve_requests, prec, n_traj=args.serve_trajectories)
    if rank == 0 and world == 1 and args.large:
        line["large_configs"] = large_configs(sq, prec)
    if rank == 0 and world == 1 and args.batch > 0:
        line["batch"] = batch_throughput(sq, prec, count=args.batch)
        m = np.floor(float(inst["r_cut"]) / (np.asarray(inst["L"]) / np.asarray(inst["n"])) + 1e-9)
        line["batch"]["single_instance_point_steps_per_s"] = (float(nd) * float(np.prod(2 * m + 1)) *
                                                              float(inst["n_pl"]) * value)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_rate(inst, args.cpu_nodes)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def launch_ranks(args) -> int:
    """--gpus N > 1 outside torchrun: start N ranks of this script on this node (127.0.0.1)."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def main():
    args = parse()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ and not args.profile_case:
        return launch_ranks(args)
    if args.profile_case:
        return run_profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
