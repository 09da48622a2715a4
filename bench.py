#!/usr/bin/env python
"""Throughput of the MacLABSWE FP32 step (Zhou, arXiv:1902.02999, Section 3)
on one GB300, printed as one JSON line.

Workload: channel flow over a seeded Gaussian bump, 8192 x 2048 nodes, FP32
perturbation storage, inflow discharge and outflow depth as Dirichlet
columns, free-slip side walls, Chezy friction (inputs.bump_channel, seed 0).
A step is one MacLABSWE time step over the whole grid (fused step kernel +
Dirichlet kernel).  The state (2 x 3 x 67 MB + 67 MB depth + 17 MB types)
is far larger than the 129 MB L2, so no flush is needed between steps.

    python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

With --gpus N > 1 (launched by torch.distributed.run) every rank advances
its own replica of the workload (the path is run as independent replicas);
value = nodes x steps summed over ranks / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("MLUPS & % of HBM roofline (FP32 step); wall time to residual 1e-8, "
          "warm-start vs plain")
BYTES_PER_NODE = {"f32": 29, "f64": 57}   # read eta,u,v,D + type, write eta,u,v
HBM_NOMINAL_GBS = 7900.0                   # GB300 HBM3e, nominal
# FP64 arithmetic of one node update, multiply-add counted as two: the
# source quantities (53, with the friction term) and the gather / update (67),
# plus one square root and one reciprocal
F64_FLOPS_PER_NODE = 120
F64_NOMINAL_TFLOPS = 1.25                  # GB300 dense FP64, nominal (the bench also measures it)
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0
PROFILE_JSON = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
# step-kernel codes of the library (maclab_step_kernel)
KERNEL_SYMBOL = {0: "step_tile_kernel<%s>", 1: "step_fast_kernel<%s>", 2: "step_tile_tma_kernel (%s)",
                 3: "step_march_kernel<%s>"}
KERNEL_LABEL = {0: "tile 64x16", 1: "warp strip", 2: "TMA-staged tile 64x16, persistent",
                3: "row march, 64-column strip blocks"}


def kernel_source_hash() -> str:
    """Hash of the device code the ncu counters describe (the step kernels'
    headers, in this order)."""
    h = hashlib.sha256()
    for name in ("maclab_kernels.cuh", "maclab_march.cuh"):
        with open(os.path.join(ROOT, "paper_1902_02999_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        for k in ("hbm_gbs", "hbm_GBs", "hbm_copy_gbs"):
            if k in d:
                return float(d[k]), "measured"
    except (OSError, ValueError):
        pass
    return FALLBACK_HBM_GBS, "fallback"


def bf16_peak():
    """Dense bf16 tensor rate (TFLOP/s) of this GPU timed alone (burst)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        if "bf16_tflops" in d:
            return float(d["bf16_tflops"]), "measured"
    except (OSError, ValueError):
        pass
    return FALLBACK_BF16_TFLOPS, "fallback"


def traffic_per_launch(precision, workload, kernel):
    try:
        with open(PROFILE_JSON) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    if d.get("source_sha256") != kernel_source_hash() or d.get("workload") != workload or \
            d.get("precision") != precision or d.get("kernel", "").split("<")[0] != kernel:
        return None
    return d.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.lines = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self):
        return time.time()

    def stop(self, t0, t1):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [r for (t, r) in self.lines if t0 - 0.25 <= t <= t1 + 0.25] or \
            [r for (_, r) in self.lines]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            f = [x.strip() for x in r.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for name, val in zip(names, f[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x, dist_mod, device):
    """The largest x over the ranks of the process group (x without one):
    the job's time is its slowest rank's."""
    if dist_mod is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist_mod.all_reduce(t, op=dist_mod.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(world, nodes, steps, ms):
    """Node updates of all ranks (each runs its own replica of `nodes`) per
    second of the slowest rank, in millions."""
    return world * nodes * steps / (ms / 1e3) / 1e6


def host_cores() -> int:
    """Threads the OpenMP oracle uses: OMP_NUM_THREADS, else every core."""
    try:
        return int(os.environ["OMP_NUM_THREADS"])
    except (KeyError, ValueError):
        return os.cpu_count() or 1


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as fh:
            info = fh.read()
    except OSError:
        return "unknown"
    for key in ("model name", "Model", "CPU part"):
        for line in info.splitlines():
            if line.startswith(key):
                return line.split(":", 1)[1].strip() + ("" if key == "model name" else " (%s)" % key)
    return "unknown"


def cpu_baseline(case, max_seconds=20.0):
    """The oracle as it stands, built with OpenMP (the rows of a step over
    every host core, the arithmetic per node unchanged), timed on full-grid
    steps of the workload for about 10-20 s."""
    import oracle
    oracle.build_omp()
    state = oracle.run_threads(case, 1)                 # warm: the build, page faults
    t0 = time.perf_counter()
    state = oracle.run_threads(case, 1, state, n0=1)
    one = time.perf_counter() - t0
    steps = max(1, min(50, int(max_seconds / max(one, 1e-3)) - 1))
    t0 = time.perf_counter()
    oracle.run_threads(case, steps, state, n0=2)
    el = time.perf_counter() - t0
    return {"value": case.nodes * steps / el / 1e6, "unit": "MLUPS", "cores": host_cores(), "kind": "oracle",
            "cpu": cpu_model(),
            "sample": "%d full-grid steps of the %dx%d workload (OpenMP over rows), %.1f s" % (
                steps, case.nx, case.ny, el)}


def run_reference(args, workload):
    """The oracle (OpenMP over rows, every host core) on samples of the
    workload: each step one oracle step of the full 8192 x 2048 channel, or
    of a horizontal slice of it when K + W full steps would not end within
    about 150 s."""
    import inputs
    import oracle
    oracle.build_omp()
    probe = inputs.bump_channel(args.nx, 64, seed=0)
    oracle.run_threads(probe, 1)
    t0 = time.perf_counter()
    oracle.run_threads(probe, 2)
    rate = probe.nodes * 2 / (time.perf_counter() - t0)   # node updates per second
    ny = int(150.0 * rate / max(1, args.steps + args.warmup) / args.nx)
    ny = max(8, min(args.ny, ny))
    case = inputs.bump_channel(args.nx, ny, seed=0) if ny < args.ny else inputs.bump_channel(args.nx, args.ny, seed=0)
    state = oracle.run_threads(case, args.warmup) if args.warmup else None
    t0 = time.perf_counter()
    oracle.run_threads(case, args.steps, state, n0=args.warmup)
    el = time.perf_counter() - t0
    value = case.nodes * args.steps / el / 1e6
    sample = ("each step: one oracle step of the full %dx%d workload" % (case.nx, case.ny) if ny >= args.ny else
              "each step: one oracle step of a %dx%d slice of the workload generator" % (case.nx, ny))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el * 1e3 / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload, "sample_nodes": case.nodes, "same_config": ny >= args.ny},
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": host_cores(), "kind": "oracle",
                             "cpu": cpu_model(), "sample": sample},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--nx", type=int, default=8192)
    ap.add_argument("--ny", type=int, default=2048)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--tile-rows", type=int, default=0)
    ap.add_argument("--kernel", default="default", choices=["default", "tile", "strip", "tma", "march"],
                    help="step kernel of the main leg (default: the library's choice)")
    ap.add_argument("--no-extra", action="store_true", help="skip the extra legs (steady state, FP64, batch, warm start, temporal blocking, "
                         "distribution form); they run only with a single rank")
    ap.add_argument("--steady-max-steps", type=int, default=2_000_000)
    ap.add_argument("--f64-steps", type=int, default=300)
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--batch-steps", type=int, default=200)
    ap.add_argument("--batch-max-steps", type=int, default=200_000)
    ap.add_argument("--ws-train", type=int, default=4096, help="lakes the warm-start network trains on (0: skip)")
    ap.add_argument("--ws-epochs", type=int, default=20)
    ap.add_argument("--ws-test", type=int, default=16, help="unseen lakes timed from rest and from the proposal")
    args = ap.parse_args()
    workload = "bump_channel_%dx%d_%s" % (args.nx, args.ny, args.precision)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, workload)
        return

    import torch
    import inputs
    from paper_1902_02999_gb300 import Simulation

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    case = inputs.bump_channel(args.nx, args.ny, seed=0)
    sim = Simulation.from_case(case, precision=args.precision)
    if args.tile_rows:
        sim.set_tile_rows(args.tile_rows)
    tuned = None
    if args.kernel != "default":
        sim.set_step_kernel(args.kernel)
    else:
        # the library's autotuner picks the launch shape and the temporal
        # block depth on this grid (state unchanged)
        tuned = sim.autotune(40)
    stream = torch.cuda.current_stream()
    info = sim.info
    n_general = info["n_fluid"] - info["n_fast"] - info["n_dirichlet"]
    # the tile and row-march kernels update the nodes with a bounce-back link
    # themselves; the other step kernels leave them to a second launch
    launches_per_step = 1 + (n_general > 0 and info["step_kernel"] not in (0, 3)) + \
        (info["n_dirichlet"] > 0 and not info["dirichlet_fused"])

    sampler = ClockSampler(local)
    sim.step(max(args.warmup, 3))
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    t_wall0 = sampler.mark()
    sim.set_profiling(True)
    ev0.record(stream)
    sim.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    t_wall1 = sampler.mark()
    kernel_ms, kernel_launches = sim.get_profile()
    sim.set_profiling(False)
    ms = ev0.elapsed_time(ev1)
    clocks = sampler.stop(t_wall0, t_wall1)
    ms = max_over_ranks(ms, dist, "cuda")
    # the extra legs describe one GPU: they run in the single-rank line only
    # (under torchrun every rank would hold its GPU for minutes)
    extra = not args.no_extra and world == 1
    nodes = case.nodes
    value = whole_job_mlups(world, nodes, args.steps, ms)

    # roofline of the dominant kernel (the fused step kernel)
    avg_kernel_s = kernel_ms / 1e3 / max(1, kernel_launches)
    achieved = BYTES_PER_NODE[args.precision] * nodes / avg_kernel_s / 1e9
    peak, peak_src = hbm_peak()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_src,
                "frac_of_nominal_7900": achieved / HBM_NOMINAL_GBS,
                "kernel": KERNEL_SYMBOL[info["step_kernel"]] % ("float" if args.precision == "f32" else "double"),
                "dirichlet_fused": bool(info["dirichlet_fused"]),
                "bytes_per_node": BYTES_PER_NODE[args.precision],
                "kernel_ms_per_launch": avg_kernel_s * 1e3,
                "traffic": traffic_per_launch(args.precision, workload,
                                              KERNEL_SYMBOL[info["step_kernel"]].split("<")[0].split(" ")[0])}

    # end to end through the public API: pinned host state in, one step, state out
    N = nodes
    hp = [torch.empty(N, dtype=torch.float64, pin_memory=True).numpy() for _ in range(3)]
    hin = [torch.empty(N, dtype=torch.float64, pin_memory=True).numpy() for _ in range(3)]
    st = sim.get_state()
    for k in range(3):
        hin[k][:] = st[k].reshape(-1)
    for _ in range(max(1, min(args.warmup, 3))):  # untimed: first use of the host buffers
        sim.set_state(*hin)
        sim.step(1)
        sim.get_state(out=hp)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        sim.set_state(*hin)
        sim.step(1)
        sim.get_state(out=hp)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dist, "cuda")
    e2e = {"value": world * N * args.e2e_steps / e2e_s / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": 3 * 8 * N, "d2h_bytes_per_step": 3 * 8 * N,
           "steps": args.e2e_steps}

    # temporal blocking: the same workload with clean tiles advanced two
    # steps per launch (bitwise the same states); 29 B per node update are
    # still counted per step, so a fraction above 1 is possible in principle
    tblock = None
    if extra and args.precision == "f32":
        sim.set_temporal_block(2)
        sim.step(max(args.warmup, 3))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        tms = e0.elapsed_time(e1) / args.steps
        tb_peak, _ = hbm_peak()
        tblock = {"k": 2, "clean_tiles": sim.info["clean_tiles"], "ms_per_step": tms,
                  "mlups": nodes / (tms / 1e3) / 1e6,
                  "frac_of_hbm_roofline": BYTES_PER_NODE[args.precision] * nodes / (tms / 1e3) / 1e9 / tb_peak,
                  "note": "per step of the whole job: 29 B/node algorithmic bytes over the step time"}
        sim.set_temporal_block(1)

    # the eLABSWE distribution form (Eq. lb.1, tau = 0.8) against MacLABSWE
    # on the same grid made periodic along x and all fluid (the form has no
    # Dirichlet rule): bytes and time per node update
    dform = None
    if extra and args.precision == "f32":
        import numpy as np
        pc = inputs.bump_channel(args.nx, args.ny, seed=0)
        pc.mask = np.full_like(pc.mask, inputs.FLUID)
        pc.edges = (inputs.PERIODIC, inputs.PERIODIC, inputs.SPECULAR, inputs.SPECULAR)
        pc.bc = np.zeros_like(np.asarray(pc.bc, dtype=np.float64))
        ds = Simulation.from_case(pc, precision="f32")
        dform = {"workload": "bump_channel_%dx%d, periodic in x, all fluid" % (args.nx, args.ny)}
        n_dist = max(200, args.steps // 10)
        for label, tau, bpn in (("macroscopic", 1.0, 29), ("distribution_tau_0.8", 0.8, 89)):
            ds.set_relaxation(tau)
            ds.set_profiling(True)
            ds.step(20)
            ds.get_profile()
            ds.step(n_dist)
            kms, kl = ds.get_profile()
            ds.set_profiling(False)
            per = kms / max(1, kl)
            dform[label] = {"ms_per_step": per, "mlups": pc.nodes / (per / 1e3) / 1e6, "bytes_per_node": bpn,
                           "achieved_gbs": bpn * pc.nodes / (per / 1e3) / 1e9}
        ds.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(case)

    # the other half of the metric: wall time to a residual of 1e-8 for the
    # seeded 256 x 256 dish lake (plain method, FP32 storage)
    steady = None
    if extra:
        lake = inputs.dish_lake(256, seed=0)
        ls = Simulation.from_case(lake, precision="f32")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ok, nsteps, r = ls.run_to_steady(tol=1e-8, max_steps=args.steady_max_steps, check_every=1000)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        steady = {"workload": lake.name, "precision": "f32", "tol": 1e-8, "converged": ok,
                  "steps": nsteps, "residual": r, "wall_s": wall,
                  "mlups": lake.nodes * nsteps / wall / 1e6, "simulated_s": nsteps * lake.dt}
        ls.close()

    # Section 4.1 as the 400 x 3 FP64 strip over two tidal periods, against
    # the asymptotic solution (horizontal surface at the tide level of
    # Eq. veri-Ini-Bc.3r, h u = 0 at x = 1500 m): level error (paper: below
    # 0.005 %) and velocity error at four sample times
    tidal = None
    if extra:
        import numpy as np
        tc = inputs.tidal_strip(400, 3)
        ts = Simulation.from_case(tc, precision="f64")
        xs = np.arange(tc.nx) * tc.dx
        om = 4 * math.pi / 86400.0
        samples, n0 = [], 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for T in (10800.0, 32400.0, 54000.0, 75600.0, 86400.0):
            n = int(round(T / tc.dt))
            ts.step(n - n0)
            n0 = n
            h, u, _ = ts.get_state()
            t = n * tc.dt
            eta = 20.0 - 4.0 * math.sin(om * t + math.pi / 2)
            ua = (xs - inputs.TIDAL_LENGTH) * 4.0 * om * math.cos(om * t + math.pi / 2) / (eta - tc.zb[0])
            samples.append({"t_s": T, "level_rel_err": float(np.abs(h + tc.zb - eta).max() / eta),
                            "u_max_abs_err_mps": float(np.abs(u - ua).max())})
        torch.cuda.synchronize()
        twall = time.perf_counter() - t0
        tidal = {"workload": "tidal_strip_400x3_f64 (Section 4.1), two tidal periods (86,400 s)",
                 "steps": n0, "dt_s": tc.dt, "wall_s": twall, "steps_per_s": n0 / twall,
                 "paper_level_bound": 5e-5, "paper_times_s": [10800.0, 32400.0], "samples": samples,
                 "note": "velocity: the scheme carries a start-up seiche the asymptotic solution lacks"}
        ts.close()

    # the FP32 path's error against the FP64 oracle, per result: (a) the
    # benchmark's channel family after 1000 steps (a 1024 x 256 channel:
    # the full grid would take the host hours), (b) the seeded 256 x 256
    # dish lake's steady state at residual 1e-8 against the oracle's own
    # steady state (oracle built with OpenMP, on the host cores)
    f32_error = None
    if extra and args.precision == "f32" and rank == 0:
        import numpy as np
        import oracle

        def errs(case, got, want):
            live = case.mask != inputs.SOLID
            sp = max(np.hypot(want[1], want[2])[live].max(), 1e-30)
            return {"h": float(np.abs(got[0] - want[0])[live].max() / np.abs(want[0][live]).max()),
                    "u": float(np.abs(got[1] - want[1])[live].max() / sp),
                    "v": float(np.abs(got[2] - want[2])[live].max() / sp)}
        cs = inputs.bump_channel(1024, 256, seed=0)
        g = Simulation.from_case(cs, precision="f32")
        g.step(1000)
        f32_error = {"norm": "max-norm over non-solid nodes; h by max|h|, u and v by the largest oracle speed",
                     "channel_1024x256_1000_steps": errs(cs, g.get_state(), oracle.run_threads(cs, 1000))}
        g.close()
        lake = inputs.dish_lake(256, seed=0)
        g = Simulation.from_case(lake, precision="f32")
        ok32, n32, r32 = g.run_to_steady(tol=1e-8, max_steps=1_000_000, check_every=1000)
        s32 = g.get_state()
        g.close()
        t0 = time.perf_counter()
        st, n, r_o = None, 0, float("inf")
        while r_o > 1e-8 and time.perf_counter() - t0 < 180.0 and n < 1_000_000:
            prev = st if st is not None else (lake.h0, lake.u0, lake.v0)
            st = oracle.run_threads(lake, 1000, st, n0=n)
            n += 1000
            r_o = oracle.residual(lake, prev, st, interval=1000)[0]
        f32_error["dish_lake_256_steady_1e-8"] = dict(
            errs(lake, s32, st), fp32_steps=n32, fp32_residual=r32, oracle_steps=n, oracle_residual=r_o,
            oracle_converged=bool(r_o <= 1e-8), oracle_wall_s=time.perf_counter() - t0)

    # the FP64 variant of the channel step (timed, not the headline)
    f64 = None
    if extra and args.precision == "f32":
        s64 = Simulation.from_case(case, precision="f64")
        choice64 = s64.autotune(10)
        s64.step(20)
        torch.cuda.synchronize()
        s64.set_profiling(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s64.step(args.f64_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        k64, n64 = s64.get_profile()
        ms64 = e0.elapsed_time(e1) / args.f64_steps
        k64_s = k64 / max(1, n64) / 1e3
        from paper_1902_02999_gb300 import measure_fp64
        p64 = measure_fp64()        # this GPU's FP64 FMA rate, measured here
        a64 = F64_FLOPS_PER_NODE * nodes / k64_s / 1e12
        f64 = {"value": nodes / (ms64 / 1e3) / 1e6, "unit": "MLUPS", "ms_per_step": ms64,
               "kernel_ms_per_launch": k64_s * 1e3,
               "alu_roofline": {"bound": "alu", "flops_per_node": F64_FLOPS_PER_NODE,
                                "achieved": a64, "peak": p64, "unit": "TFLOP/s",
                                "peak_source": "measured (maclab_measure_fp64: independent FMA chains)",
                                "frac": a64 / p64, "nominal_tflops": F64_NOMINAL_TFLOPS,
                                "frac_of_nominal": a64 / F64_NOMINAL_TFLOPS},
               "achieved_gbs": BYTES_PER_NODE["f64"] * nodes / (k64 / max(1, n64) / 1e3) / 1e9,
               "bytes_per_node": BYTES_PER_NODE["f64"],
               "step_kernel": ("tile 64x16" if choice64 == 0 else "TMA-staged tile 64x16" if choice64 == 5
                               else "row march" if choice64 == 7 else "warp strip, %d rows" % (4 << choice64))}
        s64.close()

    # the batched ensemble: 512 uneven lakes and channels advanced together
    batched = None
    if extra and args.batch_count > 0:
        from paper_1902_02999_gb300 import Batch
        ens = inputs.ensemble(args.batch_count, seed=0)
        bt = Batch(ens, precision=args.precision)
        info_b = bt.info()
        bt.step(64)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bt.step(args.batch_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        bms = e0.elapsed_time(e1) / args.batch_steps
        bt.close()
        bt = Batch(ens, precision=args.precision)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, rr, secs = bt.run_to_steady(tol=1e-8, max_steps=args.batch_max_steps, check_every=1000)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        conv = st >= 0
        import numpy as np

        def pct(values, q, bound):
            """q-th percentile over every instance, an unconverged one counting
            as infinite: (value, None), or (None, lower bound) when the
            percentile falls on an unconverged instance"""
            p = np.percentile(np.where(conv, values, np.inf), q, method="higher")
            return (float(p), None) if np.isfinite(p) else (None, bound)
        stats = {}
        for q in (50, 99):
            stats["p%d_s" % q], lb_s = pct(secs, q, wall)
            stats["p%d_steps" % q], lb_n = pct(st.astype(float), q, float(args.batch_max_steps))
            if lb_s is not None:
                stats["p%d_s_at_least" % q], stats["p%d_steps_at_least" % q] = lb_s, lb_n
        batched = {"instances": info_b["count"], "nodes": info_b["nodes"], "tiles": info_b["tiles"],
                   "mlups": info_b["nodes"] / (bms / 1e3) / 1e6, "ms_per_step": bms,
                   "steady": dict({"tol": 1e-8, "check_every": 1000, "max_steps": args.batch_max_steps,
                                   "residual": "change per step over each 1000-step check interval",
                                   "converged": int(conv.sum()), "wall_s": wall,
                                   "percentiles_over": "all instances (unconverged count as infinite)",
                                   # even instances are lakes, odd ones channels
                                   "converged_lakes": int(conv[0::2].sum()), "lakes": int(conv[0::2].size),
                                   "converged_channels": int(conv[1::2].sum()),
                                   "channels": int(conv[1::2].size)}, **stats)}
        bt.close()
        # the batched form against the plain method on the same GPU: every
        # 16th instance run to steady once as one batch and once one handle
        # at a time; the same arithmetic stops each instance at the same step
        sample = ens[::16]
        bt = Batch(sample, precision=args.precision)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sb, _, _ = bt.run_to_steady(tol=1e-8, max_steps=args.batch_max_steps, check_every=1000)
        torch.cuda.synchronize()
        wall_b = time.perf_counter() - t0
        bt.close()
        wall_p, same = 0.0, 0
        for i, c in enumerate(sample):
            one = Simulation.from_case(c, precision=args.precision)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ok, n1, _ = one.run_to_steady(tol=1e-8, max_steps=args.batch_max_steps, check_every=1000)
            torch.cuda.synchronize()
            wall_p += time.perf_counter() - t0
            same += int((n1 if ok else -1) == int(sb[i]))
            one.close()
        batched["batch_vs_plain"] = {
            "sample": "every 16th instance (%d of %d)" % (len(sample), len(ens)),
            "converged": int((sb >= 0).sum()), "same_stopping_step": same,
            "wall_batch_s": wall_b, "wall_plain_one_by_one_s": wall_p, "speedup": wall_p / wall_b}

    # learned warm start: wall time to residual 1e-8 from rest vs from the
    # network's proposal on unseen seeded 256 x 256 dish lakes (both FP32
    # batches of the plain iteration on this GPU); the network trains here,
    # on steady states of the same solver
    warm = None
    if extra and args.ws_train > 0 and rank == 0:
        from paper_1902_02999_gb300 import warmstart as ws
        net = ws.WarmStartNet(max_batch=16)
        t0 = time.perf_counter()
        train_cases = [inputs.dish_lake(256, seed=1000 + k) for k in range(args.ws_train)]
        X, T, W, scale, data_steps = ws.make_dataset(net, train_cases, tol=1e-7)
        torch.cuda.synchronize()
        t_data = time.perf_counter() - t0
        t0 = time.perf_counter()
        losses = ws.train(net, X, T, W, epochs=args.ws_epochs, batch=16, lr=1e-3)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        del X, T, W
        res = ws.compare(net, [inputs.dish_lake(256, seed=k) for k in range(args.ws_test)], scale)
        warm = {"workload": "dish_lake_256 seeds 0..%d (unseen)" % (args.ws_test - 1), "tol": 1e-8,
                "accuracy": "headline: warm and plain runs stop by a residual rule (see headline.rule), both "
                            "errors against the fp64 steady state given; 'matched' stops the warm run by its "
                            "error against that reference (not available to a user; device time)",
                "network": {"params": net.nparam, "grid": "64x64 cells of 4x4 nodes", "channels": net.channels,
                            "blocks": len(net.dilations), "precision": "bf16 activations, fp32 accumulate"},
                "train": {"lakes": args.ws_train, "epochs": args.ws_epochs, "data_s": t_data,
                          "train_s": t_train, "loss_first": losses[0], "loss_last": losses[-1]},
                "error_reference": "fp64 plain iteration to residual 1e-11"}
        warm.update(ws.summary(res))
        net.close()
        kt = ws.time_kernels(batch=16, reps=20, paths=(0,))["path0"]
        pk, pk_src = bf16_peak()
        warm["network_kernels"] = {
            "batch": 16, "forward_ms": kt["forward_ms"], "train_step_ms": kt["train_step_ms"],
            "forward_tflops": kt["forward_tflops"], "train_tflops": kt["train_tflops"],
            "peak_tflops": pk, "peak_source": pk_src, "forward_frac": kt["forward_tflops"] / pk,
            "train_frac": kt["train_tflops"] / pk,
            "flops": "2 per multiply-add of the convolutions; a training step counts three times the forward"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "fluid_mlups": world * info["n_fluid"] * args.steps / (ms / 1e3) / 1e6,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": args.precision, "data": "synthetic",
                "config": {"workload": workload, "nodes": nodes,
                           "l2": "inputs larger than L2 (state %.0f MB), no flush" %
                                 (nodes * BYTES_PER_NODE[args.precision] / 1e6),
                           "parallelism": "replicas" if world > 1 else "single-gpu",
                           "step_kernel": KERNEL_LABEL[info["step_kernel"]],
                           "autotune_choice": tuned, "temporal_block": info["temporal_block"]},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "steady_state": steady, "tidal": tidal, "f32_error": f32_error, "f64": f64, "batched": batched, "warm_start": warm,
                "temporal_block": tblock, "distribution_form": dform,
                "gpu_launches": launches_per_step * args.steps, "clocks": clocks}
        print(json.dumps(line), flush=True)
    sim.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
