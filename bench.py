"""Benchmark of the HMC hot path on GB300.

One step = one full molecular-dynamics trajectory on the 102x102 honeycomb
torus with nt = 64 (1,331,712 space-time sites): pseudofermion creation for
3 Hasenbusch masses (0.1, 0.5, 2.0), the nested Omelyan integrator with
N_MD = 30 and time-scale ratios (6, 2, 2), forces from mixed-precision FGMRES
solves (FP32 CG preconditioner, FP64 outer) at relative residual 1e-10, and
the final action solves at 1e-12. Every M M^dagger application, CG and
FGMRES iteration, force and MD update of the path runs in it.

value = sites x (M M^dagger applications in the step) / step time, in Gsite/s:
the operator throughput the whole path sustains. Inputs are resident in HBM
before timing; L2 is flushed (256 MB write) between steps, outside the per-step
CUDA-event windows. Also reported: FP64 CG vs mixed FGMRES time-to-solution on
the same lattice, the roofline of the dominant kernel, an end-to-end figure with
host buffers, and the CPU oracle timed on the host.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank runs its own independent trajectories
(replicas; no data-path collective) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gsite/s of M·M† apply (% HBM peak); solve ms @res 1e-10, mixed+batched vs FP64"
UNIT = "Gsite/s"
WORKLOAD = ("102x102 honeycomb torus, nt=64 (1,331,712 sites), kappa=1, U=3.8, beta=12: one "
            "nested-Omelyan MD trajectory (N_MD=30, N_i=(6,2,2)) with 3 Hasenbusch masses "
            "(0.1,0.5,2.0), mixed FP32/FP64 FGMRES forces at 1e-10")
WORKLOAD_A = "FGMRES inner tolerance factor a = {a}"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            if os.path.exists(self.path):
                os.unlink(self.path)
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            lines = f.readlines()
        os.unlink(self.path)
        return self.summarise(lines)

    @staticmethod
    def summarise(lines):
        """Median SM clock, the highest maximum clock, the throttle reasons seen
        active in any sample, and the peak power, from nvidia-smi CSV lines in
        the order of FIELDS (no header, no units)."""
        rows = []
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        pw = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


def cpu_oracle_apply(seconds: float):
    """The oracle's M M^dagger on the same lattice, repeated for about `seconds`."""
    import workloads as W
    from oracle import fermion
    from oracle.lattice import Lattice
    w = W.workload("L102x102x64")
    lat = Lattice.from_params(w.lat)
    reps = 0
    t0 = time.perf_counter()
    while True:
        fermion.apply_MMdag(lat, w.phi, 0.0, w.b)
        reps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return lat.N * reps / dt / 1e9, reps, dt


def cpu_oracle_cg(iters: int):
    """The oracle's FP64 CG (the same algorithm as the library's FP64 CG) on
    the same lattice and m_s = 0 system, stopped after `iters` iterations:
    milliseconds per iteration."""
    import workloads as W
    from oracle import fermion, solvers
    from oracle.lattice import Lattice
    w = W.workload("L102x102x64")
    lat = Lattice.from_params(w.lat)
    t0 = time.perf_counter()
    res = solvers.cg(lambda v: fermion.apply_MMdag(lat, w.phi, 0.0, v), w.b, tol=1e-10, maxit=iters)
    dt = time.perf_counter() - t0
    return 1e3 * dt / max(res.iters, 1), res.iters


def _c3_oracle_job(q):
    """(In a spawned process) the oracle's FP64 CG on the 36x36x64 system
    (m_s = 0) to 1e-12, timed, on the last host core only."""
    if hasattr(os, "sched_setaffinity"):
        cores = sorted(os.sched_getaffinity(0))
        os.sched_setaffinity(0, {cores[-1]})
    import workloads as W
    from oracle import fermion, solvers
    from oracle.lattice import Lattice
    w = W.workload("L36x36x64")
    lat = Lattice.from_params(w.lat)
    A = lambda v: fermion.apply_MMdag(lat, w.phi, 0.0, v)
    t0 = time.perf_counter()
    res = solvers.cg(A, w.b, tol=1e-12, maxit=100000)
    dt = time.perf_counter() - t0
    q.put({"x": res.x, "s": dt, "iters": res.iters, "true_rel_res": solvers.true_rel_residual(A, res.x, w.b)})


def start_c3_oracle():
    """Start the 36x36x64 oracle solve in a spawned process (one host core)
    so that it runs beside the GPU measurements that follow the timed region."""
    import multiprocessing as mp
    mctx = mp.get_context("spawn")
    q = mctx.Queue()
    proc = mctx.Process(target=_c3_oracle_job, args=(q,), daemon=True)
    # one thread in every numerical library of the child (the environment is
    # copied when it starts), so it leaves the other cores to the launches
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    os.environ.update({k: "1" for k in keys})
    try:
        proc.start()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return proc, q


def cpu_oracle_c3(job, sols):
    """The oracle's FP64 CG solution of the 36x36x64 system (1e-12) and the
    relative error of each GPU solution against it."""
    proc, q = job
    r = q.get(timeout=1800)
    proc.join(60)
    xr = r["x"]
    nr = float(np.linalg.norm(xr))
    return {"oracle_fp64_cg_s": r["s"], "oracle_iters": r["iters"], "oracle_tol": 1e-12,
            "oracle_true_rel_res": r["true_rel_res"], "cores": 1,
            "rel_error": {k: float(np.linalg.norm(x - xr) / nr) for k, x in sols.items()},
            "note": "run in a spawned process on one host core while the GPU measurements after the timed "
                    "region ran"}


def run_reference(args, rank):
    """Reference arm: the CPU oracle (numpy, complex128) as it stands, each step
    a bounded sample of the same workload: oracle M M^dagger applications on
    the 102x102x64 lattice for about 4 s."""
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_oracle_apply(0.5)
    vals, tms = [], []
    for _ in range(args.steps):
        v, reps, dt = cpu_oracle_apply(4.0)
        vals.append(v)
        tms.append(dt * 1e3)
    value = float(np.mean(vals))
    cores = 1
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(tms)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD + "; " + WORKLOAD_A.format(a=args.fgmres_a),
                       "sites": 1331712,
                       "sample": "each step: the oracle's M M^dagger applications on this lattice for "
                                 "about 4 s (a bounded sample of the trajectory's operator work)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "numpy complex128 oracle M M^dagger on 1,331,712 sites, ~4 s per step, "
                                       "single-threaded numpy"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--fgmres-a", type=float, default=1.0,
                    help="inner tolerance factor a of Algorithm A.1 for the trajectory's solves "
                         "(the paper's CPU choice is 5; on GB300, where FP64 runs at 1/58 of FP32, "
                         "a = 1 keeps every Arnoldi step preconditioned and is faster)")
    ap.add_argument("--cg-variant", type=int, default=0, choices=[0, 1, 2, 3, 4, 5, 6, 7],
                    help="FP32 CG design of the trajectory's context: 0 = autotuned (default); 1-6 pin "
                         "grid-stride, tiled, marching, persistent, grid-stride with two cells per "
                         "thread or single-reduction (hmc_set_cg_variant). Under a "
                         "profiler the autotuner's timings are distorted, so launch lists pin the design "
                         "the tuner chooses without one.")
    ap.add_argument("--graph-mode", type=int, default=2, choices=[1, 2],
                    help="2 = each CG solve one graph launch with a device-side loop (default); 1 = graph "
                         "chunks with host checks, the mode kernel profilers can see into")
    ap.add_argument("--kernel-case", default=None,
                    choices=["spcg", "spcg_grid", "spcg_tiled", "spcg_march", "spcg_persist", "spcg_pairs",
                             "spcg_single", "spcg_resident",
                             "mmdag32_stream", "mmdag32_stream_fused", "cg64", "fgmres", "mmdag32", "mmdag64",
                             "batched", "force", "md_short", "trajectory"],
                    help="run one solve or application on the benchmark lattice and exit "
                         "(the small case for kernel profiles)")
    ap.add_argument("--write-traffic", default=None, nargs="+", metavar="CSV",
                    help="write profiles/traffic.json from the raw-page CSVs of ncu captures of the FP32 "
                         "CG kernels (ncu -i REPORT --page raw --csv --print-units base > CSV) and exit")
    ap.add_argument("--traffic-command", default=[], action="append",
                    help="an ncu command that made one of the reports (recorded with the traffic)")
    args = ap.parse_args()
    if args.write_traffic:
        write_traffic(args.write_traffic, args.traffic_command)
        return
    ws, rank, local = dist_env()
    if args.kernel_case:
        kernel_case(args.kernel_case, args.graph_mode, args.cg_variant, args.fgmres_a)
        return

    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    import paper_1804_07195_gb300 as hmc
    from paper_1804_07195_gb300 import build
    import workloads as W

    build.build()
    dev = torch.device("cuda", local)
    w0 = W.workload("L102x102x64")
    p = w0.lat
    lat = hmc.Lattice(p.n, p.m, p.nt, p.kappa, p.U, p.beta)
    N = lat.nsites
    masses = list(W.L102_MASSES)
    integ = hmc.Integrator(0, W.L102_NMD, W.L102_NI, W.OMELYAN_ZETA, 1.0)
    md_opts = hmc.SolverOpts(method=1, tol=1e-10, a=args.fgmres_a)
    act_opts = hmc.SolverOpts(method=1, tol=1e-12, a=args.fgmres_a)

    nsteps_total = args.warmup + args.steps + 1 + args.e2e_steps

    def step_inputs(k):
        g = W.rng(replica_seed(W.SEEDS["L102x102x64"], rank, k))
        pi = W.draw_pi(g, N)
        rho = [W.draw_complex(g, N) for _ in range(len(masses) + 1)]
        return pi, rho

    host_inputs = [step_inputs(k) for k in range(nsteps_total)]
    phi0 = torch.tensor(w0.phi, device=dev)
    dev_inputs = [(torch.tensor(pi, device=dev), [torch.tensor(r, device=dev) for r in rho])
                  for pi, rho in host_inputs[: args.warmup + args.steps + 1]]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ctx = hmc.Context(lat)
    if args.cg_variant:
        ctx.set_cg_variant(args.cg_variant)
    ctx.set_graph_mode(args.graph_mode)
    stream = torch.cuda.current_stream()

    def trajectory(k, phi_t, pi_t, rho_t):
        return ctx.md_trajectory(phi_t, pi_t, masses, rho_t, integ, md_opts, act_opts)

    # warm-up
    for k in range(args.warmup):
        phi = phi0.clone()
        pi, rho = dev_inputs[k]
        trajectory(k, phi, pi.clone(), rho)
    torch.cuda.synchronize()

    # timed region
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    phis = [phi0.clone() for _ in range(args.steps)]
    pis = [dev_inputs[args.warmup + k][0].clone() for k in range(args.steps)]
    ctx.profile(False, reset=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall0 = time.perf_counter()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    applies = 0
    dH = []
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        H0, H1, info = trajectory(k, phis[k], pis[k], dev_inputs[args.warmup + k][1])
        ev[k][1].record(stream)
        applies += info["applies64"] + info["applies32"]
        dH.append(H1 - H0)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    graph_mode = ctx.graph_mode()
    clk = clocks.stop()
    if dist is not None:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = float(sum(step_ms))
    launches = ctx.profile_read()
    gpu_launches = int(sum(v["launches"] for v in launches.values()))

    # max over ranks of the time, sum of the work
    total_ms, sites_applied = aggregate_over_ranks(total_ms, float(N) * applies, dist, dev)
    value = sites_applied / (total_ms * 1e-3) / 1e9

    # one extra step with CUDA events around every library launch: per-kernel
    # durations for the roofline of the dominant kernel
    ctx.profile(True, reset=True)
    flush.zero_()
    phi = phi0.clone()
    pi, rho = dev_inputs[args.warmup + args.steps]
    trajectory(-1, phi, pi.clone(), rho)
    prof = ctx.profile_read()
    ctx.profile(False, reset=True)
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"])
    dname, dstat = dom
    hbm, peak_kind = peaks()
    bytes_launch = dstat["bytes"] / max(dstat["launches"], 1)
    avg_s = dstat["ms"] / max(dstat["launches"], 1) * 1e-3
    achieved = bytes_launch / avg_s / 1e9 if avg_s > 0 else 0.0
    tot_prof_ms = sum(v["ms"] for v in prof.values())
    traffic = None
    dfunc = TRAFFIC_FUNCS.get((dname, dstat.get("design", 0)))
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            tj = json.load(f)
        if tj.get("source_sha") == kernel_source_sha() and dfunc in tj.get("kernels", {}):
            traffic = tj["kernels"][dfunc]
    except Exception:
        pass
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": traffic, "kernel": dname, "function": dfunc,
                "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                "launches_per_step": dstat["launches"], "avg_launch_us": avg_s * 1e6,
                "share_of_kernel_time": dstat["ms"] / tot_prof_ms if tot_prof_ms else None,
                "algorithmic_bytes_per_launch": bytes_launch,
                "algorithmic_bytes_per_site": bytes_launch / N,
                "kernels": {k: {"launches": v["launches"], "ms": v["ms"]} for k, v in prof.items()
                            if v["launches"]},
                "tuned_shape": {"threads": dstat["threads"], "waves": dstat["waves"]},
                "method": "CUDA events around every launch on the context stream, one profiled "
                          "trajectory after the timed region"}
    if dname in ("cg_resident_f32", "cg_persist_f32"):
        roofline["note"] = ("one launch runs a whole FP32 CG solve; its algorithmic bytes are 96 B per site and "
                            "iteration (the CG step's operator with its dot, x and r updates with the norm, p "
                            "update, complex64) times the iterations the solve ran, although p and M^dagger p "
                            "stay in shared memory and r, x in L2 (1.33M sites: the working set fits the 126 MB "
                            "L2), hence a fraction near or above 1 of the copy peak; 'traffic' is the DRAM bytes "
                            "of one launch under ncu (one 60-iteration solve on this lattice, caches flushed "
                            "first): its cold first reads of r, x, b and phi and the final writes, which do not "
                            "grow with the iterations a launch runs, so far below the algorithmic bytes")
    else:
        roofline["note"] = ("the FP32 CG working set (59 MB) stays in L2 between iterations; 'traffic' is the "
                            "cold-cache DRAM bytes of one launch under ncu (the algorithmic reads); with warm "
                            "L2 the pair is latency-bound (ncu: L2 throughput 16 %, no eligible warp in about "
                            "half the scheduler cycles)")

    # end to end through the public API with host buffers
    e2e_val = None
    h2d = d2h = 0
    if args.e2e_steps > 0:
        pinned = []
        for k in range(args.e2e_steps):
            pi, rho = host_inputs[args.warmup + args.steps + 1 + k]
            pinned.append((torch.tensor(w0.phi).pin_memory(), torch.tensor(pi).pin_memory(),
                           [torch.tensor(r).pin_memory() for r in rho]))
        out_phi = torch.empty(N, dtype=torch.float64).pin_memory()
        out_pi = torch.empty(N, dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e_app = 0
        for ph_h, pi_h, rho_h in pinned:
            ph_d = ph_h.to(dev, non_blocking=True)
            pi_d = pi_h.to(dev, non_blocking=True)
            rho_d = [r.to(dev, non_blocking=True) for r in rho_h]
            H0, H1, info = ctx.md_trajectory(ph_d, pi_d, masses, rho_d, integ, md_opts, act_opts)
            out_phi.copy_(ph_d, non_blocking=True)
            out_pi.copy_(pi_d, non_blocking=True)
            torch.cuda.synchronize()
            e_app += info["applies64"] + info["applies32"]
        dt = time.perf_counter() - t0
        e2e_val = N * e_app / dt / 1e9
        h2d = 8 * N * 2 + 16 * N * (len(masses) + 1)
        d2h = 8 * N * 2 + 16

    # the oracle's 36x36x64 solve (CPU-baseline leg) runs in a spawned process on
    # one host core from here on, beside the device-timed measurements below;
    # the timed region, the per-launch roofline trajectory and the end-to-end
    # run above see an idle host
    c3_job = start_c3_oracle() if (rank == 0 and ws == 1 and args.cpu_seconds > 0) else None

    # time-to-solution on the same lattice: plain FP64 CG vs mixed FGMRES
    phi_t = phi0
    b = dev_inputs[0][1][0]
    solve = {}
    for name, fn in (("fp64_cg", lambda: ctx.solve_cg(phi_t, 0.0, b, tol=1e-10)),
                     ("mixed_fgmres", lambda: ctx.solve_fgmres(phi_t, 0.0, b, tol=1e-10, a=args.fgmres_a)),
                     ("mixed_fgmres_a5_paper", lambda: ctx.solve_fgmres(phi_t, 0.0, b, tol=1e-10, a=5.0)),
                     ("mixed_fgmres_a1", lambda: ctx.solve_fgmres(phi_t, 0.0, b, tol=1e-10, a=1.0)),
                     ("mixed_fcg", lambda: ctx.solve_fcg(phi_t, 0.0, b, tol=1e-10, a=args.fgmres_a))):
        fn()
        flush.zero_()
        torch.cuda.synchronize()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _, info = fn()
        z.record(stream)
        torch.cuda.synchronize()
        solve[name] = {"ms": a.elapsed_time(z), "iters": info["iters"], "inner_iters": info["iters_inner"],
                       "restarts": info["iters_outer"], "true_rel_res": info["true_rel_res"]}
    # the FP32 CG kernel designs, each pinned in its own context: 300
    # iterations of single-precision CG (no convergence test reached)
    designs = {}
    with hmc.Context(lat) as c2:
        for vname, v in (("grid_stride", 1), ("tiled", 2), ("marching", 3), ("persistent", 4),
                         ("grid_stride_two_cells", 5), ("single_reduction", 6), ("resident_tiles", 7)):
            c2.set_cg_variant(v)
            b32 = b.to(torch.complex64)
            c2.solve_spcg(phi_t, 0.0, b32, tol=1e-30, maxit=300, allow_fail=True)
            flush.zero_()
            torch.cuda.synchronize()
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            _, info = c2.solve_spcg(phi_t, 0.0, b32, tol=1e-30, maxit=300, allow_fail=True)
            z.record(stream)
            torch.cuda.synchronize()
            sh = c2.profile_read()["cg_M_update_f32"]
            designs[vname] = {"ms": a.elapsed_time(z), "iters": info["iters"],
                              "us_per_iter": 1e3 * a.elapsed_time(z) / max(info["iters"], 1),
                              "shape": {"threads": sh["threads"], "waves": sh["waves"], "design": sh["design"]}}
            if v == 6:
                designs[vname]["shape"] = dict(zip(("Ti", "Tj", "Tt", "depth", "in_use"), c2.cg_fused_tile()))
            if v == 7:
                designs[vname]["shape"] = {"design": c2.profile_read()["cg_resident_f32"]["design"]}
    solve["fp32_cg_designs"] = designs
    # the pair as production runs it (graph replay, no per-launch events): one
    # FP32 CG iteration moves 36 + 52 = 88 algorithmic bytes per site
    t_it = designs["grid_stride"]["us_per_iter"] * 1e-6
    pair = {"kernels": ["k_cg32_pmdag", "k_cg32_m"], "bytes_per_site": 88.0, "sites": N,
            "us_per_iteration": t_it * 1e6, "achieved": 88.0 * N / t_it / 1e9, "peak": hbm, "unit": "GB/s",
            "frac": 88.0 * N / t_it / 1e9 / hbm,
            "method": "300 FP32 CG iterations of the grid-stride pair replayed from its graph, CUDA events around "
                      "the solve; no per-launch events"}
    # the resident-tile design as the solver runs it: one launch per solve, 96
    # algorithmic bytes per site and iteration (the CG step)
    t_res = designs["resident_tiles"]["us_per_iter"] * 1e-6
    resident_roof = {"kernels": ["k_cg32_resident2" if designs["resident_tiles"]["shape"]["design"] == 4
                                 else "k_cg32_resident"], "bytes_per_site": 96.0, "sites": N,
                     "us_per_iteration": t_res * 1e6, "achieved": 96.0 * N / t_res / 1e9, "peak": hbm,
                     "unit": "GB/s", "frac": 96.0 * N / t_res / 1e9 / hbm,
                     "method": "300 FP32 CG iterations in one launch, CUDA events around the solve; the working "
                               "set is L2-resident (p and M^dagger p in shared memory)"}
    solve["speedup_mixed_vs_fp64"] = solve["fp64_cg"]["ms"] / solve["mixed_fgmres"]["ms"]
    solve["workload"] = "102x102x64 lattice, m_s=0, phi of the step, b = rho_0, true residual 1e-10"
    solve["fgmres_a"] = args.fgmres_a

    # the batched workload: 48 uneven lattices x 3 masses = 144 systems at 1e-10,
    # batched mixed vs batched FP64 vs FP64 CG one system at a time
    solve["batched_48_lattices"] = batched_solve_times(hmc, W, torch, stream, flush)
    solve["batched_trajectory_48_chains"] = batched_trajectory_times(hmc, W, torch, stream, flush)
    solve["c3_36x36x64"], c3_sols = c3_solves(hmc, W, torch, stream, flush)
    solve["apply"] = apply_rates(hmc, W, torch, stream, flush, hbm)

    # the first timed step's trajectory once more with FP64 solves at the same
    # tolerances (forces 1e-10, action 1e-12): dH of the mixed-precision path
    # against FP64 at the bench's own settings
    fp64_md = hmc.SolverOpts(method=0, tol=1e-10)
    fp64_act = hmc.SolverOpts(method=0, tol=1e-12)
    pi_s, rho_s = dev_inputs[args.warmup]
    phi_f = phi0.clone()
    H0f, H1f, info_f = ctx.md_trajectory(phi_f, pi_s.clone(), masses, rho_s, integ, fp64_md, fp64_act)
    # the error of the final action at the bench's action tolerance: the same
    # action (pseudofermions of this step, field phi_f) from mixed solves at 1e-12
    # and from FP64 CG solves at 1e-14
    chis_f, _ = ctx.make_chi(phi0, masses, rho_s, opts=hmc.SolverOpts(method=0, tol=1e-14))
    S12, _ = ctx.action(phi_f, masses, chis_f, opts=act_opts)
    S14, _ = ctx.action(phi_f, masses, chis_f, opts=hmc.SolverOpts(method=0, tol=1e-14))
    # a-posteriori bound of the action error of solves at the action
    # tolerance: for S_i = src_i^dagger eta_i with A eta_i = src_i, a computed
    # eta with true residual r gives |dS_i| <= |eta| |r| (Section 5.1's terms:
    # src_i = M_{mu_i} chi_i on M_{mu_{i-1}}, the top term chi_n on M_{mu_{n-1}})
    bound_terms = []
    for i in range(len(masses) + 1):
        lo = 0.0 if i == 0 else masses[i - 1]
        src = chis_f[i] if i == len(masses) else ctx.apply_M(phi_f, masses[i], chis_f[i])
        eta, _ = ctx.solve_fgmres(phi_f, lo, src, tol=1e-12, a=args.fgmres_a)
        r = src - ctx.apply_MMdag(phi_f, lo, eta)
        bound_terms.append(float(torch.linalg.vector_norm(eta)) * float(torch.linalg.vector_norm(r)))
    dH_check = {"dH_mixed": float(dH[0]), "dH_fp64": H1f - H0f, "abs_difference": abs(H1f - H0f - dH[0]),
                "action_true_rel_res_fp64": info_f["true_rel_res"],
                "action_error_bound_at_1e-12": {"terms": bound_terms, "sum": sum(bound_terms),
                                                "note": "|eta| |r| per Hasenbusch term for mixed solves at "
                                                        "1e-12 on this trajectory's final field: bounds the "
                                                        "action error those solves put into H1"},
                "action_error_at_1e-12": {"S_mixed_1e-12": S12, "S_fp64_1e-14": S14, "abs_difference": abs(S12 - S14),
                                          "note": "the action at the end of this trajectory from the bench's "
                                                  "action solves (mixed, 1e-12) against FP64 CG at 1e-14: what "
                                                  "the action tolerance contributes to dH"},
                "settings": "both runs: forces from solves at 1e-10, actions at 1e-12 (mixed: FGMRES with FP32 CG "
                            "inner solves; FP64: CG); the same phi, pi and rho",
                "note": "the difference is set by the solver tolerance of the MD forces (different rounding of "
                        "forces at 1e-10 moves the trajectory), not by the operator kernels; at solves of 1e-15 "
                        "the two agree within 1e-8 (tests/test_gpu_md.py)"}

    ctx.close()

    cpu = None
    if c3_job is not None:
        v, reps, dt = cpu_oracle_apply(args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"numpy complex128 oracle M M^dagger on the same 1,331,712-site lattice, "
                         f"{reps} applications in {dt:.1f} s (single-threaded numpy)"}
        c3 = cpu_oracle_c3(c3_job, c3_sols)
        cpu["c3"] = c3
        solve["c3_36x36x64"]["error_vs_oracle_fp64_cg"] = c3["rel_error"]
        cg_ms, cg_it = cpu_oracle_cg(6)
        gpu_cg = solve["fp64_cg"]
        cpu["cg"] = {"iterations_timed": cg_it, "ms_per_iteration": cg_ms,
                     "fp64_cg_solve_estimate_s": cg_ms * gpu_cg["iters"] / 1e3,
                     "note": f"the oracle's FP64 CG on the m_s = 0 system of this lattice; the solve estimate "
                             f"is its time per iteration times the {gpu_cg['iters']} iterations the GPU's FP64 "
                             f"CG takes to 1e-10 (same algorithm), against {gpu_cg['ms']:.1f} ms FP64 and "
                             f"{solve['mixed_fgmres']['ms']:.1f} ms mixed on the GPU"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": WORKLOAD + "; " + WORKLOAD_A.format(a=args.fgmres_a),
                           "l2": "flushed between steps (256 MB write, untimed)",
                           "sites": N, "mmdag_applies_per_step": applies / args.steps,
                           "cg_graph_mode": {2: "device-side loop, one graph launch per solve",
                                             1: "graph chunks with host checks",
                                             0: "direct launches"}[graph_mode],
                           "dH": [float(x) for x in dH], "wall_s_timed_region": t_wall,
                           "dH_mixed_vs_fp64": dH_check},
                "roofline": roofline, "roofline_pair_graph_replay": pair,
                "roofline_resident_tiles": resident_roof, "cpu_baseline": cpu,
                "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": gpu_launches, "clocks": clk, "solve_ms": solve}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def apply_rates(hmc, W, torch, stream, flush, hbm):
    """Operator applications alone: M, M^dagger and M M^dagger in FP32 and FP64
    on the 102x102x64 lattice (its vectors stay in the 135 MB L2 between
    applications) and on a 306x306x64 lattice (12M sites, L2 flushed before
    every application, so each one streams from HBM). M M^dagger runs in both
    designs: two passes (u = M^dagger x written to memory and read back) and
    the fused kernel (u kept on chip). Kernel time comes from the library's
    CUDA events around each launch (no host call overhead). frac_hbm counts
    the algorithmic bytes per site of the operation -- what it must move: the
    vector in and out and phi (FP32: 8 + 8 + 4 = 20 B; FP64: 16 + 16 + 8 =
    40 B), the same for M, M^dagger and M M^dagger -- against the measured
    copy peak. On the streaming lattice the same operations are also timed
    back to back over three rotating operand sets (x and the result: 576 MB
    in FP32, 1.15 GB in FP64, all larger than L2 together), CUDA events
    around 30 applications: no event gap per launch and no flush whose dirty
    lines the application must write back, yet no operand read from L2 that
    an earlier application left there (each application streams 240 MB,
    and its set returns two applications later). Reported beside the
    per-launch figures as us_back_to_back and frac_hbm_back_to_back."""
    out = {}
    per_site = {32: 20.0, 64: 40.0}
    kernels = {"M": ["apply_M_f{p}"], "Mdag": ["apply_Mdag_f{p}"],
               "MMdag_two_pass": ["apply_Mdag_f{p}", "apply_M_f{p}"], "MMdag_fused": ["mmdag_fused_f{p}"]}
    for name, (n, m, nt) in (("l2_resident_102x102x64", (102, 102, 64)), ("streaming_306x306x64", (306, 306, 64))):
        lat = hmc.Lattice(n, m, nt, 1.0, 3.8, 12.0)
        N = lat.nsites
        g = W.rng(9000 + n)
        phi = torch.tensor(g.normal(0.0, math.sqrt(lat.delta * 3.8), N), device="cuda")
        rows = {}
        with hmc.Context(lat) as ctx:
            ctx.load_field(phi)
            for prec in (32, 64):
                ct = torch.complex64 if prec == 32 else torch.complex128
                x = torch.randn(N, dtype=ct, device="cuda")
                xs = outs = None
                if name.startswith("streaming"):
                    xs = [x] + [torch.randn(N, dtype=ct, device="cuda") for _ in range(2)]
                    outs = [torch.empty_like(x) for _ in range(3)]
                for op in ("M", "Mdag", "MMdag_two_pass", "MMdag_fused"):
                    if op == "MMdag_two_pass":
                        ctx.set_apply_variant(1)
                    elif op == "MMdag_fused":
                        ctx.set_apply_variant(2)
                    fn = {"M": lambda: ctx.apply_M(None, 0.1, x), "Mdag": lambda: ctx.apply_Mdag(None, 0.1, x)}.get(
                        op, lambda: ctx.apply_MMdag(None, 0.1, x))
                    for _ in range(3):
                        fn()
                    torch.cuda.synchronize()
                    reps = 20
                    # a head start of GPU work, so that the host has queued
                    # every timed application before the GPU reaches it (the
                    # events around each launch would otherwise include any
                    # host delay between them)
                    for _ in range(32):
                        flush.zero_()
                    ctx.profile(True, reset=True)
                    for _ in range(reps):
                        if name.startswith("streaming"):
                            flush.zero_()
                        fn()
                    torch.cuda.synchronize()
                    prof = ctx.profile_read()
                    ctx.profile(False, reset=True)
                    t = sum(prof[k.format(p=prec)]["ms"] for k in kernels[op]) * 1e-3 / reps
                    nbytes = per_site[prec] * N
                    row = {"us": t * 1e6, "gsite_s": N / t / 1e9, "gb_s": nbytes / t / 1e9,
                           "frac_hbm": nbytes / t / 1e9 / hbm}
                    if op == "MMdag_fused":
                        row["tile"] = dict(zip(("Ti", "Tj", "Tt", "depth", "pairs"), ctx.fused_tile(prec)))
                    if name.startswith("streaming"):
                        ts = back_to_back(torch, stream, flush, op, ctx, xs, outs)
                        row["us_back_to_back"] = ts * 1e6
                        row["frac_hbm_back_to_back"] = nbytes / ts / 1e9 / hbm
                    rows[f"{op}_f{prec}"] = row
                ctx.set_apply_variant(0)
                del x, xs, outs
        out[name] = {"sites": N, **rows}
    out["streaming_102x102x64_x8"] = c5_times_eight(hmc, W, torch, stream, flush, hbm, per_site)
    out["note"] = ("mean kernel time of 20 applications (CUDA events around each launch inside the library); "
                   "the streaming lattice flushes L2 before every application (us, frac_hbm) and is also "
                   "timed back to back over three rotating operand sets larger than L2 together "
                   "(us_back_to_back, frac_hbm_back_to_back: no per-launch event gap, no flush to write "
                   "back); frac_hbm = algorithmic bytes "
                   "(20 B/site FP32, 40 B/site FP64, also for M M^dagger) / time / measured copy peak; the "
                   "fused tile is the one the library's tuner chose for this lattice")
    return out


def c5_times_eight(hmc, W, torch, stream, flush, hbm, per_site, copies=8, reps=32):
    """The benchmark lattice (102x102x64) streamed from HBM: eight contexts,
    each with its own field phi and its own vectors (together larger than L2:
    213 MB in FP32, 426 MB in FP64), applied round-robin back to back, CUDA
    events around `reps` applications; each context's tile and M M^dagger
    design are its own tuner's. Counted at the same algorithmic bytes per
    site as the other rows."""
    n, m, nt = 102, 102, 64
    lat = hmc.Lattice(n, m, nt, 1.0, 3.8, 12.0)
    N = lat.nsites
    rows = {}
    ctxs, phis = [], []
    try:
        for c in range(copies):
            g = W.rng(9100 + c)
            phis.append(torch.tensor(g.normal(0.0, math.sqrt(lat.delta * 3.8), N), device="cuda"))
            ctx = hmc.Context(lat)
            ctx.load_field(phis[-1])
            ctxs.append(ctx)
        for prec in (32, 64):
            ct = torch.complex64 if prec == 32 else torch.complex128
            xs = [torch.randn(N, dtype=ct, device="cuda") for _ in range(copies)]
            outs = [torch.empty_like(xs[0]) for _ in range(copies)]
            for op in ("M", "Mdag", "MMdag_two_pass", "MMdag_fused"):
                def app(k):
                    ctx, x, o = ctxs[k % copies], xs[k % copies], outs[k % copies]
                    if op == "M":
                        ctx.apply_M(None, 0.1, x, out=o)
                    elif op == "Mdag":
                        ctx.apply_Mdag(None, 0.1, x, out=o)
                    else:
                        ctx.apply_MMdag(None, 0.1, x, out=o)
                for ctx in ctxs:
                    ctx.set_apply_variant({"MMdag_two_pass": 1, "MMdag_fused": 2}.get(op, 0))
                for k in range(2 * copies):  # tunes each context, then warms
                    app(k)
                for _ in range(16):
                    flush.zero_()
                a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for k in range(reps):
                    app(k)
                z.record(stream)
                torch.cuda.synchronize()
                t = a.elapsed_time(z) * 1e-3 / reps
                nbytes = per_site[prec] * N
                row = {"us": t * 1e6, "gsite_s": N / t / 1e9, "gb_s": nbytes / t / 1e9, "frac_hbm": nbytes / t / 1e9 / hbm}
                if op == "MMdag_fused":
                    row["tile"] = dict(zip(("Ti", "Tj", "Tt", "depth", "pairs"), ctxs[0].fused_tile(prec)))
                rows[f"{op}_f{prec}"] = row
            del xs, outs
    finally:
        for ctx in ctxs:
            ctx.close()
    return {"sites": N, "copies": copies, **rows,
            "note": "eight independent 102x102x64 fields and vector sets applied round-robin back to back "
                    "(working set larger than L2); CUDA events around %d applications" % reps}


def back_to_back(torch, stream, flush, op, ctx, xs, outs, reps=30):
    """Seconds per application of op, applications back to back over the
    rotating operand sets xs -> outs (see apply_rates)."""
    def app(k):
        x, o = xs[k % len(xs)], outs[k % len(xs)]
        if op == "M":
            ctx.apply_M(None, 0.1, x, out=o)
        elif op == "Mdag":
            ctx.apply_Mdag(None, 0.1, x, out=o)
        else:
            ctx.apply_MMdag(None, 0.1, x, out=o)
    for k in range(len(xs)):
        app(k)
    flush.zero_()
    for _ in range(16):  # a head start of GPU work, so that the host queues ahead of the GPU
        flush.zero_()
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for k in range(reps):
        app(k)
    z.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(z) * 1e-3 / reps


def batched_solve_times(hmc, W, torch, stream, flush):
    systems, ctxs = [], {}
    for w in W.batch_instances():
        p = w.lat
        lat = hmc.Lattice(p.n, p.m, p.nt, p.kappa, p.U, p.beta)
        key = (p.n, p.m, p.nt)
        if key not in ctxs:
            ctxs[key] = hmc.Context(lat)
        phi = torch.tensor(w.phi, device="cuda")
        for ms, b in zip(w.masses, w.rho):
            systems.append({"lattice": lat, "phi": phi, "ms": ms, "b": torch.tensor(b, device="cuda"),
                            "x": torch.zeros(p.nsites, dtype=torch.complex128, device="cuda"),
                            "tol": 1e-10, "key": key})
    any_ctx = next(iter(ctxs.values()))

    def timed(fn):
        fn()  # warm (autotuning, graph capture)
        flush.zero_()
        torch.cuda.synchronize()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = fn()
        z.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(z), r

    def seq(method):
        worst = 0.0
        for sy in systems:
            c = ctxs[sy["key"]]
            if method == "cg":
                _, info = c.solve_cg(sy["phi"], sy["ms"], sy["b"], tol=1e-10)
            else:
                _, info = c.solve_fgmres(sy["phi"], sy["ms"], sy["b"], tol=1e-10)
            worst = max(worst, info["true_rel_res"])
        return worst

    out = {"systems": len(systems), "sites": int(sum(sy["lattice"].nsites for sy in systems))}

    def site_applies(infos):
        # sites x M M^dagger applications summed over the systems (both precisions)
        return float(sum(sy["lattice"].nsites * (i["applies64"] + i["applies32"]) for sy, i in zip(systems, infos)))

    ms, infos = timed(lambda: any_ctx.solve_batched(systems, mixed=True))
    out["batched_mixed_ms"] = ms
    out["batched_mixed_max_true_rel_res"] = max(i["true_rel_res"] for i in infos)
    out["batched_mixed_gsite_s"] = site_applies(infos) / (ms * 1e-3) / 1e9
    out["batched_mixed_design_chosen"] = {1: "graph_loop", 2: "persistent"}.get(any_ctx.batched_variant(), "none")
    # both FP32 CG designs of the batched solver pinned in turn
    designs = {}
    for v, name in ((1, "graph_loop"), (2, "persistent")):
        any_ctx.set_batched_variant(v)
        ms_v, infos_v = timed(lambda: any_ctx.solve_batched(systems, mixed=True))
        designs[name] = {"ms": ms_v, "max_true_rel_res": max(i["true_rel_res"] for i in infos_v)}
    any_ctx.set_batched_variant(0)
    out["batched_mixed_designs"] = designs
    ms, infos = timed(lambda: any_ctx.solve_batched(systems, mixed=False))
    out["batched_fp64_ms"] = ms
    out["batched_fp64_max_true_rel_res"] = max(i["true_rel_res"] for i in infos)
    out["batched_fp64_gsite_s"] = site_applies(infos) / (ms * 1e-3) / 1e9
    ms, worst = timed(lambda: seq("cg"))
    out["sequential_fp64_cg_ms"] = ms
    out["sequential_fp64_cg_max_true_rel_res"] = worst
    ms, worst = timed(lambda: seq("fgmres"))
    out["sequential_mixed_fgmres_ms"] = ms
    out["speedup_batched_mixed_vs_sequential_fp64"] = out["sequential_fp64_cg_ms"] / out["batched_mixed_ms"]
    out["note"] = ("gsite_s = sum over systems of sites x M M^dagger applications (FP64 and FP32) / time: "
                   "the operator throughput the batched solve sustains")
    for c in ctxs.values():
        c.close()
    return out


def batched_trajectory_times(hmc, W, torch, stream, flush):
    """The 48 batched instances run as independent Markov chains: one nested
    Omelyan trajectory per chain (3 Hasenbusch masses, N_MD and time scales of
    workloads.BATCH_NMD / BATCH_NI, mixed-precision solves at 1e-10 for the
    forces and 1e-12 for the action), all chains in lockstep with every
    schedule point's solves batched (hmc_md_trajectory_batched), against the
    same trajectories one chain at a time (hmc_md_trajectory)."""
    insts = W.batch_instances()
    extra = W.batch_chains(insts)
    masses = list(W.BATCH_MASSES)
    integ = hmc.Integrator(0, W.BATCH_NMD, W.BATCH_NI)
    md = hmc.SolverOpts(method=1, tol=1e-10, a=1.0)
    act = hmc.SolverOpts(method=1, tol=1e-12, a=1.0)
    lats = [hmc.Lattice(w.lat.n, w.lat.m, w.lat.nt, w.lat.kappa, w.lat.U, w.lat.beta) for w in insts]
    phis = [torch.tensor(w.phi, device="cuda") for w in insts]
    pis = [torch.tensor(pi, device="cuda") for pi, _ in extra]
    rhos = [[torch.tensor(r, device="cuda") for r in rho] for _, rho in extra]

    def chains():
        return [{"lattice": L, "phi": ph.clone(), "pi": pi.clone(), "rho": rh}
                for L, ph, pi, rh in zip(lats, phis, pis, rhos)]

    out = {"chains": len(insts), "sites": int(sum(L.nsites for L in lats)), "masses": masses,
           "nmd": W.BATCH_NMD, "time_scales": list(W.BATCH_NI)}
    with hmc.Context(lats[0]) as ctx:
        ctx.md_trajectory_batched(chains(), masses, integ, md, act)  # warm (contexts, tuning, graphs)
        ch = chains()
        flush.zero_()
        torch.cuda.synchronize()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        H0, H1, infos = ctx.md_trajectory_batched(ch, masses, integ, md, act)
        z.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(z)
    work = float(sum(L.nsites * (i["applies64"] + i["applies32"]) for L, i in zip(lats, infos)))
    out["batched_ms"] = ms
    out["batched_gsite_s"] = work / (ms * 1e-3) / 1e9
    out["dH"] = [h1 - h0 for h0, h1 in zip(H0, H1)]
    ctxs = {}
    for L in lats:
        key = (L.n, L.m, L.nt)
        if key not in ctxs:
            ctxs[key] = hmc.Context(L)

    def seq():
        res = []
        for L, c in zip(lats, chains()):
            res.append(ctxs[(L.n, L.m, L.nt)].md_trajectory(c["phi"], c["pi"], masses, c["rho"], integ, md, act))
        return res

    seq()  # warm
    flush.zero_()
    torch.cuda.synchronize()
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    res = seq()
    z.record(stream)
    torch.cuda.synchronize()
    out["sequential_ms"] = a.elapsed_time(z)
    work_seq = float(sum(L.nsites * (r[2]["applies64"] + r[2]["applies32"]) for L, r in zip(lats, res)))
    out["sequential_gsite_s"] = work_seq / (out["sequential_ms"] * 1e-3) / 1e9
    out["speedup_batched_vs_sequential"] = out["sequential_ms"] / out["batched_ms"]
    out["max_abs_dH_difference_batched_vs_sequential"] = max(
        abs((r[1] - r[0]) - d) for r, d in zip(res, out["dH"]))
    for c in ctxs.values():
        c.close()
    return out


def c3_solves(hmc, W, torch, stream, flush):
    """The 36x36x64 lattice (m_s = 0, b of the workload, true residual 1e-10):
    plain FP64 CG and mixed-precision FGMRES (FP32 CG inner solves, FP64
    outer) at a = 5 (the paper's value) and a = 1, with their iteration counts
    and times; the solutions are returned for the comparison with the oracle's
    FP64 CG solution in the CPU-baseline leg."""
    w = W.workload("L36x36x64")
    p = w.lat
    lat = hmc.Lattice(p.n, p.m, p.nt, p.kappa, p.U, p.beta)
    phi = torch.tensor(w.phi, device="cuda")
    b = torch.tensor(w.b, device="cuda")
    out, sols = {"lattice": "36x36x64", "sites": lat.nsites, "ms": 0.0, "tol": 1e-10}, {}
    with hmc.Context(lat) as ctx:
        for name, fn in (("fp64_cg", lambda: ctx.solve_cg(phi, 0.0, b, tol=1e-10)),
                         ("mixed_fgmres_a5", lambda: ctx.solve_fgmres(phi, 0.0, b, tol=1e-10, a=5.0)),
                         ("mixed_fgmres_a1", lambda: ctx.solve_fgmres(phi, 0.0, b, tol=1e-10, a=1.0))):
            fn()
            flush.zero_()
            torch.cuda.synchronize()
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            x, info = fn()
            z.record(stream)
            torch.cuda.synchronize()
            out[name] = {"ms": a.elapsed_time(z), "iters": info["iters"], "restarts": info["iters_outer"],
                         "inner_iters": info["iters_inner"], "true_rel_res": info["true_rel_res"]}
            sols[name] = x.cpu().numpy()
    del out["ms"]
    out["speedup_mixed_a1_vs_fp64"] = out["fp64_cg"]["ms"] / out["mixed_fgmres_a1"]["ms"]
    return out, sols


def replica_seed(base, rank, step):
    """Seed of the inputs of step `step` on rank `rank`: every rank runs its own
    independent trajectories (replicas), so the streams must differ by rank."""
    return [int(base), int(rank), int(step)]


def aggregate_over_ranks(ms, work, dist, device=None):
    """Whole-job timing of replicas: the slowest rank's time and the summed work
    (the only cross-rank communication of the benchmark; none on the data path)."""
    if dist is None:
        return float(ms), float(work)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    w = torch.tensor([float(work)], dtype=torch.float64, device=device)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())


def kernel_case(case, graph_mode=2, cg_variant=0, fgmres_a=1.0):
    """One solve (or 20 operator applications, a force, a trajectory) on the
    102x102x64 lattice: the cases the ncu kernel profiles and launch lists are
    taken on."""
    import torch
    import paper_1804_07195_gb300 as hmc
    from paper_1804_07195_gb300 import build
    import workloads as W
    build.build()
    if case in ("mmdag32_stream", "mmdag32_stream_fused"):
        # 306x306x64 (12M sites): vectors far larger than L2, L2 flushed before each
        # application; two passes, or the fused kernel on a pinned tile (no tuning launches)
        lat = hmc.Lattice(306, 306, 64, 1.0, 3.8, 12.0)
        g = W.rng(9306)
        phi = torch.tensor(g.normal(0.0, math.sqrt(lat.delta * 3.8), lat.nsites), device="cuda")
        x = torch.randn(lat.nsites, dtype=torch.complex64, device="cuda")
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
        with hmc.Context(lat) as ctx:
            ctx.load_field(phi)
            if case == "mmdag32_stream_fused":
                ctx.set_apply_variant(2)
                ctx.set_fused_tile(32, *FUSED_STREAM_TILE)
            else:
                ctx.set_apply_variant(1)
            for _ in range(8):
                flush.zero_()
                ctx.apply_MMdag(None, 0.1, x)
            torch.cuda.synchronize()
        print(json.dumps({"case": case, "sites": lat.nsites, "applications": 8}))
        return
    if case == "batched":
        sys_ = []
        for w in W.batch_instances():
            p = w.lat
            lat = hmc.Lattice(p.n, p.m, p.nt, p.kappa, p.U, p.beta)
            for ms, b in zip(w.masses, w.rho):
                sys_.append({"lattice": lat, "phi": torch.tensor(w.phi, device="cuda"), "ms": ms,
                             "b": torch.tensor(b, device="cuda"),
                             "x": torch.zeros(p.nsites, dtype=torch.complex128, device="cuda")})
        with hmc.Context(sys_[0]["lattice"]) as ctx:
            infos = ctx.solve_batched(sys_, mixed=True)
        print(json.dumps({"case": case, "systems": len(infos),
                          "max_true_rel_res": max(i["true_rel_res"] for i in infos)}))
        return
    w = W.workload("L102x102x64")
    p = w.lat
    lat = hmc.Lattice(p.n, p.m, p.nt, p.kappa, p.U, p.beta)
    phi = torch.tensor(w.phi, device="cuda")
    b = torch.tensor(w.b, device="cuda")
    with hmc.Context(lat) as ctx:
        ctx.set_graph_mode(graph_mode)
        if case in ("spcg", "spcg_grid", "spcg_tiled", "spcg_march", "spcg_persist", "spcg_pairs", "spcg_single",
                    "spcg_resident"):
            ctx.set_cg_variant({"spcg": 0, "spcg_grid": 1, "spcg_tiled": 2, "spcg_march": 3,
                                "spcg_persist": 4, "spcg_pairs": 5, "spcg_single": 6, "spcg_resident": 7}[case])
            if case == "spcg_single":
                ctx.set_cg_fused_tile(*SINGLE_REDUCTION_TILE)
            _, info = ctx.solve_spcg(phi, 0.0, b.to(torch.complex64), tol=1e-6, maxit=60, allow_fail=True)
        elif case == "cg64":
            _, info = ctx.solve_cg(phi, 0.0, b, tol=1e-10, maxit=30, allow_fail=True)
        elif case == "fgmres":
            _, info = ctx.solve_fgmres(phi, 0.0, b, tol=1e-10)
        elif case == "force":
            # the benchmark's force of all terms: pseudofermions for the three
            # masses, then dS/dphi (Gaussian + every Hasenbusch term)
            masses = list(W.L102_MASSES)
            rho = [torch.tensor(r, device="cuda") for r in w.rho]
            opts = hmc.SolverOpts(method=1, tol=1e-10, a=1.0)
            chis, _ = ctx.make_chi(phi, masses, rho, opts=opts)
            _, info = ctx.force(phi, masses, chis, opts=opts)
        elif case == "trajectory":
            # two trajectories of the benchmark step (the first one warms the
            # tuners and graphs); launch lists skip the first
            if cg_variant:
                ctx.set_cg_variant(cg_variant)
            masses = list(W.L102_MASSES)
            rho = [torch.tensor(r, device="cuda") for r in w.rho]
            integ = hmc.Integrator(0, W.L102_NMD, W.L102_NI, W.OMELYAN_ZETA, 1.0)
            md = hmc.SolverOpts(method=1, tol=1e-10, a=fgmres_a)
            act = hmc.SolverOpts(method=1, tol=1e-12, a=fgmres_a)
            for k in range(2):
                if k == 1:
                    # profilers started with collection off capture the second one only
                    torch.cuda.synchronize()
                    torch.cuda.profiler.start()
                H0, H1, info = ctx.md_trajectory(phi.clone(), torch.tensor(w.pi, device="cuda"), masses, rho, integ,
                                                 md, act)
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
        elif case == "md_short":
            # a short trajectory of the benchmark's kind (N_MD = 6, time scales 2, 1, 1):
            # the MD updates, energies and forces of the path
            masses = list(W.L102_MASSES)
            rho = [torch.tensor(r, device="cuda") for r in w.rho]
            opts = hmc.SolverOpts(method=1, tol=1e-10, a=1.0)
            H0, H1, info = ctx.md_trajectory(phi.clone(), torch.tensor(w.pi, device="cuda"), masses, rho,
                                             hmc.Integrator(0, 6, (2, 1, 1)), opts,
                                             hmc.SolverOpts(method=1, tol=1e-12, a=1.0))
        else:
            x = b.to(torch.complex64) if case == "mmdag32" else b
            ctx.load_field(phi)
            for _ in range(20):
                y = ctx.apply_MMdag(None, 0.0, x)
            info = {"applications": 20}
        torch.cuda.synchronize()
    print(json.dumps({"case": case, **{k: v for k, v in info.items()}}))


# tile of the single-reduction CG kernel profile (the tuner's choice on the
# 102x102x64 lattice): Ti, Tj, Tt, depth
SINGLE_REDUCTION_TILE = (14, 8, 16, 2)

# fused M M^dagger tile of the streaming kernel profile: Ti, Tj, Tt, depth, pairs
FUSED_STREAM_TILE = (28, 14, 22, 2, 1)

# the translation units of the FP32 CG kernels whose DRAM traffic
# profiles/traffic.json records, and everything they include
PAIR_SOURCES = ("paper_1804_07195_gb300/csrc/kernels.cu", "paper_1804_07195_gb300/csrc/cg32_fused.cu",
                "paper_1804_07195_gb300/csrc/cg32_resident.cu",
                "paper_1804_07195_gb300/csrc/kernels.h", "paper_1804_07195_gb300/csrc/ctx.h",
                "paper_1804_07195_gb300/csrc/common.cuh", "paper_1804_07195_gb300/csrc/operator.cuh",
                "paper_1804_07195_gb300/csrc/launch.cuh", "include/hmc.h")

# (profile name, design) of a CG kernel -> its CUDA function
TRAFFIC_FUNCS = {("cg_pMdag_f32", 0): "k_cg32_pmdag", ("cg_M_update_f32", 0): "k_cg32_m",
                 ("cg_pMdag_f32", 4): "k_cg32_pmdag2", ("cg_M_update_f32", 4): "k_cg32_m2",
                 ("cg1_fused_f32", 0): "k_cg32_fused1", ("cg_resident_f32", 0): "k_cg32_resident",
                 ("cg_resident_f32", 4): "k_cg32_resident2"}


def kernel_source_sha():
    import hashlib
    h = hashlib.sha256()
    for f in PAIR_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def traffic_from_csv(text):
    """Mean DRAM bytes (read + written) per launch of every kernel in the
    raw-page CSV of an ncu report printed with base units, and the launch
    counts: ({function: bytes}, {function: launches})."""
    import csv
    import re
    rows = list(csv.reader(text.splitlines()))
    start = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr, units = rows[start], rows[start + 1]
    ki, ri, wi = hdr.index("Kernel Name"), hdr.index("dram__bytes_read.sum"), hdr.index("dram__bytes_write.sum")
    if units[ri] != "byte" or units[wi] != "byte":
        raise ValueError(f"expected base units (byte), got {units[ri]!r}, {units[wi]!r}")
    per = {}
    for r in rows[start + 2:]:
        if len(r) != len(hdr):
            continue
        m = re.search(r"\b(k_\w+)", r[ki])
        if not m:
            continue
        per.setdefault(m.group(1), []).append(float(r[ri].replace(",", "")) + float(r[wi].replace(",", "")))
    return {k: sum(v) / len(v) for k, v in per.items()}, {k: len(v) for k, v in per.items()}


def write_traffic(csv_paths, commands):
    kernels, launches = {}, {}
    for path in csv_paths:
        with open(path) as f:
            k, n = traffic_from_csv(f.read())
        kernels.update(k)
        launches.update(n)
    rec = {"source_sha": kernel_source_sha(), "sources": list(PAIR_SOURCES), "capture": commands,
           "kernels": kernels, "launches_captured": launches,
           "note": "cold-cache DRAM bytes read + written per launch (caches flushed before each ncu pass)"}
    with open(os.path.join(ROOT, "profiles", "traffic.json"), "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
