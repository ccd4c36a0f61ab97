"""Benchmark of the adaptive GSIS hot path on one GB300 (or N independent replicas).

Default workload: hypersonic cylinder, Ma = 5, Kn = 0.01, wall at 2 T_inf,
128 x 128 O-grid, 48x48x24 velocity grid, FP64, adaptive with Kn_ref = 0.01.
A step is one GSIS iteration (cell equilibrium, kinetic sweep, moments and
HoT, synthetic solve, VDF correction, residual) over the resident state.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gsis|reference]
                    [--config cylinder|shock|cylinder_full|sphere|batch] [--dtype f64|f32|bf16|f16]

--config batch: 64 independent 1D shocks (seeded Ma in [1.5, 8], 100-800
cells, 24^3..64^3 velocity grids, even solves FP32 and odd BF16 VDFs) advanced
together by gsis_iterate_batch (one persistent sweep launch, one fused
synthetic-solve launch, one CUDA graph per iteration; autotuned tile shape).

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
a bounded sample of the same workload (a 12 x 12 O-grid with the same velocity
grid), in the same metric.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "cell×velocity updates/s and time-to-converged state vs plain FP64 GPU"
UNIT = "cell*velocity updates/s"
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12   # 152 SMs x 2 DFMA/clk (4 flop) x 2.07 GHz
# algorithmic FP64 flops of one point update of the kinetic sweep on a 2D
# structured mesh (4 active faces, FMA = 2), counted from the scheme: reference
# distribution and 1/tau 14, face normal speeds 4 x 5, two outgoing faces 2 x 4,
# two own limited slopes 2 x 4, two incoming MUSCL face values 2 x 8, division 1.
SWEEP_FLOPS_PER_POINT_2D = 67
# the same count on a 1D mesh (2 active faces): reference distribution and 1/tau 14, two
# normal speeds 2 x 3, one outgoing face 4, one own slope 4, one incoming MUSCL value 8, division 1.
SWEEP_FLOPS_PER_POINT_1D = 37


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gsis", choices=["gsis", "reference"])
    ap.add_argument("--config", default="cylinder",
                    choices=["cylinder", "shock", "cylinder_full", "sphere", "cylinder32", "batch"])
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32", "bf16", "f16"])
    ap.add_argument("--tile", default=None,
                    help="run the sweep with this tile shape instead of the autotuned one (for profiler captures)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-converge", action="store_true", help="skip the time-to-converged measurement")
    return ap.parse_args()


def make_case(config, small=False):
    from workloads import shock_1d_case, cylinder_case, sphere_case, shock_batch_cases
    if config == "batch":   # the first shock of the seeded batch (small: reduced to 20 cells)
        c0 = shock_batch_cases(n=1)[0]
        if not small:
            return c0
        return shock_1d_case(Ma=c0.extra["Ma"], n_cells=20, half_width=2.5, nv=c0.vgrid.n, vmax=c0.vgrid.hi[0],
                             macro_steps=c0.macro_steps)
    if config == "shock":
        return shock_1d_case(n_cells=200 if not small else 40)
    if config == "cylinder32":   # reduced mesh, same velocity grid (for profiler captures)
        return cylinder_case(n_r=32, n_theta=32, presolve_max_blocks=5)
    if config in ("cylinder", "cylinder_full"):
        adaptive = config == "cylinder"
        if small:
            return cylinder_case(n_r=12, n_theta=12, presolve_max_blocks=1, macro_steps=20, adaptive=adaptive)
        return cylinder_case(adaptive=adaptive)
    if small:
        return sphere_case(n_r=6, n_pol=4, n_az=4, presolve_max_blocks=1, macro_steps=10)
    return sphere_case()


def workload_name(config, dtype):
    return {
        "cylinder": "2D cylinder Ma=5 Kn=0.01 Tw=2, O-grid 128x128, velocity grid 48x48x24, adaptive Kn_ref=0.01",
        "cylinder_full": "2D cylinder Ma=5 Kn=0.01 Tw=2, O-grid 128x128, velocity grid 48x48x24, full kinetic",
        "cylinder32": "2D cylinder Ma=5 Kn=0.01 Tw=2, O-grid 32x32, velocity grid 48x48x24, adaptive Kn_ref=0.01",
        "shock": "1D normal shock Ma=2, 200 cells on [-25,25] mfp, velocity grid 48x24x24, all kinetic",
        "sphere": "3D sphere Ma=5 Kn=0.005 Tw=2, O-grid 96x64x64, velocity grid 48^3, adaptive Kn_ref=0.01",
        "batch": "batch of 64 1D shocks, Ma~U[1.5,8], 100-800 cells, velocity grids 24^3..64^3, "
                 "one persistent launch + CUDA graph",
    }[config] + (", VDF " + dtype if config != "batch" else ", VDF f32 (even) / bf16 (odd)")


def combine_ranks(points, ms, dist=None, device="cpu"):
    """Whole-job throughput of independent replicas: the points all ranks
    processed over the slowest rank's time (max over ranks).  Returns
    (points per second, max milliseconds); dist is torch.distributed or None."""
    if dist is None:
        return points / (ms * 1e-3), ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    p = torch.tensor([float(points)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    t_max = float(t.item())
    return float(p.item()) / (t_max * 1e-3), t_max


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """Samples nvidia-smi clocks / throttle reasons every 200 ms in the background."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def source_sha(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_from_profile(config, dtype):
    """DRAM bytes per sweep launch from the committed ncu summary, if it was
    taken on the current sweep source (else null)."""
    p = os.path.join(ROOT, "profiles", "sweep_%s_%s.json" % (config, dtype))
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    sha = source_sha(["paper_2501_02245_gb300/csrc/sweep.cu", "paper_2501_02245_gb300/csrc/sweep_device.cuh",
                      "paper_2501_02245_gb300/csrc/gsis_device.cuh"])
    if d.get("sweep_src_sha") != sha:
        return None
    return d.get("dram_bytes_per_launch_full")


def cpu_baseline(config, steps=1):
    """The oracle as it stands, timed on a bounded sample of the workload:
    one GSIS iteration on a 12x12 O-grid (same velocity grid, same physics)."""
    from oracle.gsis import OracleSolver
    case = make_case(config, small=True)
    o = OracleSolver(case)
    o.initialise()
    t = time.perf_counter()
    pts = 0
    for _ in range(steps):
        o.step()
        pts += int(o.dvm.sum()) * o.vg.nv
    dt = time.perf_counter() - t
    return pts / dt, dt, int(o.dvm.sum()), o.vg.nv, case.mesh.ncell


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle.gsis import OracleSolver
    case = make_case(args.config, small=True)
    o = OracleSolver(case)
    o.initialise()
    for _ in range(args.warmup):
        o.step()
    t = time.perf_counter()
    pts = 0
    for _ in range(args.steps):
        o.step()
        pts += int(o.dvm.sum()) * o.vg.nv
    dt = time.perf_counter() - t
    value = pts / dt
    sample = ("one GSIS iteration per step of the FP64 oracle on a %d-cell %s sample (%d DVM cells) with the "
              "workload's velocity grid (%d velocities)" % (case.mesh.ncell, args.config, int(o.dvm.sum()), o.vg.nv))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.config, args.dtype), "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def mesh_bytes(case):
    m = case.mesh
    b = m.centers.nbytes + m.volumes.nbytes + sum(a.nbytes for a in m.S) + sum(a.nbytes for a in m.xf)
    return b + case.W0.nbytes


def run_gsis(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    from paper_2501_02245_gb300 import Solver
    case = make_case(args.config)
    case.tol = 0.0   # time exactly the requested number of iterations
    stream = torch.cuda.current_stream()
    s = Solver.from_case(case, vdf_dtype=args.dtype, stream=stream)
    rep0 = s.iterate(0)
    if args.tile:
        s.set_sweep_tile(args.tile)
    for _ in range(args.warmup):
        s.iterate(1)
    clocks = Clocks(local)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    rep = s.iterate(args.steps)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ck = clocks.stop()
    if pg:
        pg.barrier()
    ms = e0.elapsed_time(e1)
    pts = rep["n_dvm"] * rep["n_v"] * args.steps
    value, t_max = combine_ranks(pts, ms, pg, "cuda")
    # dominant kernel: the sweep; its launches are bracketed by CUDA events on the context stream
    sweep_ms_per_launch = rep["phase_ms"]["sweep"] / max(rep["sweep_launches"], 1)
    pts_per_launch = rep["n_dvm"] * rep["n_v"]
    eb = {"f64": 8, "f32": 4, "bf16": 2, "f16": 2}[args.dtype]
    traffic = traffic_from_profile(args.config, args.dtype)
    if args.dtype == "f64":
        fpp = SWEEP_FLOPS_PER_POINT_1D if args.config == "shock" else SWEEP_FLOPS_PER_POINT_2D
        flops = fpp * pts_per_launch
        achieved = flops / (sweep_ms_per_launch * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                "kernel": "k_sweep<double> (one Gauss-Seidel pass)",
                "peak_source": "FP64 unit counts x clock: 152 SMs x 2 DFMA/clk x 2.07 GHz (derived)",
                "algorithmic": "%d FP64 flop per (cell, velocity) per pass" % fpp}
    else:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
        bytes_alg = 2 * eb * pts_per_launch   # read f once + write f once per pass
        achieved = bytes_alg / (sweep_ms_per_launch * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                "kernel": "k_sweep (one Gauss-Seidel pass)", "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)",
                "algorithmic": "2 x %d bytes per (cell, velocity) per pass" % eb}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": workload_name(args.config, args.dtype), "parallelism": "replicas" if ws > 1 else "1 GPU",
                       "n_dvm": rep["n_dvm"], "n_cells": case.mesh.ncell, "n_v": rep["n_v"],
                       "vdf_bytes": rep["vdf_bytes"], "l2": "VDF (%.1f GB) larger than L2" % (rep["vdf_bytes"] / 1e9),
                       "presolve_blocks": rep0["presolve_blocks"], "eps_last": rep["eps"],
                       "sweep_tile": s.tuning_info(),
                       "phase_ms_per_step": {k: v / args.steps for k, v in rep["phase_ms"].items() if v > 0}},
            "roofline": roof, "clocks": ck, "gpu_launches": rep["kernel_launches"]}
    s.close()
    if not args.no_e2e:
        line["e2e"] = e2e(args, case, stream)
    if not args.no_converge and args.config in ("cylinder", "cylinder_full", "shock"):
        line["time_to_converged"] = time_to_converged(args, case, stream)
    if rank == 0 and not args.no_cpu_baseline:
        v, dt, nd, nv, nc = cpu_baseline(args.config)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": "one GSIS iteration of the FP64 oracle on a %d-cell sample of the workload "
                                          "(%d DVM cells, %d velocities), %.1f s" % (nc, nd, nv, dt)}
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    """64 independent shocks advanced together through gsis_iterate_batch."""
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    from workloads import shock_batch_cases
    from paper_2501_02245_gb300 import Solver, iterate_batch, batch_info
    cases = shock_batch_cases()
    stream = torch.cuda.Stream()
    solvers = [Solver.from_case(c, vdf_dtype=c.extra["vdf_dtype"], stream=stream) for c in cases]
    iterate_batch(solvers, max(args.warmup, 1))   # first call: start, autotune, record the graph
    clocks = Clocks(local)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    reps = iterate_batch(solvers, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    pts_iter = sum(r["n_dvm"] * r["n_v"] for r in reps)
    value, t_max = combine_ranks(pts_iter * args.steps, ms, pg, "cuda")
    sweep_ms = reps[0]["phase_ms"]["sweep"]
    eb = {"f32": 4, "bf16": 2}
    bytes_alg = sum(2 * 2 * eb[c.extra["vdf_dtype"]] * r["n_dvm"] * r["n_v"] for c, r in zip(cases, reps))
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
        peaks = json.load(fh)
    achieved = bytes_alg / (sweep_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": traffic_from_profile("batch", "mixed"),
            "kernel": "k_sweep_batch (both Gauss-Seidel passes of all 64 solves, one launch)",
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)",
            "algorithmic": "2 passes x 2 x b bytes per (cell, velocity), b = 4 (FP32) / 2 (BF16)"}
    info = batch_info(solvers)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32/bf16", "data": "synthetic",
            "config": {"workload": workload_name("batch", "mixed"), "parallelism": "replicas" if ws > 1 else "1 GPU",
                       "n_solves": len(cases), "points_per_iteration": pts_iter,
                       "vdf_bytes": sum(r["vdf_bytes"] for r in reps),
                       "l2": "VDFs (%.1f GB) larger than L2" % (sum(r["vdf_bytes"] for r in reps) / 1e9),
                       "plan": info, "eps_max_last": max(r["eps"] for r in reps),
                       "sweep_ms_per_step": sweep_ms},
            "roofline": roof, "clocks": ck, "gpu_launches": reps[0]["kernel_launches"]}
    for sv in solvers:
        sv.close()
    if not args.no_e2e:
        torch.cuda.synchronize()
        t = time.perf_counter()
        sol2 = [Solver.from_case(c, vdf_dtype=c.extra["vdf_dtype"], stream=stream) for c in cases]
        r2 = iterate_batch(sol2, args.steps)
        Ws = [sv.W() for sv in sol2]
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        for sv in sol2:
            sv.close()
        line["e2e"] = {"value": sum(r["n_dvm"] * r["n_v"] for r in r2) * args.steps / dt, "unit": UNIT,
                       "h2d_bytes_per_step": sum(mesh_bytes(c) for c in cases) // args.steps,
                       "d2h_bytes_per_step": sum(W.nbytes for W in Ws) // args.steps,
                       "includes": "set-up upload of 64 solves, autotuning and graph recording, %d iterations, "
                                   "result read-back" % args.steps}
    if rank == 0 and not args.no_cpu_baseline:
        v, dt, nd, nv, nc = cpu_baseline("batch")
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": "one GSIS iteration of the FP64 oracle on one shock of the batch reduced "
                                          "to %d cells (%d velocities), %.1f s" % (nc, nv, dt)}
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def time_to_converged(args, case, stream, thresholds=(1e-3, 2e-4), cap=80):
    """Wall-clock time (device synchronised) from a fresh context (host data,
    presolve, region) until the residual of Sec. 4 first falls below each
    threshold, at most `cap` GSIS iterations.  The 1e-6 criterion of the paper
    is not reached by these runs (see the convergence status in the design
    notes), so the precision forms are compared at these thresholds."""
    import torch
    from paper_2501_02245_gb300 import Solver
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = Solver.from_case(case, vdf_dtype=args.dtype, stream=stream)
    s.iterate(0)
    torch.cuda.synchronize()
    out = {"criterion": "epsilon of Sec. 4 between consecutive iterations", "cap": cap,
           "start_s": time.perf_counter() - t0, "reached": {}}
    eps_min = 1e300
    it = 0
    for it in range(cap):
        r = s.iterate(1)
        eps_min = min(eps_min, r["eps"])
        for th in thresholds:
            key = "%.0e" % th
            if key not in out["reached"] and r["eps"] < th:
                torch.cuda.synchronize()
                out["reached"][key] = {"iterations": it + 1, "seconds": time.perf_counter() - t0}
        if len(out["reached"]) == len(thresholds):
            break
    out["eps_min"] = eps_min
    out["iterations_run"] = it + 1
    s.close()
    return out


def e2e(args, case, stream):
    """The same metric through the public API from host data: context creation,
    mesh and velocity-grid upload (host -> device), the adaptive start, the
    timed iterations, and the macroscopic result read back to the host."""
    import torch
    from paper_2501_02245_gb300 import Solver
    torch.cuda.synchronize()
    t = time.perf_counter()
    s = Solver.from_case(case, vdf_dtype=args.dtype, stream=stream)
    s.iterate(0)
    rep = s.iterate(args.steps)
    W = s.W()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    s.close()
    pts = rep["n_dvm"] * rep["n_v"] * args.steps
    return {"value": pts / dt, "unit": UNIT, "h2d_bytes_per_step": mesh_bytes(case) // args.steps,
            "d2h_bytes_per_step": (W.nbytes + 16 * args.steps) // args.steps,
            "includes": "set-up upload, NS presolve and region, %d iterations, result read-back" % args.steps}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.config == "batch":
        return run_batch(args)
    return run_gsis(args)


if __name__ == "__main__":
    sys.exit(main())
