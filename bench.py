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
                    choices=["cylinder", "shock", "cylinder_full", "cylinder_reduced", "sphere", "cylinder32",
                             "batch"])
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32", "bf16", "f16"])
    ap.add_argument("--tile", default=None,
                    help="run the sweep with this tile shape instead of the autotuned one (for profiler captures)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-converge", action="store_true", help="skip the time-to-converged measurement")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the reduced-precision forms and the full-kinetic arm (default cylinder run)")
    ap.add_argument("--no-peaks", action="store_true", help="skip the FMA peak probe (derived FP64 peak instead)")
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
    if config in ("cylinder", "cylinder_full", "cylinder_reduced"):
        adaptive = config != "cylinder_full"
        reduced = config == "cylinder_reduced"
        if small:
            return cylinder_case(n_r=12, n_theta=12, presolve_max_blocks=1, macro_steps=20, adaptive=adaptive,
                                 reduced=reduced)
        return cylinder_case(adaptive=adaptive, reduced=reduced)
    if small:
        return sphere_case(n_r=6, n_pol=4, n_az=4, presolve_max_blocks=1, macro_steps=10)
    return sphere_case()


def workload_name(config, dtype):
    return {
        "cylinder": "2D cylinder Ma=5 Kn=0.01 Tw=2, O-grid 128x128, velocity grid 48x48x24, adaptive Kn_ref=0.01",
        "cylinder_full": "2D cylinder Ma=5 Kn=0.01 Tw=2, O-grid 128x128, velocity grid 48x48x24, full kinetic",
        "cylinder_reduced": "2D cylinder Ma=5 Kn=0.01 Tw=2, O-grid 128x128, reduced distributions (xi_z "
                            "integrated out) on a 48x48 velocity grid, adaptive Kn_ref=0.01",
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


def traffic_per_point(config, dtype):
    """DRAM bytes per (cell, velocity) point of one sweep launch, from the
    committed ncu summary, if it was taken on the current sweep source (else
    None)."""
    p = os.path.join(ROOT, "profiles", "sweep_%s_%s.json" % (config, dtype))
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    sha = source_sha(["paper_2501_02245_gb300/csrc/sweep.cu", "paper_2501_02245_gb300/csrc/sweep_device.cuh",
                      "paper_2501_02245_gb300/csrc/sweep_pair.cuh", "paper_2501_02245_gb300/csrc/gsis_device.cuh"])
    if d.get("sweep_src_sha") != sha:
        return None
    return d.get("dram_bytes_per_point")


def _cpu_model():
    """CPU model name of this host (for the record of the CPU baseline)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _oracle_sample(config, steps):
    """One worker of the CPU baseline: the oracle as it stands on the bounded
    sample of the workload (set-up untimed), `steps` GSIS iterations timed.
    Returns (points, seconds, n_dvm, n_v, n_cells)."""
    from oracle.gsis import OracleSolver
    case = make_case(config, small=True)
    o = OracleSolver(case)
    o.initialise()
    t = time.perf_counter()
    pts = 0
    for _ in range(steps):
        o.step()
        pts += int(o.dvm.sum()) * o.vg.nv
    return pts, time.perf_counter() - t, int(o.dvm.sum()), o.vg.nv, case.mesh.ncell


def cpu_baseline(config, steps=1, cores=None):
    """The oracle as it stands, timed on every host core: one independent
    instance of the bounded sample per core (a process pool started with
    `spawn`, one BLAS thread each), throughput = all points of all instances
    over the wall time of the slowest.  Returns (updates/s, seconds, n_dvm,
    n_v, n_cells, cores, cpu model)."""
    import multiprocessing as mp
    cores = cores or os.cpu_count() or 1
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        t0 = time.perf_counter()
        res = pool.starmap(_oracle_sample, [(config, steps)] * cores)
        wall = time.perf_counter() - t0
    pts = sum(r[0] for r in res)
    slowest = max(r[1] for r in res)
    _, _, nd, nv, nc = res[0]
    return pts / slowest, slowest, nd, nv, nc, cores, _cpu_model(), wall


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands on every host core of
    rank 0, each core running its own instance of the bounded sample of the
    workload (warm-up iterations untimed, then `steps` timed ones)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import multiprocessing as mp
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    cores = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.starmap(_oracle_reference_steps, [(args.config, args.warmup, args.steps)] * cores)
    pts = sum(r[0] for r in res)
    dt = max(r[1] for r in res)
    value = pts / dt
    nd, nv, nc = res[0][2], res[0][3], res[0][4]
    sample = ("%d independent instances (one per host core, %s) of the FP64 oracle, each one GSIS iteration per "
              "step on a %d-cell %s sample (%d DVM cells) with the workload's velocity grid (%d velocities)"
              % (cores, _cpu_model(), nc, args.config, nd, nv))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.config, args.dtype), "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu": _cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _oracle_reference_steps(config, warmup, steps):
    from oracle.gsis import OracleSolver
    case = make_case(config, small=True)
    o = OracleSolver(case)
    o.initialise()
    for _ in range(warmup):
        o.step()
    t = time.perf_counter()
    pts = 0
    for _ in range(steps):
        o.step()
        pts += int(o.dvm.sum()) * o.vg.nv
    return pts, time.perf_counter() - t, int(o.dvm.sum()), o.vg.nv, case.mesh.ncell


def mesh_bytes(case):
    m = case.mesh
    b = m.centers.nbytes + m.volumes.nbytes + sum(a.nbytes for a in m.S) + sum(a.nbytes for a in m.xf)
    return b + case.W0.nbytes


def measured_alu_peaks(stream, local):
    """FP64 and FP32 FMA throughput of this GPU's CUDA cores, measured by the
    library's probe kernel (CUDA events, best of four ~40 ms launches), with
    the SM clock sampled during the probes."""
    from paper_2501_02245_gb300.gsis import fma_peak
    clocks = Clocks(local)
    clocks.start()
    out = {}
    try:
        for name, fp64 in (("fp64", True), ("fp32", False)):
            r, ms = fma_peak(fp64, stream)
            out[name + "_tflops"] = r / 1e12
            out[name + "_launch_ms"] = ms
    finally:
        ck = clocks.stop()
    out["clocks"] = ck
    out["how"] = ("8 independent FMA chains per thread, 8 CTAs x 256 threads per SM, 2 flop per FMA; "
                  "k_fma_probe in paper_2501_02245_gb300/csrc/peaks.cu")
    if ck.get("sm_mhz"):
        out["derived_fp64_tflops_at_sampled_clock"] = 152 * 4 * ck["sm_mhz"] * 1e6 / 1e12
    return out


def sweep_roofline(args, rep, steps, peaks, traffic):
    """Roofline of the dominant kernel (the kinetic sweep) in the unit of one
    GSIS iteration -- every (cell, velocity) point updated once: read f once,
    write f once (2b bytes), one point update's flops -- over the measured
    duration of the sweep launches of one iteration (two Gauss-Seidel passes
    on 2D/3D meshes), with the same figures per pass beside it."""
    sweep_ms_iter = rep["phase_ms"]["sweep"] / steps
    launches_iter = rep["sweep_launches"] / steps
    pts = rep["n_dvm"] * rep["n_v"]
    eb = {"f64": 8, "f32": 4, "bf16": 2, "f16": 2}[args.dtype]
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
        mp = json.load(fh)
    trf = None if traffic is None else traffic * pts * launches_iter   # per GSIS iteration, like achieved
    if args.dtype == "f64":
        fpp = SWEEP_FLOPS_PER_POINT_1D if args.config == "shock" else SWEEP_FLOPS_PER_POINT_2D
        peak = peaks.get("fp64_tflops") if peaks else None
        src = "measured FP64 FMA throughput (gsis_probe_fma_peak, this run)"
        if not peak:
            peak, src = FP64_PEAK_TFLOPS, "FP64 unit counts x clock: 152 SMs x 2 DFMA/clk x 2.07 GHz (derived)"
        achieved = fpp * pts / (sweep_ms_iter * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": trf, "kernel": "k_sweep<double>", "peak_source": src,
                "per": "GSIS iteration: %g sweep launches (Gauss-Seidel passes) per iteration" % launches_iter,
                "algorithmic": "%d FP64 flop per (cell, velocity) per GSIS iteration (one point update)" % fpp,
                "per_pass": {"achieved": achieved * launches_iter, "frac": achieved * launches_iter / peak,
                             "algorithmic": "%d FP64 flop per (cell, velocity) per pass" % fpp},
                "hbm_frac": 2 * eb * pts / (sweep_ms_iter * 1e-3) / 1e9 / mp["hbm_gbs"]}
    else:
        achieved = 2 * eb * pts / (sweep_ms_iter * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": mp["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / mp["hbm_gbs"], "traffic": trf, "kernel": "k_sweep",
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth)",
                "per": "GSIS iteration: %g sweep launches (Gauss-Seidel passes) per iteration" % launches_iter,
                "algorithmic": "2 x %d bytes per (cell, velocity) per GSIS iteration (read f once, write once)" % eb,
                "per_pass": {"achieved": achieved * launches_iter, "frac": achieved * launches_iter / mp["hbm_gbs"],
                             "algorithmic": "2 x %d bytes per (cell, velocity) per pass" % eb}}
        if peaks and peaks.get("fp32_tflops"):
            fpp = SWEEP_FLOPS_PER_POINT_1D if args.config == "shock" else SWEEP_FLOPS_PER_POINT_2D
            roof["fp32_alu_frac_per_pass"] = fpp * pts * launches_iter / (sweep_ms_iter * 1e-3) / 1e12 / peaks[
                "fp32_tflops"]
    return roof


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
    reference_state = (s.W(), s.moments(["wall_q"])["wall_q"], args.warmup + args.steps)
    tuning = s.tuning_info()
    s.close()
    peaks = None
    if not args.no_peaks:
        try:
            peaks = measured_alu_peaks(stream, local)
        except Exception as exc:   # the roofline then falls back to the derived FP64 peak, and says so
            peaks = {"error": str(exc)}
    roof = sweep_roofline(args, rep, args.steps, peaks, traffic_per_point(args.config, args.dtype))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": workload_name(args.config, args.dtype), "parallelism": "replicas" if ws > 1 else "1 GPU",
                       "n_dvm": rep["n_dvm"], "n_cells": case.mesh.ncell, "n_v": rep["n_v"],
                       "vdf_bytes": rep["vdf_bytes"], "l2": "VDF (%.1f GB) larger than L2" % (rep["vdf_bytes"] / 1e9),
                       "presolve_blocks": rep0["presolve_blocks"], "presolve_ms": rep0["phase_ms"]["presolve"],
                       "eps_last": rep["eps"], "sweep_tile": tuning,
                       "phase_ms_per_step": {k: v / args.steps for k, v in rep["phase_ms"].items() if v > 0}},
            "roofline": roof, "measured_peaks": peaks, "clocks": ck, "gpu_launches": rep["kernel_launches"]}
    if not args.no_e2e:
        line["e2e"] = _arm(lambda: e2e(args, case, stream))
    converged_state = None
    if not args.no_converge and args.config in ("cylinder", "cylinder_full", "shock"):
        ttc = _arm(lambda: time_to_converged(args, case, stream, args.dtype, keep_state=True))
        if isinstance(ttc, tuple):
            line["time_to_converged"], converged_state = ttc
        else:
            line["time_to_converged"] = ttc
    if not args.no_forms and args.config == "cylinder" and args.dtype == "f64" and rank == 0:
        line["precision_forms"] = _arm(lambda: precision_forms(args, case, stream, reference_state,
                                                               line.get("time_to_converged"), t_max / args.steps,
                                                               converged_state))
        line["full_kinetic"] = _arm(lambda: full_kinetic_arm(args, stream, rep, t_max / args.steps))
        line["reduced_2d"] = _arm(lambda: reduced_arm(args, stream, rep, reference_state, t_max / args.steps))
        line["other_workloads"] = _arm(lambda: other_workloads(stream, local))
    if rank == 0 and not args.no_cpu_baseline:
        v, dt, nd, nv, nc, cores, cpu, wall = cpu_baseline(args.config)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu,
                                "sample": "%d independent instances of the FP64 oracle (one per host core), one GSIS "
                                          "iteration each on a %d-cell sample of the workload (%d DVM cells, %d "
                                          "velocities); slowest instance %.1f s" % (cores, nc, nd, nv, dt)}
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def _error_vs(Wr, qr, W, q):
    """Largest error of density, temperature (relative to their largest value)
    and wall heat flux (relative to its largest magnitude)."""
    def rel(a, b):
        return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
    return {"rho": rel(W[:, 0], Wr[:, 0]), "T": rel(W[:, 4], Wr[:, 4]), "wall_q": rel(q, qr)}


def _arm(fn):
    """One auxiliary measurement of the JSON line: its result, or the solver's
    error status (a run that stopped with GSIS_ERR_NONFINITE, say) recorded in
    its place, so that the headline line is still printed."""
    from paper_2501_02245_gb300 import GsisError
    try:
        return fn()
    except GsisError as e:
        return {"error": str(e)}


def precision_forms(args, case, stream, reference_state, f64_ttc, f64_ms_per_iter, converged_state=None):
    """The cylinder with FP32, BF16 and FP16 VDF storage (FP32 sweep
    arithmetic; FP64 moments, conservation correction and synthetic solve):
    throughput, time to the residual thresholds from a fresh context, VDF
    memory, and the error in density, temperature and wall heat flux against
    the FP64 GPU run (the parity-tested path) after the same number of
    iterations from the same start: at the iteration where the FP64 run first
    reached epsilon < 2e-4 (near the steady state; the headline error), and
    early in the transient (the benchmark's warm-up + timed iterations, where
    a small shift of the transient dominates the difference)."""
    import torch
    from paper_2501_02245_gb300 import Solver, GsisError
    Wr, qr, n_ref = reference_state
    out = {"reference": "FP64 GPU run of this benchmark after %d GSIS iterations" % n_ref}
    n_conv = None
    if converged_state is not None:
        Wc, qc, n_conv = converged_state
        out["reference_converged"] = ("FP64 GPU run from a fresh context after %d GSIS iterations (its first "
                                      "epsilon < 2e-4)" % n_conv)
    thresholds = (1e-3, 2e-4, 1e-4)
    for dt in ("f32", "bf16", "f16"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = Solver.from_case(case, vdf_dtype=dt, stream=stream)
        s.iterate(0)
        reached, err, err_conv, it_ms = {}, None, None, []
        eps_min = 1e300
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        n_dvm = vdf = 0
        stopped = None
        for it in range(max(n_ref, n_conv or 0, 100)):
            e0.record(stream)
            try:
                r = s.iterate(1)
            except GsisError as e:   # recorded, and the other forms still run
                stopped = "iteration %d: %s" % (it + 1, e)
                break
            e1.record(stream)
            torch.cuda.synchronize()
            if it >= 2:
                it_ms.append(e0.elapsed_time(e1))
            n_dvm, vdf = r["n_dvm"], r["vdf_bytes"]
            eps_min = min(eps_min, r["eps"])
            for th in thresholds:
                k = "%.0e" % th
                if k not in reached and r["eps"] < th:
                    reached[k] = {"iterations": it + 1, "seconds": time.perf_counter() - t0}
            if it + 1 == n_ref:
                err = _error_vs(Wr, qr, s.W(), s.moments(["wall_q"])["wall_q"])
            if n_conv is not None and it + 1 == n_conv:
                err_conv = _error_vs(Wc, qc, s.W(), s.moments(["wall_q"])["wall_q"])
            if it + 1 >= max(n_ref, n_conv or 0) and len(reached) == len(thresholds):
                break
        s.close()
        ms_it = float(np.median(it_ms)) if it_ms else None
        d = {"ms_per_iteration": ms_it, "updates_per_s": n_dvm * case.vgrid.nv / (ms_it * 1e-3) if ms_it else None,
             "vdf_bytes": vdf, "error_vs_f64": err_conv, "error_vs_f64_early": err,
             "time_to_converged": reached, "eps_min": eps_min}
        if stopped:
            d["stopped"] = stopped
        if f64_ms_per_iter and ms_it:
            d["speedup_per_iteration_vs_f64"] = f64_ms_per_iter / ms_it
        if f64_ttc:
            d["speedup_to_threshold_vs_f64"] = {
                k: f64_ttc["reached"][k]["seconds"] / v["seconds"] for k, v in reached.items()
                if k in f64_ttc.get("reached", {})}
        out[dt] = d
    return out


def reduced_arm(args, stream, rep_3d, reference_state, ms_per_iter_3d, steps=5):
    """The cylinder with the reduced distributions of a 2D flow (xi_z
    integrated out: G and H on the 48 x 48 (xi_x, xi_y) grid, the paper's 2D
    memory saver) against the 3D velocity grid: throughput, VDF memory, time
    to the residual thresholds, and the largest difference of density,
    temperature and wall heat flux from the 3D run after the same number of
    iterations (two discretisations of the same flow: the reduced one is
    exact in xi_z)."""
    import torch
    from paper_2501_02245_gb300 import Solver
    Wr, qr, n_ref = reference_state
    case = make_case("cylinder_reduced")
    case.tol = 0.0
    s = Solver.from_case(case, vdf_dtype=args.dtype, stream=stream)
    s.iterate(0)
    s.iterate(n_ref - steps)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r = s.iterate(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    diff = _error_vs(Wr, qr, s.W(), s.moments(["wall_q"])["wall_q"])
    s.close()
    out = {"workload": workload_name("cylinder_reduced", args.dtype), "ms_per_iteration": ms,
           "updates_per_s": r["n_dvm"] * r["n_v"] / (ms * 1e-3), "n_dvm": r["n_dvm"], "n_v": r["n_v"],
           "vdf_bytes": r["vdf_bytes"], "vdf_fraction_of_3d": r["vdf_bytes"] / rep_3d["vdf_bytes"],
           "time_per_iteration_fraction_of_3d": ms / ms_per_iter_3d,
           "phase_ms_per_step": {k: v / steps for k, v in r["phase_ms"].items() if v > 0},
           "difference_from_3d_after_%d_iterations" % n_ref: diff}
    if not args.no_converge:
        out["time_to_converged"] = time_to_converged(args, case, stream, args.dtype, cap=60)
    return out


def _single(config, dtype, stream, warmup, steps):
    """Throughput of one single-solve workload (warm-up iterations untimed,
    then `steps` timed with CUDA events on the library's stream)."""
    import torch
    from paper_2501_02245_gb300 import Solver
    case = make_case(config)
    case.tol = 0.0
    s = Solver.from_case(case, vdf_dtype=dtype, stream=stream)
    r0 = s.iterate(0)
    s.iterate(warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r = s.iterate(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    s.close()
    eb = {"f64": 8, "f32": 4, "bf16": 2, "f16": 2}[dtype]
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
        hbm = json.load(fh)["hbm_gbs"]
    sweep_ms = r["phase_ms"]["sweep"] / steps
    pts = r["n_dvm"] * r["n_v"]
    return {"workload": workload_name(config, dtype), "ms_per_iteration": ms,
            "updates_per_s": pts / (ms * 1e-3), "n_dvm": r["n_dvm"], "n_v": r["n_v"], "vdf_bytes": r["vdf_bytes"],
            "presolve_ms": r0["phase_ms"]["presolve"],
            "phase_ms_per_step": {k: v / steps for k, v in r["phase_ms"].items() if v > 0},
            "sweep_hbm_frac_per_iteration": 2 * eb * pts / (sweep_ms * 1e-3) / 1e9 / hbm, "eps_last": r["eps"]}


def _batch(stream, steps=3):
    """The 64-shock batch through gsis_iterate_batch (first call: start,
    autotuning, graph recording; then `steps` timed iterations)."""
    import torch
    from workloads import shock_batch_cases
    from paper_2501_02245_gb300 import Solver, iterate_batch
    cases = shock_batch_cases()
    solvers = [Solver.from_case(c, vdf_dtype=c.extra["vdf_dtype"], stream=stream) for c in cases]
    iterate_batch(solvers, 1)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    reps = iterate_batch(solvers, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    for sv in solvers:
        sv.close()
    pts = sum(r["n_dvm"] * r["n_v"] for r in reps)
    eb = {"f32": 4, "bf16": 2}
    bytes_alg = sum(2 * eb[c.extra["vdf_dtype"]] * r["n_dvm"] * r["n_v"] for c, r in zip(cases, reps))
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
        hbm = json.load(fh)["hbm_gbs"]
    sweep_ms = reps[0]["phase_ms"]["sweep"]
    return {"workload": workload_name("batch", "mixed"), "ms_per_iteration": ms, "updates_per_s": pts / (ms * 1e-3),
            "points_per_iteration": pts, "vdf_bytes": sum(r["vdf_bytes"] for r in reps), "sweep_ms": sweep_ms,
            "sweep_hbm_frac_per_iteration": bytes_alg / (sweep_ms * 1e-3) / 1e9 / hbm}


def other_workloads(stream, local):
    """The other configurations, measured in the same run: the 1D Ma 2 shock
    (FP64, 200 cells, 48 x 24 x 24), the 3D sphere (BF16 VDF, 96 x 64 x 64,
    48^3) and the 64-shock batch (FP32/BF16)."""
    import torch
    clocks = Clocks(local)
    clocks.start()
    out = {}
    try:
        out["shock_f64"] = _single("shock", "f64", stream, 3, 5)
        out["batch"] = _batch(torch.cuda.Stream())
        out["sphere_bf16"] = _single("sphere", "bf16", stream, 2, 3)
    except Exception as exc:   # reported, not hidden: the headline line still prints
        out["error"] = "%s: %s" % (type(exc).__name__, exc)
    out["clocks"] = clocks.stop()
    return out


def full_kinetic_arm(args, stream, rep_adaptive, adaptive_ms_per_iter, steps=3):
    """The other arm of the cylinder configuration: every cell kinetic (no
    adaptation), same mesh, velocity grid and precision: throughput, VDF
    memory and time to the residual thresholds, against the adaptive run."""
    import torch
    from paper_2501_02245_gb300 import Solver
    case = make_case("cylinder_full")
    case.tol = 0.0
    s = Solver.from_case(case, vdf_dtype=args.dtype, stream=stream)
    s.iterate(0)
    s.iterate(2)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r = s.iterate(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    s.close()
    out = {"workload": workload_name("cylinder_full", args.dtype), "ms_per_iteration": ms,
           "updates_per_s": r["n_dvm"] * r["n_v"] / (ms * 1e-3), "n_dvm": r["n_dvm"], "vdf_bytes": r["vdf_bytes"],
           "adaptive_vdf_fraction": rep_adaptive["vdf_bytes"] / r["vdf_bytes"],
           "adaptive_time_per_iteration_fraction": adaptive_ms_per_iter / ms}
    if not args.no_converge:
        out["time_to_converged"] = time_to_converged(args, case, stream, args.dtype, cap=60)
    return out


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
    torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    reps = iterate_batch(solvers, args.steps)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
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
            "frac": achieved / peaks["hbm_gbs"], "traffic": None,
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
        v, dt, nd, nv, nc, cores, cpu, wall = cpu_baseline("batch")
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu,
                                "sample": "%d independent instances of the FP64 oracle (one per host core), one GSIS "
                                          "iteration each on one shock of the batch reduced to %d cells (%d "
                                          "velocities); slowest instance %.1f s" % (cores, nc, nv, dt)}
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def time_to_converged(args, case, stream, dtype, thresholds=(1e-3, 2e-4, 1e-4), cap=100, keep_state=False):
    """Wall-clock time (device synchronised) from a fresh context (host data,
    presolve, region) until the residual of Sec. 4 first falls below each
    threshold, at most `cap` GSIS iterations.  The 1e-6 criterion of the paper
    is not reached by these runs (see the convergence status in the design
    notes), so the precision forms are compared at these thresholds.  With
    keep_state the state (W, wall heat flux) of the last iteration is returned
    beside the report (not in it)."""
    import torch
    from paper_2501_02245_gb300 import Solver
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = Solver.from_case(case, vdf_dtype=dtype, stream=stream)
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
    state = (s.W(), s.moments(["wall_q"])["wall_q"], it + 1) if keep_state else None
    s.close()
    return (out, state) if keep_state else out


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
