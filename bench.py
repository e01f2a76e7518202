"""Benchmark of the SRMC backward solve on GB300.

One step = one whole backward solve of Alg. SRMDP (N step launches over all
strata) on the selected workload, inputs already resident on the device.
The metric is stratum-path-steps per second: K M N (N+1) / 2 units per solve.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload cfg5]
                  [--impl reference] [--no-cpu-baseline]

With N > 1 (torchrun, one process per GPU) every rank solves its own
independent instance (replicas, weak scaling, no collective on the data
path); value = units of all ranks / max elapsed over ranks.
The reference arm (--impl reference) times the FP64 CPU oracle on a bounded
sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2407_21085_gb300 import workloads as W  # noqa: E402

METRIC = "stratum-path-steps/s"
UNIT = "path-steps/s"
L2_FLUSH_BYTES = 512 << 20


def flops_per_path_step(d: int) -> float:
    """Algorithmic FP32 FLOPs of one stratum-path-step: Euler, locate, centre,
    y and z evaluation, clamps, driver and response update (2 d^2 + 13 d + 20)
    plus the q = d normals by inversion (a degree-9 polynomial: 18 each)."""
    return 2.0 * d * d + 13.0 * d + 20.0 + 18.0 * d


def z_eval_flops(d: int) -> float:
    """The part of flops_per_path_step that evaluates z at every path-step: the
    d (d + 1) multiply-adds of the z row and the 2 d of its clamps.  A driver that
    does not read z (the cos model without kapz) needs none of it."""
    return 2.0 * d * (d + 1) + 2.0 * d


def fp32_peak_tflops(sms: int, mhz: float) -> float:
    """FP32 FMA pipe peak from unit counts: SMs x 128 lanes x 2 FLOP x clock."""
    return sms * 128 * 2 * mhz * 1e6 / 1e12


def measured_fp32_peak(sms: int, stream, iters: int = 400000, reps: int = 3):
    """FP32 FMA throughput measured with the library's probe kernel
    (srmc_fp32_fma_probe: independent FFMA2 or FFMA chains, 4 blocks of 256
    threads per SM), best of reps CUDA-event timings per form; returns
    {"tflops": max over forms, "packed": ..., "scalar": ...}."""
    import torch
    from paper_2407_21085_gb300 import srmc
    grid, threads = 4 * sms, 256
    out = torch.empty(grid * threads, dtype=torch.float32, device="cuda")
    res = {}
    for packed, name in ((1, "packed"), (0, "scalar")):
        srmc.srmc_fp32_fma_probe(grid, threads, 1000, packed, out, stream)
        best = 0.0
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            srmc.srmc_fp32_fma_probe(grid, threads, iters, packed, out, stream)
            b.record(stream)
            b.synchronize()
            best = max(best, grid * threads * iters * 32.0 / (a.elapsed_time(b) / 1e3) / 1e12)
        res[name] = best
    res["tflops"] = max(res["packed"], res["scalar"])
    return res


STEP_KERNEL_SOURCES = ("srmc_step.cu", "srmc_device.cuh", "srmc_internal.h")


def kernel_source_hash() -> str:
    """sha256 of the sources the step kernel is compiled from (a traffic record
    taken from an ncu capture is used only while this hash matches)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2407_21085_gb300", "csrc")
    for name in STEP_KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode() + b"\0" + fh.read())
    return h.hexdigest()


def recorded_traffic(workload_name: str, control):
    """DRAM bytes per step-kernel launch from profiles/step_kernel_traffic.json
    (written from an ncu capture of the same build and workload), else None."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    for e in rec.get("records", []):
        if (e.get("workload") == workload_name and e.get("control", False) == control
                and e.get("kernel_source_sha256") == kernel_source_hash()):
            return e.get("dram_bytes_per_launch")
    return None


def control_kind(args):
    """False (plain), True (tabulated control rows) or "own" (the run's own z)."""
    return "own" if args.control_own else bool(args.control_random)


def install_control(args, solver, stream):
    """--control-random: the timed kernel becomes the control-variate step
    kernel with rows tabulated from an untrained network (its cost does not
    depend on them); --control-own: the kernel with the run's own z control."""
    from paper_2407_21085_gb300 import srmc
    if args.control_own:
        solver.srmc_set_own_control()
    elif args.control_random:
        net = srmc.MLP(solver.w.d + 1, seed=args.seed)
        net.srmc_cv_tabulate(solver, stream)
        net.close()


def workload(name: str) -> W.Workload:
    makers = {"cfg1": W.cfg1, "cfg2": W.cfg2, "cfg2_fp64": lambda: W.cfg2(precision="fp64"),
              "cfg2_lp0": lambda: W.cfg2(basis="lp0"), "cfg3": W.cfg3, "cfg5": W.cfg5,
              "cfg5_M1024": lambda: W.cfg5(M=1024, name="cfg5_d6_K262144_N40_M1024"),
              # reduced-M cases of the same kernels, for profiler captures
              "cfg3_M2048": lambda: W.cfg3(M=2048, name="cfg3_d4_K20736_N50_M2048"),
              "cfg5_M512": lambda: W.cfg5(M=512, name="cfg5_d6_K262144_N40_M512"),
              # same cell width as cfg5 (0.75) on a smaller box, for profiler captures
              "cfg5_small_M512": lambda: W.cfg5(M=512, C=5, a=1.875, name="cfg5small_d6_K15625_N40_M512"),
              "cfg5_small": lambda: W.cfg5(C=5, a=1.875, name="cfg5small_d6_K15625_N40_M4096")}
    return makers[name]()


# ---- distributed plumbing (replicas only) -----------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, backend_device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=backend_device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_workload(name: str, rank: int) -> W.Workload:
    """The replica solved by rank r: the named workload with its own Philox
    instance (instance + 1000 r), so that ranks draw independent clouds."""
    w = workload(name)
    return w.replace(instance=w.instance + 1000 * rank)


def whole_job_rate(units_per_rank: int, world: int, steps: int, local_ms: float, device=None):
    """Units of all ranks / the slowest rank's elapsed time (weak scaling:
    every rank solves its own instance of the same size); returns (rate, max ms)."""
    max_ms = max_over_ranks(local_ms, device)
    return units_per_rank * world * steps / (max_ms / 1e3), max_ms


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ---- clocks during the timed region -----------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        with open(self.path) as fh:
            lines = fh.readlines()
        os.unlink(self.path)
        return summarize_clocks(lines)


THROTTLE_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")


def summarize_clocks(lines):
    """Median SM clock, maximum SM clock and the throttle reasons seen in
    nvidia-smi samples of ClockSampler.FIELDS (CSV, no header, no units);
    None when no complete sample was taken.  Fields that are not numbers
    (e.g. "[N/A]") are left out of the clock figures."""
    rows = []
    for line in lines:
        v = [a.strip() for a in line.split(",")]
        if len(v) >= 9:
            rows.append(v)
    if not rows:
        return None
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    reasons = sorted({THROTTLE_REASONS[c] for r in rows for c in range(4) if r[5 + c].lower() == "active"})
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons, "samples": len(rows)}


# ---- the GPU arm ---------------------------------------------------------------
def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2407_21085_gb300 import srmc

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count

    w = rank_workload(args.workload, rank)
    units = w.path_steps()
    stream = torch.cuda.current_stream()
    solver = srmc.Solver(w, block_threads=args.block_threads)
    install_control(args, solver, stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def one_step(events=None):
        if events is None:
            solver.srmc_solve(stream)
            return
        for i in range(w.N - 1, -1, -1):
            a, b = events[i]
            a.record(stream)
            solver.srmc_solve_step(i, stream)
            b.record(stream)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    launch_ms = []
    step_ms = []
    barrier()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.fill_(1.0)                     # evict the tables from L2 between steps
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(w.N)]
        one_step(ev)
        torch.cuda.synchronize()
        per = [ev[i][0].elapsed_time(ev[i][1]) for i in range(w.N)]
        launch_ms.extend(per)
        step_ms.append(ev[w.N - 1][0].elapsed_time(ev[0][1]))
    torch.cuda.synchronize()
    barrier()
    # the FP32 FMA peak of this GPU at this moment (inside the clock sampling window)
    fma_peak = measured_fp32_peak(sms, stream)
    clocks = sampler.stop()
    total_ms = sum(step_ms)
    value, total_ms_max = whole_job_rate(units, ws, args.steps, total_ms, dev)

    # End to end through the public API with host buffers: create (host
    # parameters -> device), solve, copy the FP64 coefficient tables to pinned
    # host memory, destroy.
    e2e_ms = []
    h2d = sum(w.cells) * 3 * (8 + 4) + (w.N + 1) * 2 * (8 + 4)
    info = solver.srmc_table()
    ny, nz = w.N * w.K * info["ry"], w.N * w.K * info["rz"]
    host_y = torch.empty(ny, dtype=torch.float64, pin_memory=True)
    host_z = torch.empty(nz, dtype=torch.float64, pin_memory=True)
    for r in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = srmc.Solver(w, block_threads=args.block_threads)
        install_control(args, s2, stream)
        s2.srmc_solve(stream)
        s2.srmc_read_table(host_y, host_z, stream)
        stream.synchronize()
        s2.close()
        if r > 0:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_value = whole_job_rate(units, ws, len(e2e_ms), sum(e2e_ms), dev)[0] if e2e_ms else None
    tab_bytes = (ny + nz) * 8

    # Roofline of the dominant kernel (the step kernel: every launch is one).
    avg_launch_s = (sum(launch_ms) / len(launch_ms)) / 1e3
    flops_per_launch = flops_per_path_step(w.d) * units / w.N
    achieved = flops_per_launch / avg_launch_s / 1e12
    peak_mhz = 2070.0
    peak_units = fp32_peak_tflops(sms, peak_mhz)
    peak = fma_peak["tflops"]
    reads_z = (w.model != "cos" or (len(w.params) > 2 and w.params[2] != 0.0) or control_kind(args) is not False
               or any(v != 0.0 for v in list(w.b or []) + list(w.theta or [])))
    needed = flops_per_path_step(w.d) - (0.0 if reads_z else z_eval_flops(w.d))

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if w.precision == "fp32" else "f64",
        "data": "synthetic",
        "config": {"workload": w.name + {False: "", True: " + control variate",
                                          "own": " + own-z control"}[control_kind(args)],
                   "d": w.d, "strata": w.K, "N": w.N, "M": w.M, "basis": w.basis,
                   "precision": w.precision, "model": "cos (u = e^{lam(T-t)} cos(sum x/sqrt d))",
                   "path_steps_per_solve": units, "l2": "flushed between steps (512 MiB write)",
                   "parallelism": f"replicas x{ws}", "block_threads": args.block_threads or "library"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "traffic": args.traffic if args.traffic is not None
                     else recorded_traffic(w.name, control_kind(args)),
                     "kernel": "step_kernel", "flops_per_unit": flops_per_path_step(w.d),
                     "peak_basis": "measured in this run: FP32 FMA probe kernel (srmc_fp32_fma_probe), "
                                   "best of packed FFMA2 and scalar FFMA chains",
                     "peak_probe": fma_peak,
                     "peak_unit_count": peak_units,
                     "frac_of_unit_count": achieved / peak_units,
                     "flops_per_unit_needed": needed,
                     "frac_of_needed_flops": achieved * needed / flops_per_path_step(w.d) / peak,
                     "needed_basis": "flops_per_unit less the z evaluation (z_eval_flops) when the driver "
                                     "does not read z and no control runs: the work this workload's "
                                     "kernel must do",
                     "unit_count_basis": f"{sms} SMs x 128 FP32 lanes x 2 x {peak_mhz:.0f} MHz"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": tab_bytes},
        "gpu_launches": w.N * args.steps,
        "clocks": clocks,
    }
    solver.close()
    return out, rank, w


# ---- the precision form (cfg3): FP32 paths + FP64 solves against all-FP64 ---------
def precision_compare(args, stream):
    """cfg3 (d = 4, 12^4 strata on [-3.5, 3.5]^4, N = 50, z in the driver): the FP32
    form (FP32 paths and moments, FP64 Cholesky solves) at full size, device-timed;
    then the FP32 error per result against the all-FP64 GPU form on the same Philox
    streams (the FP64 form matches the FP64 oracle within 1e-10 (1 + |y|) in the
    parity tests).  The FP32 form solves cfg3's shape with M = --prec-M; an FP64
    solver is given those rows (srmc_set_rows) and fits steps N-1, N/2 and 0 from
    them, so both fit each step from the same later functions (teacher forcing on
    the GPU); y and z are compared at every stratum centre and at the 2d points
    half a basis unit off it along each axis."""
    import torch
    from paper_2407_21085_gb300 import srmc

    def ev():
        return torch.cuda.Event(enable_timing=True)

    full = W.cfg3()
    s = srmc.Solver(full)
    s.srmc_solve(stream)
    torch.cuda.synchronize()
    ms = []
    for _ in range(2):
        a, b = ev(), ev()
        a.record(stream)
        s.srmc_solve(stream)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    s.close()
    sec = statistics.median(ms) / 1e3
    out = {"workload": full.name, "fp32_full": {"M": full.M, "s_per_solve": sec,
                                                "path_steps_per_s": full.path_steps() / sec}}

    w32 = W.cfg3(M=args.prec_M, name=f"cfg3_d4_K20736_N50_M{args.prec_M}")
    w64 = w32.replace(precision="fp64")
    s32 = srmc.Solver(w32)
    s32.srmc_solve(stream)
    t = s32.srmc_table()
    y32t = torch.empty((w32.N, w32.K, t["ry"]), dtype=torch.float64, device="cuda")
    z32t = torch.empty((w32.N, w32.K, t["rz"]), dtype=torch.float64, device="cuda")
    s32.srmc_read_table(y32t, z32t, stream)
    s64 = srmc.Solver(w64)
    for i in range(w64.N - 1, -1, -1):
        s64.srmc_set_rows(i, y32t[i], z32t[i], stream)
    ctr = s32.centres()
    unit = torch.tensor([(w32.hi[l] - w32.lo[l]) / w32.cells[l] / 2 for l in range(w32.d)],
                        dtype=torch.float64, device=ctr.device)
    pts = [ctr]
    for l in range(w32.d):
        for sgn in (-0.5, 0.5):
            p = ctr.clone()
            p[:, l] += sgn * unit[l]
            pts.append(p)
    pts = torch.cat(pts)
    steps = {}
    fp64_ms, fp64_units = 0.0, 0
    for i in (w64.N - 1, w64.N // 2, 0):
        a, b = ev(), ev()
        a.record(stream)
        s64.srmc_solve_step(i, stream)
        b.record(stream)
        b.synchronize()
        fp64_ms += a.elapsed_time(b)
        fp64_units += w64.K * w64.M * (w64.N - i)
        y32, z32 = s32.evaluate(i, pts)
        y64, z64 = s64.evaluate(i, pts)
        ey = (y32 - y64).abs() / (1 + y64.abs())
        ez = (z32 - z64).abs() / (1 + z64.abs())
        ezm = ez.max(dim=1).values
        centre = slice(0, ctr.shape[0])
        steps[str(i)] = {"y_max": float(ey.max()), "z_max": float(ez.max()),
                         "y_max_centres": float(ey[centre].max()), "z_max_centres": float(ez[centre].max()),
                         "y_rms": float((ey * ey).mean().sqrt()), "z_rms": float((ez * ez).mean().sqrt()),
                         "frac_points_within_1e-4": float(((ey <= 1e-4) & (ezm <= 1e-4)).double().mean())}
        s64.srmc_set_rows(i, y32t[i], z32t[i], stream)
    s32.close()
    s64.close()
    out["fp32_vs_fp64"] = {
        "M": args.prec_M, "points_per_step": int(pts.shape[0]), "by_step": steps,
        "fp64_path_steps_per_s": fp64_units / (fp64_ms / 1e3),
        "measure": "|d| / (1 + |FP64 value|) of y and of each z component; step i fitted in FP32 (the "
                   "FP32 form's own solve) and in FP64 (an FP64 solver given the FP32 solve's rows of "
                   "steps > i), same Philox streams"}
    return out


# ---- the second half of the metric: time to sup|y - u| <= eps, CV vs plain ------
def cv_compare(args, stream):
    """cfg5 (d = 6, 8^6 strata, N = 40): the plain scheme at M = 4096 against the
    learned control variate (coarse plain run at M = 256 -> train u_theta ->
    tabulate sigma grad u_theta -> CV run at M = 1024), with the plain scheme at
    M = 1024 as an ablation, and the run's own control (the fitted z of the
    later steps, no network) at M = 1024 as the zero-cost baseline of a
    control.  eps = the median over seeds 1..S of the sup error of the plain
    M = 4096 run against the closed form at the centres of the inner strata,
    over all steps; the CV form reaches eps when the median of its sup errors
    over the same seeds (each seed its own coarse run, network and CV run) is
    <= eps.  Wall times are host-measured with the device synchronised,
    set-up (allocation, graph capture) included; medians over the seeds.  The
    statistical error of a form is estimated from two independent cloud seeds
    (the same network for the CV form): rms(y_A - y_B) / sqrt(2) over the
    inner centres and all steps (the
    closed-form error also holds the O(dt) and LP1 biases, which no control
    variate removes)."""
    import torch
    from paper_2407_21085_gb300 import srmc

    w = W.cfg5() if not args.cv_small else W.cfg5(C=5, a=1.875, name="cfg5small_d6_K15625_N40_M4096")
    seeds = [w.seed + r for r in range(args.cv_seeds)]
    wcv = w.replace(M=args.cv_M)
    # load the d = 6 kernels (plain and CV) on a tiny problem first
    tiny = W.cos_model("warm", d=6, N=2, C=3, a=3.0, M=64, s0=0.3, lam=0.2, kap=0.5)
    ws = srmc.Solver(tiny); ws.srmc_solve(stream)
    wn = srmc.MLP(7, seed=0); wn.srmc_cv_tabulate(ws, stream); ws.srmc_solve(stream)
    ws.srmc_set_own_control(); ws.srmc_solve(stream)
    wn.srmc_mlp_fit(ws, n_data=4096, iters=2, batch=4096, lr=1e-3, seed=0, stream=stream)
    torch.cuda.synchronize()
    ws.close(); wn.close()

    cells = torch.stack(torch.meshgrid(*[torch.arange(c) for c in w.cells[::-1]], indexing="ij"), -1)
    cells = cells.reshape(-1, w.d).flip(-1).to("cuda")
    inner = ((cells > 0) & (cells < w.cells[0] - 1)).all(-1)

    def clock():
        torch.cuda.synchronize()
        return time.perf_counter()

    def values(solver):
        x = solver.centres()
        return torch.stack([solver.evaluate(i, x)[0][inner] for i in range(w.N)])

    def summary(solver, wall):
        e_in, e_all = solver.closed_form_error(inner=True), solver.closed_form_error()
        return {"M": solver.w.M, "seed": solver.w.seed, "wall_s": wall,
                "sup_err_inner": float(e_in[:, 0].max()),
                "rms_err_inner": float(math.sqrt(e_in[:, 1].mean())), "sup_err_all": float(e_all[:, 0].max())}

    def median_of(runs, key):
        return statistics.median(r[key] for r in runs)

    out = {"workload": w.name, "seeds": seeds,
           "metric": "wall time to sup|y - u| <= eps at inner stratum centres (all steps)"}
    plain_runs = []
    for sd in seeds:
        t0 = clock()
        sp = srmc.Solver(w.replace(seed=sd))
        sp.srmc_solve(stream)
        r = summary(sp, clock() - t0)
        r["path_steps_per_s"] = w.path_steps() / r["wall_s"]
        plain_runs.append(r)
        sp.close()
    plain = {"runs": plain_runs, "wall_s": median_of(plain_runs, "wall_s"),
             "sup_err_inner": median_of(plain_runs, "sup_err_inner"),
             "path_steps_per_s": median_of(plain_runs, "path_steps_per_s")}

    t0 = clock()
    sa = srmc.Solver(wcv)
    sa.srmc_solve(stream)
    abl = summary(sa, clock() - t0)
    ya = values(sa)
    sa.close()
    sb = srmc.Solver(wcv.replace(seed=w.seed + 1))
    sb.srmc_solve(stream)
    abl["stat_err_rms"] = float(((ya - values(sb)).pow(2).mean() / 2).sqrt())
    abl["sup_err_inner_seed2"] = float(sb.closed_form_error(inner=True)[:, 0].max())
    sb.close()

    t0 = clock()
    so = srmc.Solver(wcv)
    so.srmc_set_own_control()
    so.srmc_solve(stream)
    own = summary(so, clock() - t0)
    own["path_steps_per_s"] = wcv.path_steps() / own["wall_s"]
    yo = values(so)
    so.close()
    so = srmc.Solver(wcv.replace(seed=w.seed + 1))
    so.srmc_set_own_control()
    so.srmc_solve(stream)
    own["stat_err_rms"] = float(((yo - values(so)).pow(2).mean() / 2).sqrt())
    so.close()

    cv_runs, cv_vals = [], []
    for sd in seeds:
        stages = {}
        t0 = clock()
        co = srmc.Solver(w.replace(M=args.cv_coarse_M, seed=sd + 100))
        co.srmc_solve(stream)
        t1 = clock(); stages["coarse_solve"] = t1 - t0
        net = srmc.MLP(w.d + 1, seed=args.seed + sd)
        net.srmc_mlp_fit(co, n_data=args.cv_data, iters=args.cv_iters, batch=8192, lr=3e-3, seed=args.seed + sd,
                         stream=stream)
        t2 = clock(); stages["train"] = t2 - t1
        sc = srmc.Solver(wcv.replace(seed=sd))
        net.srmc_cv_tabulate(sc, stream)
        t3 = clock(); stages["tabulate"] = t3 - t2
        sc.srmc_solve(stream)
        t4 = clock(); stages["cv_solve"] = t4 - t3
        r = summary(sc, t4 - t0)
        r.update({"stages_s": stages, "cv_solve_path_steps_per_s": wcv.path_steps() / stages["cv_solve"]})
        cv_runs.append(r)
        if not cv_vals:
            # statistical error: the same network, a second independent cloud seed
            cv_vals.append(values(sc))
            sd2 = srmc.Solver(wcv.replace(seed=sd + 1))
            net.srmc_cv_tabulate(sd2, stream)
            sd2.srmc_solve(stream)
            cv_vals.append(values(sd2))
            sd2.close()
        sc.close(); co.close(); net.close()
    cv = {"runs": cv_runs, "coarse_M": args.cv_coarse_M, "train_points": args.cv_data,
          "train_iters": args.cv_iters, "wall_s": median_of(cv_runs, "wall_s"),
          "sup_err_inner": median_of(cv_runs, "sup_err_inner"),
          "cv_solve_path_steps_per_s": median_of(cv_runs, "cv_solve_path_steps_per_s"),
          "stat_err_rms": float(((cv_vals[0] - cv_vals[1]).pow(2).mean() / 2).sqrt()) if len(cv_vals) > 1 else None}

    eps = plain["sup_err_inner"]
    spread = [r["sup_err_inner"] for r in plain_runs]
    out.update({"eps": eps, "eps_seed_spread": max(spread) - min(spread), "plain": plain,
                "plain_same_M_as_cv": abl, "own_z_control_same_M": own, "cv": cv,
                "cv_reaches_eps": cv["sup_err_inner"] <= eps,
                "cv_runs_reaching_eps": sum(r["sup_err_inner"] <= eps for r in cv_runs),
                "plain_same_M_reaches_eps": abl["sup_err_inner"] <= eps,
                "own_z_control_reaches_eps": own["sup_err_inner"] <= eps,
                "variance_ratio_own_z_same_M": (abl["stat_err_rms"] / own["stat_err_rms"]) ** 2,
                "plain_over_cv_time": plain["wall_s"] / cv["wall_s"],
                "variance_ratio_same_M": ((abl["stat_err_rms"] / cv["stat_err_rms"]) ** 2
                                          if cv["stat_err_rms"] else None)})
    return out


# ---- the paper's own experiment (Sec. 5.1): error indicators over many runs ----------
def paper_table_rows(table: str):
    """Rows (N, cells per dimension, M, runs) of tables of Sec. 5.2: d = 11 LP0
    with #C = floor(sqrt N), M = N^2 and LP1 with #C = 2, 3 at dt = 0.2; d = 4 LP1
    with #C = floor(3 sqrt(d sqrt(N)) - 5), M = (d+1) N^2 and LP0 with
    #C = floor(4 sqrt(N)), M = N^2; d = 6 LP1 with #C = floor(1.5 sqrt(d sqrt(N))
    - 3), M = (d+1) N^2 and LP0 with #C = floor(2 sqrt(N)), M = N^2.  The run
    counts are ours (10^3 in the paper), fewer where one run takes seconds."""
    if table == "lp0_d11":
        # #C = floor(sqrt(N)), M = N^2 (the paper's LP0 table at d = 11)
        d, rows = 11, [(5, 1000), (10, 50), (20, 3)]
        return d, "lp0", [(N, int(math.floor(math.sqrt(N))), N * N, R) for N, R in rows]
    if table == "lp1_d11":
        # the paper's LP1 table at d = 11: dt = 0.2 with #C = 2, M = 2000 and #C = 3, M = 4000
        return 11, "lp1", [(5, 2, 2000, 1000), (5, 3, 4000, 20)]
    if table == "lp1_d12_19":
        # the paper's LP1 tables at d = 12..19 (dt = 0.2): rows (N, #C, M, runs, d)
        return 12, "lp1", [(5, 2, 2000, 100, 12), (5, 3, 4000, 3, 12), (5, 2, 3000, 100, 13),
                           (5, 2, 4000, 100, 13), (5, 2, 2000, 100, 14), (5, 2, 4000, 50, 14),
                           (5, 2, 5000, 20, 15), (5, 2, 6000, 10, 16), (5, 2, 5000, 5, 17),
                           (5, 2, 4000, 3, 18), (5, 2, 3200, 3, 19)]
    if table == "lp1_d6":
        d, rows = 6, [(5, 1000), (10, 1000), (20, 200), (50, 3)]
        return d, "lp1", [(N, int(math.floor(1.5 * math.sqrt(d * math.sqrt(N)) - 3)), (d + 1) * N * N, R)
                          for N, R in rows]
    if table == "lp0_d6":
        d, rows = 6, [(5, 1000), (10, 200), (20, 40)]
        return d, "lp0", [(N, int(math.floor(2 * math.sqrt(N))), N * N, R) for N, R in rows]
    d = 4
    if table == "lp1_d4":
        rows = [(5, 1000), (10, 1000), (20, 1000), (50, 10)]
        return d, "lp1", [(N, int(math.floor(3 * math.sqrt(d * math.sqrt(N)) - 5)), (d + 1) * N * N, R)
                          for N, R in rows]
    if table == "lp0_d4":
        rows = [(5, 1000), (10, 1000), (20, 200)]
        return d, "lp0", [(N, int(math.floor(4 * math.sqrt(N))), N * N, R) for N, R in rows]
    raise ValueError(table)


def paper_table(args, stream):
    """The error indicators of Sec. 5.1 (eq. mse) for the paper's test BSDE
    (X = W, logistic model, mu = 1, T = 1, strata on [-6.5, 6.5]^d, FP32 paths):
    R independent runs (Philox seeds 1..R), each evaluated against the closed
    form at n points per step drawn i.i.d. from nu independently of the
    clouds; MSE_Y,max = ln(max_i S_i^y / (R n)), MSE_Y,av = ln(sum_i S_i^y /
    (R n N)), MSE_Z,av likewise with |z_i - z*|^2, S_i the sums over runs and
    points.  (The paper pairs run m with one point R_{i,m}; n points per run
    estimate the same expectation with less noise.)  GPU time per run = CUDA
    events around srmc_solve on the stream."""
    import torch
    from paper_2407_21085_gb300 import srmc

    d, basis, rows = paper_table_rows(args.paper_table)
    n = args.paper_points
    out = []
    gen = torch.Generator(device="cuda")
    gen.manual_seed(12345)
    for row in rows:
        N, C, M, R = row[:4]
        d = row[4] if len(row) > 4 else d
        w0 = W.logistic_paper(d=d, N=N, C=C, M=M, basis=basis)
        sums = torch.zeros((N, 2), dtype=torch.float64, device="cuda")
        part = torch.empty((N, 2), dtype=torch.float64, device="cuda")
        ms = []
        t0 = time.perf_counter()
        for r in range(R):
            s = srmc.Solver(w0.replace(seed=r + 1))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s.srmc_solve(stream)
            b.record(stream)
            U = torch.rand((N, n, d), dtype=torch.float64, device="cuda", generator=gen)
            U = U.clamp_(1e-300, 1.0 - 2.0 ** -53)
            X = torch.log(U) - torch.log1p(-U)              # logistic, mu = 1
            s.srmc_point_error(X, part, stream)
            sums += part
            b.synchronize()
            ms.append(a.elapsed_time(b))
            s.close()
        wall = time.perf_counter() - t0
        S = sums.cpu().numpy()
        out.append({"d": d, "dt": 1.0 / N, "N": N, "cells_per_dim": C, "K": C ** d, "M": M, "runs": R,
                    "points_per_step_per_run": n,
                    "MSE_Y_max": float(math.log(S[:, 0].max() / (R * n))),
                    "MSE_Y_av": float(math.log(S[:, 0].sum() / (R * n * N))),
                    "MSE_Z_av": float(math.log(S[:, 1].sum() / (R * n * N))),
                    "gpu_ms_per_run": statistics.median(ms), "wall_s_all_runs": wall,
                    "path_steps_per_run": w0.path_steps()})
    return {"paper_table": args.paper_table, "model": "logistic (Sec. 5.1)", "precision": "fp32",
            "basis": basis, "rows": out}


# ---- the batched form: 256 heterogeneous instances ---------------------------------
def batched_compare(args, stream):
    """cfg4: 256 seeded instances (d in {1,2,3}, 16..64 cells per dimension,
    N in {10,20,40}, M in {1024,4096}) solved by the tuned batched form (the
    fastest of: per-round multi-instance launches, one graph branch per
    instance, one persistent launch per kernel variant) and, for comparison,
    one after another by single-instance solves on the same stream.  Device
    time by CUDA events on the stream, after one untimed pass of each."""
    import torch
    from paper_2407_21085_gb300 import srmc

    ws = W.cfg4_instances()
    units = sum(w.path_steps() for w in ws)
    solvers = [srmc.Solver(w) for w in ws]
    batch = srmc.Batch(solvers)
    t0 = time.perf_counter()
    threads = batch.srmc_batch_tune(stream)
    tune_s = time.perf_counter() - t0

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3 / reps

    t_batch = timed(lambda: batch.srmc_batch_solve(stream), args.batch_reps)
    mode = batch.srmc_batch_mode()
    # the three strategies as timed by the tuner (one whole-batch solve each)
    t_mode = dict(zip(("rounds", "branches", "persistent"), (v / 1e3 for v in batch.srmc_batch_strategy_ms())))

    # one after another, with CUDA events around every instance's solve
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in solvers]

    def sequential(record):
        for s, (a, b) in zip(solvers, evs):
            if record:
                a.record(stream)
            s.srmc_solve(stream)
            if record:
                b.record(stream)
    sequential(False)
    torch.cuda.synchronize()
    a0, b0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    sequential(True)
    b0.record(stream)
    torch.cuda.synchronize()
    t_seq = a0.elapsed_time(b0) / 1e3
    per_inst = [a.elapsed_time(b) / 1e3 for a, b in evs]
    # The instances with K >= 4096 strata fill the GPU on their own (every
    # launch is several waves of stratum blocks): no strategy that keeps the
    # kernels can solve them in less than the sum of their single solves.
    big = [r for r, w in enumerate(ws) if w.K >= 4096]
    floor_s = sum(per_inst[r] for r in big)
    batch.close()
    for s in solvers:
        s.close()
    return {"workload": "cfg4: 256 instances (seed 4)", "instances": len(ws), "path_steps": units,
            "batched_s": t_batch, "batched_path_steps_per_s": units / t_batch,
            "sequential_s": t_seq, "sequential_path_steps_per_s": units / t_seq,
            "speedup": t_seq / t_batch, "tuned_threads_per_group": threads, "tune_s": tune_s,
            "floor_s": floor_s, "batched_over_floor": t_batch / floor_s,
            "floor_basis": f"sum of the single-instance solve times of the {len(big)} instances with "
                           f"K >= 4096 strata ({100.0 * sum(ws[r].path_steps() for r in big) / units:.0f} % of "
                           "the path-steps), each of which fills the GPU alone",
            "strategy_s": t_mode,
            "strategy": ["rounds of multi-instance launches", "one graph branch per instance",
                         "one persistent launch per kernel variant"][mode]}


# ---- the CPU oracle (cpu_baseline leg and the reference arm) -------------------
def cpu_model() -> str:
    """The host CPU's model name (lscpu), or the platform string."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_cores():
    return os.cpu_count() or 1


def oracle_fits(w: W.Workload, plan, threads: int, seed: int = 0):
    """Time the FP64 oracle's fits of sampled strata of the workload at its
    full M: plan = [(step i, number of strata)], each group fitted in
    parallel over `threads` host threads (orc_fit_many).  The rows of the
    later steps a fit reads are not there, so the oracle is told to read
    them as the zero function (orc_set_missing_zero): every operation of the
    fit -- start points, all N - i Euler steps with their normals, cell
    location, row evaluation, driver, least squares -- runs as in a full
    solve, only the table values differ.  Returns [(i, n, seconds,
    path_steps)]."""
    import numpy as np
    from oracle import oracle as o
    o.build()
    orc = o.Oracle(w.replace(precision="fp64"))
    orc.set_missing_zero(True)
    rng = np.random.default_rng(seed)
    out = []
    for i, n in plan:
        ks = rng.choice(w.K, size=min(n, w.K), replace=False)
        before = orc.path_steps
        t0 = time.perf_counter()
        orc.fit_many(i, ks, threads)
        out.append((i, len(ks), time.perf_counter() - t0, orc.path_steps - before))
    orc.close()
    return out


def extrapolate_full(w: W.Workload, fits):
    """Seconds of a full backward solve (all K strata, all N steps) on the
    threads the fits used: the wall time of n fits at step i is modelled as
    (n / threads_batch) (a + b (N - i)), fitted by least squares over the
    measured steps, and summed over i = 0..N-1 for K strata."""
    import numpy as np
    A = np.array([[1.0, w.N - i] for i, n, sec, _ in fits])
    y = np.array([sec / n for i, n, sec, _ in fits])
    a, b = np.linalg.lstsq(A, y, rcond=None)[0]
    return float(sum(w.K * (a + b * (w.N - i)) for i in range(w.N)))


def oracle_plan(w: W.Workload, threads: int, single: bool):
    """Sampled steps 0, N/2, N-1; strata per step sized to about 10 s of CPU
    work in total per workload (fewer single-threaded)."""
    per = max(1, threads) * (1 if w.d >= 4 else 4)
    if single:
        return [(0, 1), (w.N // 2, 1), (w.N - 1, 4)]
    return [(0, per), (w.N // 2, per), (w.N - 1, 4 * per)]


def cpu_baseline(w: W.Workload):
    """The oracle timed on this host on bounded samples of the workload (and
    of cfg3, cfg2 for context): all cores and one thread, with the full-solve
    time extrapolated from the samples (marked as extrapolated)."""
    cores = cpu_cores()
    res = {"kind": "oracle", "cores": cores, "cpu_model": cpu_model(), "unit": UNIT,
           "sample": (f"{w.name}: oracle fits of sampled strata at steps 0, N/2, N-1 with the full "
                      f"M={w.M} (later rows read as zero: same arithmetic), FP64"),
           "workloads": {}}
    for ww in (w, W.cfg3(), W.cfg2()):
        if ww.name in res["workloads"]:
            continue
        entry = {}
        for label, th in (("all_cores", cores), ("one_thread", 1)):
            fits = oracle_fits(ww, oracle_plan(ww, th, th == 1), th)
            sec = sum(f[2] for f in fits)
            steps = sum(f[3] for f in fits)
            full = extrapolate_full(ww, fits)
            entry[label] = {"threads": th, "path_steps_per_s": steps / sec, "sample_seconds": sec,
                            "sample_path_steps": steps,
                            "fits": [{"i": i, "strata": n, "seconds": t} for i, n, t, _ in fits],
                            "full_solve_seconds_extrapolated": full,
                            "full_solve_path_steps_per_s_extrapolated": ww.path_steps() / full}
        res["workloads"][ww.name] = entry
    main = res["workloads"][w.name]["all_cores"]
    res["value"] = main["path_steps_per_s"]
    res["seconds"] = main["sample_seconds"]
    return res


# the sampled steps of the reference arm, cycled through by its steps
REF_STEPS = (0, 10, 20, 30, 39)


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return None
    w = workload(args.workload)
    cores = cpu_cores()
    n = args.ref_strata or cores

    def one(k):
        i = REF_STEPS[k % len(REF_STEPS)] * (w.N - 1) // 39
        return oracle_fits(w, [(i, n)], cores, seed=k)[0]
    for k in range(args.warmup):
        one(k)
    secs, units = 0.0, 0
    for k in range(args.steps):
        _, _, sec, st = one(args.warmup + k)
        secs += sec
        units += st
    value = units / secs
    sample = (f"{w.name}: per step, oracle fits of {n} sampled strata at one step i (cycling through "
              f"{', '.join(str(v * (w.N - 1) // 39) for v in REF_STEPS)}) with the full M={w.M}, "
              "later rows read as zero (same arithmetic), FP64")
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "d": w.d, "strata": w.K, "N": w.N, "M": w.M, "basis": w.basis,
                   "sample_strata_per_step": n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                         "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="cfg5")
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-strata", type=int, default=0,
                    help="strata fitted per reference-arm step (0: one per host core)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--block-threads", type=int, default=0, help="threads per stratum block (0: library)")
    ap.add_argument("--no-cv-compare", action="store_true", help="skip the CV-vs-plain comparison (cfg5)")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-form measurement (cfg4)")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the precision-form measurement (cfg3: FP32 vs all-FP64)")
    ap.add_argument("--prec-M", type=int, default=4096, help="paths per stratum of the FP32 vs FP64 comparison")
    ap.add_argument("--batch-reps", type=int, default=2)
    ap.add_argument("--cv-small", action="store_true",
                    help="CV comparison on 5^6 strata of the same width (for profiler captures)")
    ap.add_argument("--control-random", action="store_true",
                    help="time the control-variate step kernel (rows from an untrained network)")
    ap.add_argument("--control-own", action="store_true",
                    help="time the step kernel with the run's own z control")
    ap.add_argument("--paper-table", choices=["lp1_d4", "lp0_d4", "lp1_d6", "lp0_d6", "lp0_d11", "lp1_d11",
                                              "lp1_d12_19"],
                    default=None,
                    help="instead of the benchmark: the error indicators of Sec. 5.1 over many runs")
    ap.add_argument("--paper-points", type=int, default=1000, help="nu points per step per run")
    ap.add_argument("--cv-M", type=int, default=1024)
    ap.add_argument("--cv-coarse-M", type=int, default=256)
    ap.add_argument("--cv-data", type=int, default=1 << 20)
    ap.add_argument("--cv-iters", type=int, default=2000)
    ap.add_argument("--cv-seeds", type=int, default=3, help="seeds of the plain and CV runs of the eps comparison")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per step-kernel launch from an ncu capture of this kernel")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    if args.paper_table:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(paper_table(args, torch.cuda.current_stream())), flush=True)
        return

    if args.impl == "reference":
        out = run_reference(args)
        if out is not None:
            print(json.dumps(out), flush=True)
        return

    out, rank, w = run_gpu(args)
    if rank == 0 and out["n_gpus"] == 1 and not args.no_cv_compare:
        import torch
        out["cv_vs_plain"] = cv_compare(args, torch.cuda.current_stream())
    if rank == 0 and out["n_gpus"] == 1 and not args.no_batched:
        import torch
        out["batched_cfg4"] = batched_compare(args, torch.cuda.current_stream())
    if rank == 0 and out["n_gpus"] == 1 and not args.no_precision:
        import torch
        out["precision_cfg3"] = precision_compare(args, torch.cuda.current_stream())
    if rank == 0:
        if not args.no_cpu_baseline and out["n_gpus"] == 1:
            out["cpu_baseline"] = cpu_baseline(w)
        else:
            out["cpu_baseline"] = None
        print(json.dumps(out), flush=True)
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
