"""Throughput of the black-oil Newton step on GB300, in cell-steps/s.

A "step" is one report step of the simulation (Newton iterations with
assembly, ILU(0) factorisation and BiCGStab solves, time-step cuts included)
on the 60x220x85 layered model with 5-spot wells (1,122,000 cells, report
steps of 10 days).  W warm-up report steps run untimed from the initial
state; the state and step control are then put back, so the K timed report
steps are report steps 1..K of the workload (its 20-step schedule at K = 20).

One timed loop.  Per report step the state goes in from pinned host memory
through bo_set_state, the step runs (bo_step), and the state comes back out
through bo_get_state.  CUDA events on the library's stream around bo_step
give `value` (inputs resident in HBM); events around all three give `e2e`.

Prints one JSON line.  --impl reference times the CPU FP64 oracle instead
(all host cores; each step a bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Algorithmic bytes per cell of each timed kernel (FP64 values, the minimum
# each kernel must move; index arrays and cache re-reads are not counted).
ALGO_BYTES_PER_CELL = {
    # forward sweep: D^-1 and 3 scaled lower blocks (36 doubles), r in, y out
    "ilu_fwd_sweep": 36 * 8 + 24 + 24,
    # backward sweep: 3 scaled upper blocks (27 doubles), y in, z out
    "ilu_bwd_sweep": 27 * 8 + 24 + 24,
    # operator: 7 blocks (63 doubles), x in, y out, one dot operand in
    "spmv_wells": 63 * 8 + 24 + 24 + 24,
    # factorisation: 7 blocks of A in, 7 blocks of P out
    "ilu_factor": 63 * 8 * 2,
}
# Mixed precision: the forward stage reads D^-1 (FP64) and the FP64 residual
# to form q = D^-1 r, then the three scaled lower blocks in FP32, and leaves an
# FP32 intermediate; the backward sweep reads the three scaled upper blocks in
# FP32 and the intermediate and writes the FP64 result.
ALGO_BYTES_PER_CELL_MIXED = dict(ALGO_BYTES_PER_CELL)
ALGO_BYTES_PER_CELL_MIXED.update({
    "ilu_fwd_sweep": 9 * 8 + 24 + 27 * 4 + 12,
    "ilu_bwd_sweep": 27 * 4 + 12 + 24,
})

# FP64 floating-point operations per cell of each timed kernel (an FMA counts
# two), the co-limit on GB300 where FP64 runs at 1/64 of the FP32 rate:
ALGO_FP64_FLOPS_PER_CELL = {
    # D^-1 r (9 FMA) and three scaled lower blocks times a 3-vector (27 FMA)
    "ilu_fwd_sweep": 2 * 36,
    # three scaled upper blocks times a 3-vector
    "ilu_bwd_sweep": 2 * 27,
    # seven 3x3 blocks times a 3-vector
    "spmv_wells": 2 * 63,
    # D -= A_ck (D_k^-1 A_kc) for three lower neighbours (81 FMA), the 3x3
    # inverse (~40 operations), six scaled blocks D^-1 A_cj (162 FMA)
    "ilu_factor": 2 * (81 + 162) + 40,
}
# FP64 FMA throughput of this GPU, measured by a timing probe of dependent-free
# DFMA streams on every SM (1.9 DFMA per clock per SM at 2070 MHz)
FP64_PEAK_TFLOPS = 1.19


def fp64_colimit(kernel, n, avg_s):
    """Achieved FP64 rate of one launch of `kernel` over n cells taking avg_s
    seconds, against the measured FP64 peak (None for a kernel not listed)."""
    f = ALGO_FP64_FLOPS_PER_CELL.get(kernel)
    if f is None or not avg_s > 0:
        return None
    tf = f * n / avg_s / 1e12
    return {"flops_per_cell": f, "achieved_tflops": round(tf, 4), "peak_tflops": FP64_PEAK_TFLOPS,
            "frac": round(tf / FP64_PEAK_TFLOPS, 4), "peak_source": "of measured (FP64 FMA probe)"}


WORKLOADS = {
    0: "spe1-shaped 10x10x3, 30-day report steps",
    1: "layered 60x220x85 black-oil, 5-spot wells, 10-day report steps",
    2: "Gaussian-random-field 100x100x50 black-oil, 5-spot wells, 5-day report steps",
}
def subdomain_name(ysub, zsub):
    cuts = [f"{ysub} cell rows in y"] * bool(ysub) + [f"{zsub} cell layers in z"] * bool(zsub)
    return f" as block-Jacobi over slabs of {' and '.join(cuts)}" if cuts else ""
LEARNED_NAME = (" + learned stage (63-128-128-9 MLP on BF16 tensor cores, trained online "
                "on the first warm-up report step's solver residuals)")
PRECISION_NAMES = {"fp64": "plain FP64 ILU0-BiCGStab",
                   "mixed": "FP32 ILU0 factors and sweeps, FP64 assembly/Krylov/Newton"}
CPR_NAME = (" with the two-stage CPR preconditioner (aggregation-AMG V-cycle on the "
            "quasi-IMPES pressure matrix, then ILU0)")


def peaks():
    """Roofline denominators: MEASURED_PEAKS.json (measured on this
    pool's GB300s), else the profiling recipe's fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "of measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "source": "of fallback"}


# Operations per report step of a workload (assemblies, ILU(0)
# factorisations, BiCGStab iterations), recorded by this bench's GPU arm
# (--record-ops) over the timed report steps.  The oracle takes the same
# Newton, cut and linear-solver decisions (the parity tests compare them on
# smaller models) but needs hours of CPU time per report step of the
# 60x220x85 model, so it cannot count them in a bounded run; the CPU
# figures are therefore the oracle's measured per-operation times scaled by
# these counts, and every line that uses them says so.
def ops_record_path(config):
    return os.path.join(ROOT, "profiles", f"op_counts_config{config}.json")


def load_ops(config):
    try:
        with open(ops_record_path(config)) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return None


def ncu_traffic(kernel, cells):
    """DRAM bytes per launch of `kernel` from the committed ncu summary
    (profiles/traffic.json), scaled by the cells swept; None once the
    kernel's source has changed since the counters were taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            rec = json.load(fh)[kernel]
        with open(os.path.join(ROOT, rec["source"]), "rb") as fh:
            sha = hashlib.sha1(fh.read()).hexdigest()
    except (OSError, KeyError, ValueError):
        return None
    if not sha.startswith(rec["sha1_prefix"]):
        return None
    return rec["bytes_per_cell"] * cells


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--no-restore", action="store_true",
                    help="time the K report steps after the warm-up ones instead of "
                         "restarting from the initial state")
    ap.add_argument("--record-ops", action="store_true",
                    help="write the timed steps' operation counts per report step to "
                         "profiles/op_counts_config<C>.json (the CPU scaling record)")
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", type=int, default=1, choices=[0, 1, 2, 3])
    ap.add_argument("--sweep-ctas-per-sm", type=int, default=0,
                    help="persistent CTAs per SM of the FP64 sweeps (1 or 2; 0: the library's default)")
    ap.add_argument("--members", type=int, default=256, help="ensemble members (config 3)")
    ap.add_argument("--ens-streams", type=int, default=0,
                    help="config 3: worker streams (0: the autotuner picks them)")
    ap.add_argument("--ens-precond", default="auto", choices=["auto", "ilu0", "cpr", "ilu0,cpr"],
                    help="config 3: preconditioner of every member, or 'small,large' by size "
                         "class (auto: the autotuner picks per size class)")
    ap.add_argument("--ens-small-schedule", default="tiled", choices=["auto", "tiled", "block"],
                    help="config 3: solve schedule of the members up to the median size "
                         "(auto: the autotuner's short probe picks it; that probe does not "
                         "separate the two, and the one-CTA solve is the slower on whole "
                         "report steps, so the default is tiled)")
    ap.add_argument("--seq-sample", type=int, default=32,
                    help="members stepped one at a time for the sequential comparison (config 3)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="ILU(0) preconditioner precision (mixed: FP32 factors and sweeps)")
    ap.add_argument("--precond", default="ilu0", choices=["ilu0", "cpr"],
                    help="BiCGStab preconditioner (cpr: two-stage CPR, AMG pressure stage + ILU(0))")
    ap.add_argument("--ysub", type=int, default=0,
                    help="block-Jacobi ILU(0) over slabs of YSUB cell rows in y (multiple of 8)")
    ap.add_argument("--zsub", type=int, default=0,
                    help="and over slabs of ZSUB cell layers in z (multiple of 4)")
    ap.add_argument("--learned", action="store_true",
                    help="learned preconditioner stage: trained online during the first "
                         "--train-steps warm-up report steps, then on inside BiCGStab")
    ap.add_argument("--train-steps", type=int, default=1)
    ap.add_argument("--train-samples", type=int, default=8)
    ap.add_argument("--train-lr", type=float, default=1e-3)
    ap.add_argument("--grid", default=None,
                    help="NXxNYxNZ: a layered model of this size instead of the config (profiling)")
    ap.add_argument("--report-days", type=float, default=None,
                    help="report-step length override (profiling windows)")
    ap.add_argument("--scan-slabs", nargs="+", default=None, metavar="Y,Z",
                    help="profiling: the first report step from the hydrostatic state "
                         "once per block-Jacobi slab shape (ysub,zsub), one JSON line each")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-its", type=int, default=8,
                    help="BiCGStab iterations in one CPU sample")
    ap.add_argument("--cpu-threads", type=int, default=0,
                    help="oracle threads of the all-cores CPU leg (0: every host core)")
    return ap.parse_args()


def max_over_ranks(value, world, device="cpu"):
    """Largest value over all ranks (the slowest rank sets the job time)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_throughput(cells, steps, world, ms_max):
    """cell-steps/s of all replicas together: every rank advanced its own model
    by `steps` report steps; the job took the slowest rank's time."""
    return cells * steps * world / (ms_max / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def model_for(config, grid=None):
    import synth
    if grid:
        nx, ny, nz = (int(v) for v in grid.lower().split("x"))
        return synth.layered_model(nx, ny, nz, config=1, name=f"layered {nx}x{ny}x{nz}")
    return {0: synth.config0, 1: synth.config1, 2: synth.config2,
            3: lambda: synth.config3_member(0)}[config]()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def host_cpu():
    """Core count and CPU model of this host (nproc / lscpu)."""
    cores = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": cores, "model": model}


def oracle_sample(o, dt, sample_its):
    """One bounded sample of the workload on the oracle: an assembly, an
    ILU(0) factorisation and `sample_its` BiCGStab iterations of the current
    system.  Returns (seconds per assembly, per factorisation, per BiCGStab
    iteration, total seconds)."""
    t0 = time.perf_counter()
    o.assemble(dt)
    t_asm = time.perf_counter() - t0
    t0 = time.perf_counter()
    o.ilu0()
    t_fac = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, its, _ = o.solve(tol=1e-30, maxit=sample_its)   # the solve repeats the factorisation
    t_sol = time.perf_counter() - t0
    t_it = max(t_sol - t_fac, 0.0) / max(its, 1)
    return t_asm, t_fac, t_it, t_asm + t_fac + t_sol


def cpu_rate(n, ops, t_asm, t_fac, t_it):
    """cell-steps/s of the oracle: its measured time per assembly,
    factorisation and BiCGStab iteration times the operations of a report
    step (ops per report step)."""
    sec = ops["assemblies"] * t_asm + ops["solves"] * t_fac + ops["lin_its"] * t_it
    return n / sec if sec > 0 else None, sec


def cpu_baseline(config, ops, sample_its, threads):
    """The oracle on the same model at its initial state, one bounded sample
    on one thread and one on `threads` threads (all host cores), scaled by
    the operation counts per report step of the GPU run's timed steps (the
    same algorithm takes the same decisions)."""
    import oracle
    m = model_for(config)
    n = m["nx"] * m["ny"] * m["nz"]
    o = oracle.Oracle(m)
    o.init_hydrostatic()
    o.begin_step()
    legs = {}
    for nt in (1, threads):
        oracle.set_threads(nt)
        t_asm, t_fac, t_it, tot = oracle_sample(o, m["dt"], sample_its)
        v, sec = cpu_rate(n, ops, t_asm, t_fac, t_it)
        legs[nt] = {"value": v, "cores": nt, "sec_per_report_step": sec,
                    "sample": (f"1 assembly ({t_asm:.2f} s), 1 ILU0 ({t_fac:.2f} s), "
                               f"{sample_its} BiCGStab its ({t_it:.3f} s each), {tot:.1f} s")}
    oracle.set_threads(1)
    hc = host_cpu()
    top = legs[threads]
    return {"value": top["value"], "unit": "cell-steps/s", "cores": threads, "kind": "oracle",
            "sample": (f"oracle on the same model at its initial state on {threads} threads: "
                       f"{top['sample']}; scaled to {ops['assemblies']:.1f} assemblies, "
                       f"{ops['solves']:.1f} factorisations and {ops['lin_its']:.1f} BiCGStab "
                       "iterations per report step, counted by the GPU run's timed steps "
                       "(the oracle takes the same decisions; a report step of this model "
                       f"takes it about {top['sec_per_report_step'] / 3600:.1f} h)"),
            "single_thread": {"value": legs[1]["value"], "cores": 1, "sample": legs[1]["sample"]},
            "host": hc}


def workload_name(args, m):
    if args.grid:
        return f"{m['name']}, report steps of {args.report_days or m['dt'] / 86400.0:g} days"
    return WORKLOADS[args.config]


def pinned_state(sim):
    """Pinned host buffers for one state (p, sw, x, flag, bhp), as NumPy
    views that bo_set_state / bo_get_state read and write directly."""
    import torch
    n, nw = sim.n, max(sim.nw, 1)
    ts = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(3)]
    ts.append(torch.empty(n, dtype=torch.uint8).pin_memory())
    ts.append(torch.empty(nw, dtype=torch.float64).pin_memory())
    return ts, [t.numpy() for t in ts]


def run_gb300(args):
    import torch
    import torch.distributed as dist

    from paper_1910_06059_gb300 import Sim

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    m = model_for(args.config, args.grid)
    n = m["nx"] * m["ny"] * m["nz"]
    dt = m["dt"] if args.report_days is None else args.report_days * 86400.0
    sim = Sim(m, stream=stream)
    sim.precision = args.precision
    if args.ysub or args.zsub:
        sim.subdomains, sim.subdomains_z = args.ysub, args.zsub
    sim.preconditioner = args.precond
    if args.sweep_ctas_per_sm:
        sim.set_sweep_ctas_per_sm(args.sweep_ctas_per_sm)
    sim.init_hydrostatic()
    if args.learned:
        import synth
        sim.learn_set_params(synth.learned_init(0))
    init_state, init_dt = sim.get_state(), sim.dt_next

    def barrier():
        if world > 1:
            dist.barrier()

    def progress(tag, k, rep, sec):
        if rank == 0:
            print(json.dumps({"bench": tag, "report_step": k, "sec": round(sec, 2),
                              "newton": rep["newton_its"], "lin": rep["lin_its"],
                              "cuts": rep["cuts"], "substeps": rep["substeps"]}),
                  file=sys.stderr, flush=True)

    for w in range(args.warmup):
        if args.learned:
            if w == 0 and args.train_steps > 0:
                sim.learn_online(samples=args.train_samples, epochs=1, lr=args.train_lr)
            if w == args.train_steps:
                sim.learn_online(on=False)
                sim.learn_enable(True)
        t0 = time.perf_counter()
        _, rep = sim.step(dt, raise_on_fail=True)
        progress("warmup", w + 1, rep, time.perf_counter() - t0)
    if args.learned and args.warmup <= args.train_steps:
        sim.learn_online(on=False)
        sim.learn_enable(True)
    torch.cuda.synchronize()

    # pinned host state: the timed loop starts from the initial state (or,
    # with --no-restore, from the state the warm-up reached)
    keep_in, h_in = pinned_state(sim)       # the tensors own the pinned memory
    keep_out, h_out = pinned_state(sim)
    start = init_state if not args.no_restore else sim.get_state()
    for dst, src in zip(h_in, start):
        dst[:len(src)] = src
    if not args.no_restore:
        sim.dt_next = init_dt

    # ---- timed region: K report steps, one loop ---------------------------
    sim.set_timing(True)
    launches0 = sim.launches
    clocks = ClockSampler(torch.cuda.current_device())
    reps = []
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        e = ev[k]
        t0 = time.perf_counter()
        e[0].record(stream)
        sim.set_state(*h_in)                    # host -> device through the C ABI
        e[1].record(stream)
        _, rep = sim.step(dt, raise_on_fail=True)
        e[2].record(stream)
        sim.get_state(out=h_out)                # device -> host through the C ABI
        e[3].record(stream)
        reps.append(rep)
        h_in, h_out = h_out, h_in               # the next step starts from what came back
        progress("timed", k + 1, rep, time.perf_counter() - t0)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    launches = sim.launches - launches0
    ms = sum(e[1].elapsed_time(e[2]) for e in ev)
    ms_e2e = sum(e[0].elapsed_time(e[3]) for e in ev)
    timers = sim.timing()
    sim.set_timing(False)
    ms_max = max_over_ranks(ms, world, "cuda")
    ms_e2e = max_over_ranks(ms_e2e, world, "cuda")
    h2d = int(sum(a.nbytes for a in h_in[:4]) + 8 * sim.nw)
    d2h = h2d

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel ----------------------------------
    dominant = max((k for k in timers if k in ALGO_BYTES_PER_CELL), key=lambda k: timers[k][0])
    tot_ms, nlaunch = timers[dominant]
    avg_s = tot_ms / 1e3 / max(nlaunch, 1)
    algo_table = ALGO_BYTES_PER_CELL_MIXED if args.precision == "mixed" else ALGO_BYTES_PER_CELL
    algo = algo_table[dominant] * n
    achieved = algo / avg_s / 1e9
    pk = peaks()
    roof = {"bound": "hbm", "kernel": dominant, "achieved": round(achieved, 1),
            "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": round(achieved / pk["hbm_gbs"], 4),
            "traffic": ncu_traffic(dominant, n) if args.precision == "fp64" else None,
            "algorithmic_bytes": algo, "peak_source": pk["source"],
            "avg_launch_ms": round(avg_s * 1e3, 4), "launches": nlaunch,
            "fp64": fp64_colimit(dominant, n, avg_s) if args.precision == "fp64" else None}

    counts = {"steps": args.steps,
              "assemblies": sum(r["newton_its"] + r["substeps"] + r["cuts"] for r in reps),
              "solves": sum(r["newton_its"] for r in reps),
              "lin_its": sum(r["lin_its"] for r in reps)}
    per_step = {k: counts[k] / args.steps for k in ("assemblies", "solves", "lin_its")}
    if args.record_ops and not args.grid and args.precision == "fp64" and not args.learned \
            and not (args.ysub or args.zsub) and args.precond == "ilu0":
        with open(ops_record_path(args.config), "w") as fh:
            json.dump({"workload": WORKLOADS[args.config], "report_steps": args.steps,
                       "from_initial_state": not args.no_restore, **per_step,
                       "source": "bench.py --record-ops, GPU arm, timed report steps"}, fh,
                      indent=1)
            fh.write("\n")
    cpu = None
    if not args.no_cpu_baseline and world == 1 and args.precond == "ilu0":
        cpu = cpu_baseline(args.config if not args.grid else 1, per_step, args.cpu_sample_its,
                           args.cpu_threads or (os.cpu_count() or 1))

    value = whole_job_throughput(n, args.steps, world, ms_max)
    out = {
        "metric": "cell-steps/s at 1e-6 Newton tol: plain FP64 vs mixed/learned/batched",
        "value": value, "unit": "cell-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": ("f64" if args.precision == "fp64" else "f64+f32") + ("+bf16" if args.learned else ""),
        "data": "synthetic",
        "config": {"workload": (f"{workload_name(args, m)}, {PRECISION_NAMES[args.precision]}"
                                f"{CPR_NAME if args.precond == 'cpr' else ''}"
                                f"{LEARNED_NAME if args.learned else ''}"
                                f"{subdomain_name(args.ysub, args.zsub)}, "
                                "Newton tol 1e-6"),
                   "precision": args.precision, "precond": args.precond,
                   "ysub": args.ysub, "zsub": args.zsub,
                   "cells": n, "newton_tol": 1e-6, "linear_tol": 1e-3,
                   "timed_report_steps": (f"{args.warmup + 1}..{args.warmup + args.steps}"
                                          if args.no_restore else f"1..{args.steps}"),
                   "l2": (f"inputs larger than L2 (Jacobian {504 * n / 1e6:.0f} MB, ILU data "
                          f"{504 * n / 1e6:.0f} MB per model)"),
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "clocks": clk,
        "e2e": {"value": whole_job_throughput(n, args.steps, world, ms_e2e), "unit": "cell-steps/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "path": "bo_set_state (pinned host) + bo_step + bo_get_state (pinned host)"},
        "gpu_launches": launches,
        "roofline": roof,
        "cpu_baseline": cpu,
        "iterations": counts,
        "kernel_ms": {k: {"ms": round(v[0], 3), "launches": v[1]} for k, v in timers.items()},
    }
    if args.learned:
        out["learned"] = sim.learn_report()
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def run_reference(args):
    """The CPU oracle as it stands, on all host cores, on the same model:
    each of the W + K steps is one bounded sample (an assembly, an ILU(0)
    factorisation and --cpu-sample-its BiCGStab iterations at the model's
    initial state).  `ms_per_step` is the measured time of a sample; `value`
    converts the measured per-operation times to cell-steps/s with the
    operation counts per report step that the GPU arm recorded for this
    workload (profiles/op_counts_config<C>.json), and says so."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    m = model_for(args.config)
    n = m["nx"] * m["ny"] * m["nz"]
    threads = args.cpu_threads or (os.cpu_count() or 1)
    oracle.set_threads(threads)
    o = oracle.Oracle(m)
    o.init_hydrostatic()
    o.begin_step()
    samples = []
    for k in range(args.warmup + args.steps):
        r = oracle_sample(o, m["dt"], args.cpu_sample_its)
        if k >= args.warmup:
            samples.append(r)
    t_asm, t_fac, t_it = (float(np.median([x[q] for x in samples])) for q in range(3))
    ms_sample = 1e3 * float(np.mean([x[3] for x in samples]))
    ops = load_ops(args.config)
    if ops is not None:
        value, sec = cpu_rate(n, ops, t_asm, t_fac, t_it)
        basis = (f"measured per-operation times scaled by {ops['assemblies']:.1f} assemblies, "
                 f"{ops['solves']:.1f} factorisations and {ops['lin_its']:.1f} BiCGStab "
                 "iterations per report step, counted by the GPU arm on this workload "
                 f"({os.path.relpath(ops_record_path(args.config), ROOT)}); a report step "
                 f"would take the oracle about {sec / 3600:.2f} h")
    else:
        value, sec = None, None
        basis = "no operation-count record for this workload: no cell-steps/s estimate"
    sample = (f"per step: 1 assembly ({t_asm:.2f} s), 1 ILU0 ({t_fac:.2f} s), "
              f"{args.cpu_sample_its} BiCGStab its ({t_it:.3f} s each) on the model's "
              f"initial state, {threads} threads (medians over {len(samples)} timed samples)")
    out = {"impl": "reference",
           "metric": "cell-steps/s at 1e-6 Newton tol: plain FP64 vs mixed/learned/batched",
           "value": value, "unit": "cell-steps/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_sample, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": (f"{WORKLOADS[args.config]}, plain FP64 ILU0-BiCGStab, "
                                   "Newton tol 1e-6"), "cells": n},
           "value_basis": basis,
           "step": "one bounded sample of the workload (ms_per_step is its measured time)",
           "extrapolated_sec_per_report_step": sec,
           "cpu_baseline": {"value": value, "unit": "cell-steps/s", "cores": threads,
                            "kind": "oracle", "sample": sample, "host": host_cpu()},
           "e2e": {"value": value, "unit": "cell-steps/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def shard_members(count, rank, world):
    """Members of this rank when the ensemble is split over `world` GPUs:
    member q goes to rank q mod world (members are independent, so the
    ranks exchange nothing but the timing)."""
    return [q for q in range(count) if q % world == rank]


def ensemble_cpu_baseline(models, snap, dt, threads, budget_s=25.0):
    """The oracle, as it stands, on whole report steps of ensemble members
    (smallest first, from the same state as the timed steps) until about
    budget_s seconds of CPU work: no extrapolation, the cells of the members
    it finished over its time."""
    import oracle
    oracle.set_threads(threads)
    order = sorted(range(len(models)), key=lambda q: models[q]["nx"] * models[q]["ny"] * models[q]["nz"])
    cells, sec, done = 0, 0.0, []
    for q in order:
        if sec >= budget_s:
            break
        m = models[q]
        o = oracle.Oracle(m)
        st, d = snap[q]
        o.set_state(*st)
        o.dt_next = d
        t0 = time.perf_counter()
        status, _ = o.step(dt)
        sec += time.perf_counter() - t0
        if status == 0:
            cells += m["nx"] * m["ny"] * m["nz"]
            done.append(q)
    oracle.set_threads(1)
    if not done:
        return None
    return {"value": cells / sec, "unit": "cell-steps/s", "cores": threads, "kind": "oracle",
            "sample": (f"one whole report step of {len(done)} members, smallest first "
                       f"({cells} cells, {sec:.1f} s on {threads} threads)"),
            "host": host_cpu()}


def run_ensemble(args):
    """Config 3: the ensemble of uneven members stepped together (batched
    form), against the same members stepped one at a time on one stream.
    Under torchrun every rank steps its shard of the members."""
    import torch
    import torch.distributed as dist
    import synth
    from paper_1910_06059_gb300 import Ensemble

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    all_cells = sum(m["nx"] * m["ny"] * m["nz"] for m in synth.config3(args.members))
    models = [synth.config3_member(q) for q in shard_members(args.members, rank, world)]
    n = sum(m["nx"] * m["ny"] * m["nz"] for m in models)
    dt = models[0]["dt"] if args.report_days is None else args.report_days * 86400.0
    ens = Ensemble(models, streams=8)
    ens.init_hydrostatic()
    cand = (1, 4, 8, 16, 32, 64)
    sizes = [sm.n for sm in ens.members]
    median = sorted(sizes)[(len(sizes) - 1) // 2]
    if args.ens_streams > 0:
        ens.set_schedule(args.ens_streams, largest_first=True)
        tune = {"chosen": ens.schedule, "given": True}
    else:
        tune = ens.autotune(0.05 * 86400.0, candidates=cand)
    if args.ens_precond == "auto":
        tune_pc = ens.autotune_precond(0.05 * 86400.0)
    else:
        small, large = (args.ens_precond.split(",") * 2)[:2]
        for sm, sz in zip(ens.members, sizes):
            sm.preconditioner = small if sz <= median else large
        tune_pc = {"chosen": {"small": small, "large": large}, "probe_s": None}
    if args.ens_small_schedule == "auto":
        tune_sc = ens.autotune_schedule(0.05 * 86400.0)
    else:
        for sm, sz in zip(ens.members, sizes):
            sm.solve_schedule = args.ens_small_schedule if sz <= median else "tiled"
        tune_sc = {"chosen": {"small": args.ens_small_schedule, "streams": ens.schedule["streams"]},
                   "probe_s": None}
    for _ in range(args.warmup):
        ens.step(dt)
    torch.cuda.synchronize()
    snap = [(s.get_state(), s.dt_next) for s in ens.members]
    # ---- timed region: K report steps, one loop; every step takes each
    # member's state in from pinned host memory and back out through the
    # C ABI; the device time of the step itself comes from the ensemble's
    # CUDA events (members run on up to 64 streams)
    bufs = [(pinned_state(sm), pinned_state(sm)) for sm in ens.members]
    h_in = [b[0][1] for b in bufs]
    h_out = [b[1][1] for b in bufs]
    for hb, (st, _) in zip(h_in, snap):
        for dst, src in zip(hb, st):
            dst[:len(src)] = src
    for sm in ens.members:
        sm.set_timing(True)
    launches0 = sum(sm.launches for sm in ens.members)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    reps, dev_ms, e2e_s = [], 0.0, 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for sm, hb in zip(ens.members, h_in):
            sm.set_state(*hb)
        _, r = ens.step(dt)
        ms = ens.last_step_ms()
        for sm, hb in zip(ens.members, h_out):
            sm.get_state(out=hb)
        torch.cuda.synchronize()
        e2e_s += time.perf_counter() - t0
        dev_ms = dev_ms + ms if ms >= 0 and dev_ms >= 0 else -1.0
        reps.append(r)
        h_in, h_out = h_out, h_in
    clk = clocks.stop()
    launches = sum(sm.launches for sm in ens.members) - launches0
    timers = [sm.timing() for sm in ens.members]
    for sm in ens.members:
        sm.set_timing(False)
    sec = dev_ms / 1e3 if dev_ms > 0 else e2e_s
    sec = max_over_ranks(sec, world, "cuda")
    e2e_s = max_over_ranks(e2e_s, world, "cuda")
    h2d = int(sum(sum(a.nbytes for a in hb[:4]) + 8 * sm.nw for sm, hb in zip(ens.members, h_in)))
    if rank != 0:
        ens.close()
        dist.destroy_process_group()
        return
    # roofline of the forward sweep, averaged over every member's launches
    # (members share the SMs, so a launch takes longer than alone)
    fw = [(t["ilu_fwd_sweep"], sm.n) for t, sm in zip(timers, ens.members) if "ilu_fwd_sweep" in t]
    tot_ms = sum(v[0][0] for v in fw)
    nl = sum(v[0][1] for v in fw)
    byt = sum(ALGO_BYTES_PER_CELL["ilu_fwd_sweep"] * c * v[1] for v, c in fw)
    pk = peaks()
    roof = None
    if tot_ms > 0 and nl > 0:
        ach = byt / (tot_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": "ilu_fwd_sweep", "achieved": round(ach, 1),
                "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": round(ach / pk["hbm_gbs"], 4),
                "traffic": None, "algorithmic_bytes": int(byt / nl),
                "peak_source": pk["source"], "avg_launch_ms": round(tot_ms / nl, 4),
                "launches": nl, "note": "all members' launches; members run concurrently"}
    # one-CTA solves of the small members (BO_SCHEDULE_BLOCK), when chosen
    bl = [t["block_bicgstab"] for t in timers if "block_bicgstab" in t]
    block = None
    if bl:
        bms, bn = sum(v[0] for v in bl), sum(v[1] for v in bl)
        block = {"members": len(bl), "launches": bn, "ms_total": round(bms, 1),
                 "avg_launch_ms": round(bms / max(bn, 1), 3),
                 "note": "one launch of one CTA per linear solve; members overlap on the SMs"}
    # the same first report step, members one at a time on one stream, on a
    # sample of the members (largest and smallest mixed as in the ensemble)
    k = min(args.seq_sample, len(models))
    sample = ens.members[:k]
    for s, (st, d) in zip(sample, snap[:k]):
        s.set_state(*st)
        s.dt_next = d
    seq = Ensemble(sims=sample, streams=1)
    seq.set_schedule(1, largest_first=False)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    seq.step(dt)
    torch.cuda.synchronize()
    sec_seq = time.perf_counter() - t1
    ms_seq = seq.last_step_ms()
    seq.close()
    cells_sample = sum(s.n for s in sample)
    seq_value = cells_sample / (ms_seq / 1e3 if ms_seq > 0 else sec_seq)
    value = all_cells * args.steps / sec
    lin = sum(r["lin_its"] for rs in reps for r in rs)
    newton = sum(r["newton_its"] for rs in reps for r in rs)
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = ensemble_cpu_baseline(models, snap, dt, host_cpu()["nproc"])
    out = {
        "metric": "cell-steps/s at 1e-6 Newton tol: plain FP64 vs mixed/learned/batched",
        "value": value, "unit": "cell-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sec * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": (f"batched ensemble of {len(models)} members (nx, ny in 20..64, "
                                f"nz in 5..16; {all_cells} cells), {dt / 86400.0:g}-day report steps, "
                                "FP64 BiCGStab per member with ILU0 or CPR and the tiled or "
                                "one-CTA solve schedule chosen per size class by the autotuner, "
                                "Newton tol 1e-6"),
                   "cells": all_cells, "members": args.members,
                   "schedule": tune["chosen"],
                   "precond_by_size": tune_pc["chosen"],
                   "solve_schedule_small": tune_sc["chosen"]["small"],
                   "streams": tune_sc["chosen"]["streams"],
                   "timing": "CUDA events bracketing every worker stream of the step",
                   "l2": "members' Jacobians and ILU data together exceed L2",
                   "parallelism": f"members split over {world} GPUs" if world > 1 else "single GPU"},
        "clocks": clk,
        "e2e": {"value": all_cells * args.steps / e2e_s, "unit": "cell-steps/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d,
                "path": "bo_set_state (pinned host) per member + bo_ensemble_step + "
                        "bo_get_state (pinned host) per member"},
        "gpu_launches": launches,
        "roofline": roof,
        "cpu_baseline": cpu,
        "autotune_probe_s": tune,
        "autotune_precond_probe_s": tune_pc["probe_s"],
        "autotune_schedule_probe_s": tune_sc["probe_s"],
        "block_solve": block,
        "sequential": {"value": seq_value, "unit": "cell-steps/s",
                       "sample": f"first report step of {k} members one at a time on one stream "
                                 f"({cells_sample} cells, {sec_seq:.2f} s host clock, "
                                 f"{ms_seq / 1e3:.2f} s device events)"},
        "iterations": {"newton": newton, "lin_its": lin},
    }
    print(json.dumps(out))
    ens.close()
    if world > 1:
        dist.destroy_process_group()


def run_slab_scan(args):
    """The same report step (the first, from the hydrostatic state) under
    each block-Jacobi slab shape: wall time of the step, Newton and BiCGStab
    iterations, time-step cuts and the per-launch kernel times."""
    import torch
    from paper_1910_06059_gb300 import Sim
    shapes = [tuple(int(v) for v in a.split(",")) for a in args.scan_slabs]
    m = model_for(args.config, args.grid)
    n = m["nx"] * m["ny"] * m["nz"]
    dt = m["dt"] if args.report_days is None else args.report_days * 86400.0
    torch.cuda.set_device(0)
    sim = Sim(m)
    sim.init_hydrostatic()
    snap = sim.get_state()
    dtn = sim.dt_next
    for ysub, zsub in shapes:
        sim.subdomains, sim.subdomains_z = ysub, zsub
        sim.set_state(*snap)
        sim.dt_next = dtn
        sim.set_timing(False)
        sim.set_timing(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, rep = sim.step(dt, raise_on_fail=True)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        tm = sim.timing()
        sim.set_timing(False)
        print(json.dumps({
            "workload": workload_name(args, m), "ysub": ysub, "zsub": zsub,
            "sec": round(sec, 3), "cell_steps_per_s": round(n / sec, 1),
            "newton": rep["newton_its"], "lin": rep["lin_its"], "cuts": rep["cuts"],
            "substeps": rep["substeps"],
            "ms_per_launch": {k: round(v[0] / max(v[1], 1), 4) for k, v in tm.items()},
            "launches": {k: v[1] for k, v in tm.items()}}), flush=True)


def main():
    args = parse()
    if args.scan_slabs:
        run_slab_scan(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.config == 3:
        run_ensemble(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
