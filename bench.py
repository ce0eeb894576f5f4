#!/usr/bin/env python
"""Benchmark of the dp-adaptive MTO hot path on GB300.

Metric: TO iterations/s (solve + sensitivity) and MDOF x PCG-iterations/s, mixed precision vs the
plain FP64 GPU path.

Default workload: the large MBB half-beam, 1024 x 512 Q3 elements with 8 x 8 design subcells
(8192 x 4096 density field, 9,446,402 DOFs), smooth seeded densities at volume fraction 0.2,
Emin = 1e-9 E0, quoted on 20 optimality-criteria iterations.  One step is one TO iteration of one
optimization run, through the whole hot path: element build (step a), PCG solve warm-started from
the previous displacement to a relative compliance accuracy of 1e-8 (b), sensitivities (c), the
composite indicator with the dp map update (d) and the OC design update.  The warm-up steps are
the run's first iterations (the first solve starts from zero); the timed steps continue the same
run.  ``value`` is the mixed path (split-precision operator in the inner PCG); the same run in
plain FP64 is timed beside it, and the accuracy of both is checked after the timed region by an
FP64 re-solve on the same design.

``--mode pass`` repeats one pass over a fixed design instead (the 160 x 80 binary beam).

Multi-GPU: every rank solves its own replica (independent problems, no data-path collective);
value = total steps of all ranks / max over ranks of the timed wall.  The oracle (CPU, FP64) is
timed on a bounded sample as ``cpu_baseline``; ``--impl reference`` times only the oracle.
"""
import argparse
import functools
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TO iterations/s (solve+sensitivity) & MDOF·PCG-iter/s, mixed vs plain FP64 GPU"
UNIT = "TO-iter/s"
DEFAULT_WORKLOAD = "mbb_1024x512_p3_d8"
# the bounded sample the CPU oracle is timed on for each workload (same generator recipe)
SAMPLE_WORKLOAD = {"mbb_1024x512_p3_d8": "mbb_64x32_p3_d8", "mbb_160x80_p3_d8": "mbb_40x20_p3_d8",
                   "dp_cantilever_320x160": "dp_cantilever_40x20", "cantilever_20x10_p2_d4": "cantilever_20x10_p2_d4",
                   "mbb_40x20_p3_d8": "mbb_40x20_p3_d8", "mbb_480x240_p3_d8": "mbb_40x20_p3_d8",
                   "mbb_64x32_p3_d8": "mbb_64x32_p3_d8"}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--mode", default=None, choices=["oc", "pass"],
                    help="oc: steps are iterations of one optimization run (default for the large beam); "
                         "pass: repeated passes over one fixed design (default for the other workloads)")
    ap.add_argument("--rtol", type=float, default=1e-8, help="relative compliance accuracy of every solve")
    ap.add_argument("--mg-degree", type=int, default=2, help="Chebyshev degree of the fine-level smoothing")
    ap.add_argument("--smoother", default="block", choices=["block", "jacobi"],
                    help="fine-level smoothing: element blocks (default) or point Jacobi")
    ap.add_argument("--mg-operator", default=None, choices=["lead", "split", "auto"],
                    help="the multigrid cycle of the mixed path: in FP32 on the leading part of the split pair "
                         "(default for the single-instance workloads), on the split pair, or the library's "
                         "choice (default for batched_64, whose binary instances the FP32-rounded element "
                         "blocks do not always keep definite)")
    ap.add_argument("--build", default="tensor", choices=["tensor", "simt"],
                    help="element build: tcgen05 sliced GEMM (default) or FP64 CUDA cores")
    ap.add_argument("--fp64-steps", type=int, default=2, help="timed steps of the plain FP64 leg")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison leg")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--max-iters", type=int, default=400000,
                    help="cap on the PCG iterations of a solve (profiler captures of a few iterations only; "
                         "a capped solve is not a bench number)")
    ap.add_argument("--only-timed", action="store_true",
                    help="stop after the timed steps (no FP64 leg, end-to-end leg, accuracy check or CPU "
                         "baseline; for profiler captures of the timed region)")
    return ap.parse_args(argv)


# ------------------------------------------------------------------------------------ CPU oracle
def cpu_model():
    """Host CPU model and core count (the oracle runs single-threaded on it)."""
    name = None
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                name = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if not name:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.strip().lower().startswith("model name"):
                    name = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return f"{name or platform.processor() or 'unknown'} ({platform.machine()}, {os.cpu_count()} cores on the host)"


def oracle_step_script(workload):
    """Python source that times one oracle TO iteration (build, assemble, exact solve, sensitivity,
    indicators, map update, OC update) on `workload` and prints JSON."""
    return f"""
import json, sys, time
sys.path.insert(0, {ROOT!r})
import numpy as np
import workloads as W
from oracle import mesh as om, solve as osv, sensitivity as ose, indicators as oi, oc as ooc
pr = W.named({workload!r})
t0 = time.perf_counter()
m = om.DPMesh(pr.nelx, pr.nely, pr.p, pr.d)
fixed, f = (om.mbb_bc if pr.load == W.MBB else om.cantilever_bc)(m)
K = osv.assemble(m, osv.element_matrices(m, pr.rho, pr.E0, pr.Emin, pr.nu, pr.q))
u = osv.solve_direct(K, f, fixed)
t1 = time.perf_counter()
dc = ose.sensitivity(m, u, pr.rho, pr.E0, pr.Emin, pr.nu, pr.q)
C = ose.compliance(f, u)
t2 = time.perf_counter()
ga = oi.kelly(m, u); gd = oi.gamma_d(m, pr.rho); eq = oi.qr_error(m, u, pr.rho, pr.E0, pr.Emin, pr.nu, pr.q)
oi.map_update(pr.nelx, pr.nely, pr.p, ga, gd, eq)
t3 = time.perf_counter()
ooc.oc_update(pr.rho, dc, ooc.subcell_areas(m), float(np.mean(pr.rho)) * m.nel)
t4 = time.perf_counter()
print(json.dumps(dict(seconds=t4 - t0, build_solve=t1 - t0, sens=t2 - t1, indicator=t3 - t2, oc=t4 - t3,
                      free_dofs=int(m.ndof - len(fixed)), C=C)))
"""


def run_oracle_sample(workload, steps=1):
    """Time the oracle single-threaded (BLAS/OpenMP pinned to 1 thread) on a bounded sample of the
    workload; returns (median seconds per pass, info of the last pass)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    res = []
    for _ in range(steps):
        r = subprocess.run([sys.executable, "-c", oracle_step_script(workload)], capture_output=True, text=True,
                           env=env, timeout=900)
        if r.returncode != 0:
            raise RuntimeError(r.stderr[-2000:])
        res.append(json.loads(r.stdout.strip().splitlines()[-1]))
    return statistics.median(x["seconds"] for x in res), res[-1]


@functools.lru_cache(maxsize=None)
def free_dofs_of(workload):
    import workloads as W
    from oracle import mesh as om
    pr = W.named(workload)
    m = om.DPMesh(pr.nelx, pr.nely, pr.p, pr.d)
    fixed, _ = (om.mbb_bc if pr.load == W.MBB else om.cantilever_bc)(m)
    return int(m.ndof - len(fixed))


def oracle_rate(workload, steps=1):
    """(scaled TO-iter/s, measured seconds per sample step, description).  The oracle's TO iteration
    on the sample is timed; its rate is scaled to the workload by free DOFs, which is optimistic for
    the oracle at full size (its sparse factorisation grows faster than linearly)."""
    sample = SAMPLE_WORKLOAD.get(workload, workload)
    sec, info = run_oracle_sample(sample, steps)
    scale = info["free_dofs"] / free_dofs_of(workload)
    desc = (f"{sample}: one oracle TO iteration (assemble, equilibrated sparse LU + refinement, sensitivity, "
            f"indicators, map update, OC) timed single-threaded: median {sec:.2f} s of {steps}; the rate is "
            f"scaled to {workload} by free DOFs {info['free_dofs']}/{free_dofs_of(workload)} (optimistic for "
            f"the oracle); CPU {cpu_model()}")
    return scale / sec, sec, desc


def cpu_baseline(workload, steps=1):
    value, sec, desc = oracle_rate(workload, steps)
    return dict(value=value, unit=UNIT, cores=1, kind="oracle", sample=desc, sample_seconds_per_step=sec)


# ------------------------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.proc, self.lines = index, None, []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------ GPU arm
def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def max_over_ranks(ms, world, device):
    """The slowest rank's timed milliseconds, on every rank (all-reduce MAX; NCCL on the GPU path,
    any initialised backend works)."""
    if world == 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, steps, max_ms):
    """Steps of all ranks per second of the slowest rank (every rank runs `steps` steps)."""
    return world * steps / (max_ms * 1e-3)


# DRAM bytes (read + write) of one launch of the staged operator kernels, from ncu captures on the
# 480 x 240 beam (115,200 Q3 elements), per element; scaled to a launch by the elements it
# processes.  Split pair with FP64 vectors (the
# outer PCG), and the FP32 leading part with FP32 vectors (the multigrid cycle).
TMA_TRAFFIC_PER_ELEMENT = {"split": (542182400 + 15464704) / 115200, "lead": (274720256 + 7731968) / 115200}


def lead_bytes(pr, ndof):
    """Algorithmic bytes of one launch of the leading-part operator of the FP32 multigrid cycle: per
    element the hi row of its matrix ((n_e/2 + 1) n_e entries, 4 bytes) and its node map (4 bytes
    per node); per DOF one FP32 read of x and one FP32 write of y."""
    nn = [(int(p) + 1) ** 2 for p in pr.p]
    return sum(4 * (n + 1) * (2 * n) + 4 * n for n in nn) + 8 * ndof


def iteration_share(breakdown, iters):
    """Per PCG iteration of the bracketed step: the element-operator kernels' time (the outer PCG's
    split pair, the cycle's leading parts of the operator and of the element blocks) against the
    time of the solve's families (operators, the rest of the cycle and its per-step set-up,
    vectors)."""
    ms = lambda k: breakdown.get(k, {}).get("ms", 0.0)
    op = ms("applydf64") + ms("applylead")
    it = op + ms("precond") + ms("vector")
    return {"operator_ms_per_iter": op / max(iters, 1), "solve_ms_per_iter": it / max(iters, 1),
            "ratio": it / op if op else None}


def roofline(families, fam, bytes_per_launch, pr, hbm, lead):
    """HBM roofline of one operator kernel from the sampled CUDA-event timing of its family (average
    launch duration; one apply = one launch per order class)."""
    n, ms = families.get(fam, (0, 0.0))
    if not n:
        return None
    ncls = len(set(int(p) for p in pr.p))
    avg_ms = ms / n * ncls
    achieved = bytes_per_launch / (avg_ms * 1e-3) / 1e9
    p0 = int(pr.p[0])
    row_bytes = len(pr.p) * ((2 * (p0 + 1) ** 2) // 2 + 1) * 2 * (p0 + 1) ** 2 * (4 if lead else 8)
    big = row_bytes > (64 << 20)
    if lead:
        kernel = ("ebe_df_tma_kernel<3,false,float> (FP32 leading part of the split pair, FP32 vectors: the "
                  "multigrid cycle's operator)" if big else "ebe_df_pipe_kernel<3,false,float> (FP32 leading part)")
    else:
        kernel = ("ebe_df_tma_kernel<3,true,double> (split-precision pair, FP64 vectors: the outer PCG's "
                  "operator)" if big else "ebe_df_pipe_kernel<3,true,double> (split-precision pair)")
    key = "lead" if lead else "split"
    return {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": (achieved / hbm) if hbm else None,
            "traffic": TMA_TRAFFIC_PER_ELEMENT[key] * len(pr.p) if big else None,
            "traffic_note": ("stored ncu capture of this kernel on the 480x240 beam (115,200 elements), "
                             "dram__bytes_read.sum + dram__bytes_write.sum scaled by elements to this launch; "
                             "not measured in this run" if big else "no stored capture for this kernel here"),
            "peak_note": "measured HBM copy of MEASURED_PEAKS.json" if hbm else "no measured peak file",
            "bytes_per_launch": bytes_per_launch, "avg_launch_us": avg_ms * 1e3, "sampled_launches": n}


def smoother_of(args):
    import paper_1811_09821_gb300 as mto
    return mto.SMOOTH_BLOCK if args.smoother == "block" else mto.SMOOTH_JACOBI


def mg_operator_of(args, batched=False):
    import paper_1811_09821_gb300 as mto
    choice = args.mg_operator or ("auto" if batched else "lead")
    return {"lead": mto.MG_OP_LEAD, "split": mto.MG_OP_SPLIT, "auto": mto.MG_OP_AUTO}[choice]


def operator_bytes(pr, ndof):
    """Algorithmic bytes of one split-operator launch: per element the hi/lo pair of its matrix in
    the circulant-diagonal row ((n_e/2 + 1) n_e entries, 2 x 4 bytes) and its node map (4 bytes per
    node); per DOF one FP64 read of x and one FP64 write of y."""
    nn = [(int(p) + 1) ** 2 for p in pr.p]
    return sum(8 * (n + 1) * (2 * n) + 4 * n for n in nn) + 16 * ndof


class Run:
    """One problem instance on the GPU with the state of an optimization run."""

    def __init__(self, mto, W, pr, dev, stream, local_rank, args):
        import numpy as np
        import torch
        self.mto, self.torch, self.args = mto, torch, args
        self.pr, self.dev, self.stream = pr, dev, stream
        self.h = mto.Handle(local_rank, stream=stream)
        self.ndof, self.dlen = self.h.setup(pr.nelx, pr.nely, pr.p, pr.d)
        self.h.set_build_path(mto.BUILD_TENSOR if args.build == "tensor" else mto.BUILD_SIMT)
        self.fixed, self.f = mto.load_case(self.h, pr.load)
        self.h.set_supports(self.fixed)
        self.nfree = self.ndof - len(self.fixed)
        self.mat = mto.material(pr.E0, pr.Emin, pr.nu, pr.q)
        self.vol = float(np.mean(pr.rho))
        self.rho0 = torch.tensor(pr.rho, dtype=torch.float64, device=dev)
        self.reset()

    def reset(self):
        t = self.torch
        self.rho = self.rho0.clone()
        self.rho_new = t.empty_like(self.rho)
        self.u = t.zeros(self.ndof, dtype=t.float64, device=self.dev)
        self.dc = t.zeros(self.dlen, dtype=t.float64, device=self.dev)
        self.k = 0

    def step(self, prec, advance=True):
        """One pass of the hot path: build, solve, sensitivity, indicator + map update, OC update.
        advance: continue the optimization run (the next design is the OC update), else keep the
        design."""
        mto, h = self.mto, self.h
        h.build_elements(self.rho, self.mat, prec)
        it, rr = h.solve(self.f, self.u, precision=prec, rtol=self.args.rtol, norm=mto.NORM_ENERGY,
                         max_iter=self.args.max_iters, check_every=32, precond=mto.PREC_MG,
                         mg_degree=self.args.mg_degree, mg_smoother=smoother_of(self.args),
                         mg_operator=mg_operator_of(self.args), warm_start=advance and self.k > 0, raise_on_noconv=self.args.max_iters >= 400000)
        h.sensitivity(self.u, self.f, self.rho, self.mat, self.dc, precision=mto.MTO_FP64, want_C=False)
        h.indicator(self.u, self.rho, self.mat)
        h.oc_update(self.rho, self.dc, self.vol, self.rho_new, want_lambda=False)
        if advance:
            self.rho, self.rho_new = self.rho_new, self.rho
            self.k += 1
        return it

    def compliance(self, rho):
        return self.h.compliance_energy(self.u, self.f, rho, self.mat)


def timed_steps(run, prec, steps, warmup, advance, flush):
    """warmup untimed steps then `steps` steps timed with CUDA events on the run's stream (L2 flushed
    before each).  Returns dict(ms, iters, launches, families, last) with the design and the solved
    displacement of the last timed step kept for the accuracy check."""
    torch = run.torch
    for _ in range(warmup):
        run.step(prec, advance)
    torch.cuda.synchronize(run.dev)
    run.h.timing_enable("sampled")
    l0 = run.h.launch_count()
    total_ms, iters = 0.0, 0
    for _ in range(steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed_step")     # for profiler filters (ncu --nvtx-include timed_step/)
        e0.record(run.stream)
        rho_in = run.rho
        it = run.step(prec, advance)
        e1.record(run.stream)
        e1.synchronize()
        torch.cuda.nvtx.range_pop()
        total_ms += e0.elapsed_time(e1)
        iters += it
    launches = run.h.launch_count() - l0
    tm = run.h.timing_read()
    run.h.timing_enable(False)
    last = dict(rho=rho_in.clone(), u=run.u.clone())   # the last step's design (before its update) and u
    return dict(ms=total_ms, iters=iters, launches=launches, families=tm, last=last)


def accuracy_check(run, last, prec):
    """The compliance (energy form) of a timed step's own solution against an FP64 re-solve on the
    same design to 1e-2 of the bench tolerance, warm-started from it.  Returns a dict."""
    mto, h = run.mto, run.h
    rho, u = last["rho"], last["u"].clone()
    C = h.compliance_energy(u, run.f, rho, run.mat)
    h.build_elements(rho, run.mat, mto.MTO_FP64)
    it, _ = h.solve(run.f, u, precision=mto.MTO_FP64, rtol=run.args.rtol * 1e-2, norm=mto.NORM_ENERGY,
                    max_iter=400000, check_every=32, precond=mto.PREC_MG, mg_degree=run.args.mg_degree,
                    mg_smoother=smoother_of(run.args), warm_start=True)
    Cr = h.compliance_energy(u, run.f, rho, run.mat)
    return {"path": "mixed" if prec == mto.MTO_MIXED else "fp64", "C": C, "C_fp64_ref": Cr,
            "rel_err": abs(C - Cr) / abs(Cr), "ref_iters": it}


def run_gpu(args, rank, world, local_rank):
    import torch
    import paper_1811_09821_gb300 as mto
    import workloads as W

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    t_gen = time.perf_counter()
    pr = W.named(args.workload)
    t_gen = time.perf_counter() - t_gen
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    run = Run(mto, W, pr, dev, stream, local_rank, args)
    advance = args.mode == "oc"
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 512 MB > L2

    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local_rank) as clk:
        mixed = timed_steps(run, mto.MTO_MIXED, args.steps, args.warmup, advance, flush)
    torch.cuda.synchronize(dev)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    mixed_ms_max = max_over_ranks(mixed["ms"], world, dev)
    steps = args.steps
    if args.only_timed:
        run.h.close()
        return {"metric": METRIC, "value": whole_job_rate(world, steps, mixed_ms_max), "unit": UNIT,
                "n_gpus": world, "steps": steps, "warmup": args.warmup, "ms_per_step": mixed_ms_max / steps,
                "higher_is_better": True, "config": {"workload": args.workload, "note": "timed steps only"}}

    # where one step's device time goes (one more step with every kernel family bracketed by events;
    # outside the timed region, since the events add overhead)
    run.h.timing_enable(True)
    run.step(mto.MTO_MIXED, advance)
    breakdown = {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in run.h.timing_read().items() if v[0]}
    run.h.timing_enable(False)

    # end to end through the public API with host buffers: design and load in, displacement and
    # sensitivities out, every step (the mixed path, continuing the same run)
    rho_h = run.rho.cpu().pin_memory()
    f_h = run.f.cpu().pin_memory()
    u_h = torch.empty(run.ndof, dtype=torch.float64).pin_memory()
    dc_h = torch.empty(run.dlen, dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(steps, 3))
    e2e_ms = 0.0
    for _ in range(e2e_steps):
        flush.fill_(1.0)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        run.rho.copy_(rho_h, non_blocking=True)
        run.f.copy_(f_h, non_blocking=True)
        run.step(mto.MTO_MIXED, advance)
        u_h.copy_(run.u, non_blocking=True)
        dc_h.copy_(run.dc, non_blocking=True)
        rho_h.copy_(run.rho, non_blocking=True)      # the updated design returns to the host
        torch.cuda.synchronize(dev)
        e2e_ms += (time.perf_counter() - t0) * 1e3

    fp64 = None
    if not args.no_fp64:
        run.reset()
        fsteps = max(1, min(steps, args.fp64_steps))
        fp64 = timed_steps(run, mto.MTO_FP64, fsteps, args.warmup, advance, flush)

    # accuracy of both paths on their last timed step: the step's own solution against an FP64
    # re-solve on the same design
    checks = [accuracy_check(run, mixed["last"], mto.MTO_MIXED)]
    if fp64:
        checks.append(accuracy_check(run, fp64["last"], mto.MTO_FP64))

    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    rl_split = roofline(mixed["families"], "applydf64", operator_bytes(pr, run.ndof), pr, hbm, lead=False)
    rl_lead = roofline(mixed["families"], "applylead", lead_bytes(pr, run.ndof), pr, hbm, lead=True)
    # the dominant kernel: the one with more of the step's time (per-family totals of the bracketed step)
    t_split = breakdown.get("applydf64", {}).get("ms", 0.0)
    t_lead = breakdown.get("applylead", {}).get("ms", 0.0)
    rl_main, rl_other = (rl_lead, rl_split) if (rl_lead and t_lead > t_split) else (rl_split, rl_lead)
    out = {
        "metric": METRIC,
        "value": whole_job_rate(world, steps, mixed_ms_max),
        "unit": UNIT,
        "n_gpus": world,
        "steps": steps,
        "warmup": args.warmup,
        "ms_per_step": mixed_ms_max / steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32x2 split operator (f32 pipes) in the inner PCG; f64 vectors, dots, refinement, compliance",
        "data": "synthetic",
        "config": {"workload": args.workload, "nelx": pr.nelx, "nely": pr.nely, "p": int(pr.p[0]),
                   "d": int(pr.d[0]), "free_dofs": run.nfree, "design_values": run.dlen,
                   "mode": args.mode, "step": ("one TO iteration of one optimization run (build, warm-started "
                                               "solve, sensitivity, indicator + map update, OC update); warm-up = "
                                               "its first iterations" if advance else
                                               "one pass over the fixed design from a zero start"),
                   "solve_accuracy": f"relative compliance error {args.rtol:g} (energy test)",
                   "precond": (f"multigrid, {args.smoother} smoothing of degree {args.mg_degree} on the fine level; "
                               + ("cycle on the FP32 leading part of the split matrices"
                                  if mg_operator_of(args) == mto.MG_OP_LEAD else "cycle on the split pair")),
                   "element_build": "tcgen05 sliced GEMM" if args.build == "tensor" else "FP64 CUDA cores",
                   "l2_flush": "512 MB write before each timed step",
                   "parallelism": f"replicas x{world}"},
        "mdof_pcg_iter_per_s": run.nfree * mixed["iters"] / (mixed["ms"] * 1e-3) / 1e6,
        "pcg_iters_per_step": mixed["iters"] / steps,
        "sampled_operator_launches": {k: {"launches": v[0], "avg_us": round(1e3 * v[1] / max(v[0], 1), 3)}
                                      for k, v in mixed["families"].items() if v[0]},
        "gpu_launches": mixed["launches"],
        "launches_per_step": mixed["launches"] / steps,
        "launches_per_pcg_iter": mixed["launches"] / max(mixed["iters"], 1),   # includes the per-step kernels
        "operator_share_of_iteration": iteration_share(breakdown, mixed["iters"] / steps),
        "roofline": rl_main,
        "roofline_other_operator": rl_other,
        "operator_step_ms": {"applylead": t_lead, "applydf64": t_split},
        "accuracy": checks,
        "step_breakdown_ms": breakdown,
        "clocks": clk.summary(),
        "e2e": {"value": world * e2e_steps / (e2e_ms * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": 8 * (run.dlen + run.ndof),
                "d2h_bytes_per_step": 8 * (run.ndof + (2 * run.dlen if advance else run.dlen))},
        "host_generation_s": t_gen,
    }
    if fp64:
        fsteps = max(1, min(steps, args.fp64_steps))
        out["fp64_path"] = {"value": fsteps / (fp64["ms"] * 1e-3), "unit": UNIT, "steps": fsteps,
                            "ms_per_step": fp64["ms"] / fsteps,
                            "mdof_pcg_iter_per_s": run.nfree * fp64["iters"] / (fp64["ms"] * 1e-3) / 1e6,
                            "pcg_iters_per_step": fp64["iters"] / fsteps,
                            "sampled_operator_launches": {k: {"launches": v[0],
                                                              "avg_us": round(1e3 * v[1] / max(v[0], 1), 3)}
                                                          for k, v in fp64["families"].items() if v[0]}}
        out["speedup_vs_fp64"] = out["value"] / world / out["fp64_path"]["value"]
    run.h.close()
    return out


def run_batched(args, rank, world, local_rank):
    """The 64-instance workload: every step builds, solves (compliance accuracy, from zero) and
    differentiates all instances through the batched entry points (the instances run concurrently,
    each on its own stream with its own captured iteration graphs).  value = instance TO iterations
    per second of the whole batch."""
    import numpy as np
    import torch
    import paper_1811_09821_gb300 as mto
    import workloads as W

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    prs = W.batched()
    mat = mto.material()
    hs, fs, us, rhos, dcs, nfree, tune = [], [], [], [], [], 0, {}
    for pr in prs:
        h = mto.Handle(local_rank, stream=torch.cuda.Stream(dev))
        nd, dl = h.setup(pr.nelx, pr.nely, pr.p, pr.d)
        fixed, f = mto.load_case(h, pr.load)
        h.set_supports(fixed)
        nfree += nd - len(fixed)
        hs.append(h)
        fs.append(f)
        us.append(torch.zeros(nd, dtype=torch.float64, device=dev))
        rhos.append(torch.tensor(pr.rho, dtype=torch.float64, device=dev))
        dcs.append(torch.zeros(dl, dtype=torch.float64, device=dev))
    mto.build_elements_batched(hs, rhos, mat, mto.MTO_MIXED)
    for h, pr in zip(hs, prs):
        for p, (k, t) in h.autotune().items():
            tune[f"p{p}_{pr.nelx}x{pr.nely}"] = ["pipe", "staged", "generic"][k]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(prec):
        mto.build_elements_batched(hs, rhos, mat, prec)
        its, _, _ = mto.solve_batched(hs, fs, us, precision=prec, rtol=args.rtol, norm=mto.NORM_ENERGY,
                                      mg_degree=args.mg_degree, mg_smoother=smoother_of(args),
                                      mg_operator=mg_operator_of(args, batched=True))
        mto.sensitivity_batched(hs, us, fs, rhos, mat, dcs, want_C=False)
        torch.cuda.synchronize(dev)
        return int(its.sum())

    def timed(prec, steps, warmup):
        for _ in range(warmup):
            step(prec)
        l0 = sum(h.launch_count() for h in hs)
        total, iters = 0.0, 0
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            iters += step(prec)
            total += (time.perf_counter() - t0) * 1e3
        return total, iters, sum(h.launch_count() for h in hs) - l0

    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    with ClockSampler(local_rank) as clk:
        ms, iters, launches = timed(mto.MTO_MIXED, args.steps, args.warmup)
    ms_max = max_over_ranks(ms, world, dev)
    fsteps = max(1, min(args.steps, args.fp64_steps))
    ms64, iters64, _ = timed(mto.MTO_FP64, fsteps, 1) if not args.no_fp64 else (None, None, None)
    out = {
        "metric": METRIC, "value": whole_job_rate(world, args.steps * len(hs), ms_max), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32x2 split operator (f32 pipes) in the inner PCG; f64 vectors, dots, refinement, compliance",
        "data": "synthetic",
        "config": {"workload": "batched_64", "instances": len(hs),
                   "sizes": sorted({f"{p.nelx}x{p.nely}" for p in prs}),
                   "orders": sorted({int(p.p[0]) for p in prs}), "design_counts": sorted({int(p.d[0]) for p in prs}),
                   "free_dofs_total": nfree, "step": "build + compliance-accuracy solve from zero + sensitivities "
                                                     "of all instances (batched entry points)",
                   "solve_accuracy": f"relative compliance error {args.rtol:g}", "autotuned_kernels": tune,
                   "timing": "host wall around each synchronised batched step (the instances run on 64 streams)",
                   "l2_flush": "512 MB write before each timed step", "parallelism": f"replicas x{world}"},
        "mdof_pcg_iter_per_s": None,
        "pcg_iters_per_step": iters / args.steps, "gpu_launches": launches, "clocks": clk.summary(),
        "e2e": None,
    }
    if ms64:
        out["fp64_path"] = {"value": fsteps * len(hs) / (ms64 * 1e-3), "unit": UNIT, "steps": fsteps,
                            "pcg_iters_per_step": iters64 / fsteps}
        out["speedup_vs_fp64"] = out["value"] / world / out["fp64_path"]["value"]
    for h in hs:
        h.close()
    return out


def main(argv=None):
    args = parse(argv)
    if args.mode is None:
        args.mode = "oc" if args.workload == DEFAULT_WORKLOAD else "pass"
    batched = args.workload == "batched_64"
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return 0
        sample = SAMPLE_WORKLOAD.get(args.workload, args.workload)
        for _ in range(args.warmup):
            run_oracle_sample(sample, 1)
        value, sec, desc = oracle_rate(args.workload, args.steps)
        import workloads as W
        pr = W.named(args.workload)
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "nelx": pr.nelx, "nely": pr.nely, "p": int(pr.p[0]),
                       "d": int(pr.d[0]), "free_dofs": free_dofs_of(args.workload),
                       "design_values": int(len(pr.rho)), "sample": sample,
                       "parallelism": "rank 0 only (host cores)"},
            "note": "ms_per_step is the measured time of one oracle step on the sample; value is that rate "
                    "scaled to the workload by free DOFs",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }), flush=True)
        return 0

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    out = run_batched(args, rank, world, local_rank) if batched else run_gpu(args, rank, world, local_rank)
    if rank == 0:
        if not args.no_cpu and not batched and not args.only_timed:
            try:
                out["cpu_baseline"] = cpu_baseline(args.workload)
            except Exception as ex:      # the oracle is only a reported baseline
                out["cpu_baseline"] = {"error": str(ex)[:300]}
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
