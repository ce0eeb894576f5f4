#!/usr/bin/env python
"""Benchmark of the dp-adaptive MTO hot path on GB300.

Metric: TO iterations/s (solve + sensitivity) and MDOF x PCG-iterations/s, mixed precision vs the
plain FP64 GPU path.  One step = one pass of the whole hot path over one design: element build
(step a), PCG solve to the stated residual from a zero start (b), compliance and sensitivities (c)
and the composite indicator with the dp map update (d).

Default workload: the 160 x 80 MBB half-beam, Q3 elements with 8 x 8 design subcells (1280 x 640
density field), a seeded binary design at volume fraction 0.3, Emin = 1e-9 E0, relative residual
1e-8 (l2).  Both paths run the same steps; `value` is the mixed path.

Multi-GPU: every rank solves its own replica (independent problems, no data-path collective);
value = total steps of all ranks / max over ranks of the timed wall.  The oracle (CPU, FP64) is
timed on a bounded sample as `cpu_baseline`; `--impl reference` times only the oracle.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TO iterations/s (solve+sensitivity) & MDOF·PCG-iter/s, mixed vs plain FP64 GPU"
UNIT = "TO-iter/s"
DEFAULT_WORKLOAD = "mbb_160x80_p3_d8"
# DRAM bytes (read + write) per launch of the split operator ebe_df_pipe_kernel<3,double> on this
# workload inside the solve, from one ncu capture with warm caches (mean of 3 launches); to be
# re-taken whenever that kernel changes
MEASURED_TRAFFIC = {"mbb_160x80_p3_d8": 55921408 + 72619}
SAMPLE_WORKLOAD = {"mbb_160x80_p3_d8": "mbb_40x20_p3_d8", "dp_cantilever_320x160": "dp_cantilever_40x20",
                   "cantilever_20x10_p2_d4": "cantilever_20x10_p2_d4", "mbb_40x20_p3_d8": "mbb_40x20_p3_d8",
                   "mbb_1024x512_p3_d8": "mbb_40x20_p3_d8", "mbb_480x240_p3_d8": "mbb_40x20_p3_d8"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--precond", default="mg", choices=["schwarz", "jacobi", "mg"])
    ap.add_argument("--mg-degree", type=int, default=4, help="Chebyshev degree of the multigrid smoothing")
    ap.add_argument("--solve", default="mixed", choices=["mixed", "mixed32"],
                    help="mixed: FP64 refinement around inner PCG on the split-precision operator with FP64 "
                         "vectors; mixed32: the same with FP32 inner vectors")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison leg")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--oc-iters", type=int, default=0,
                    help="instead of repeated passes over one design, time one optimization run of this "
                         "many optimality-criteria iterations (each: build, warm-started mixed solve, "
                         "sensitivity, OC update of the design; the 1024x512 beam is quoted at 20)")
    return ap.parse_args()


# ------------------------------------------------------------------------------------ CPU oracle
def oracle_step_script(workload):
    """Python source that times one full oracle pass (build, assemble, exact solve, sensitivity,
    indicators, map update) on `workload` and prints JSON."""
    return f"""
import json, sys, time
sys.path.insert(0, {ROOT!r})
import workloads as W
from oracle import mesh as om, solve as osv, sensitivity as ose, indicators as oi
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
print(json.dumps(dict(seconds=t3 - t0, build_solve=t1 - t0, sens=t2 - t1, indicator=t3 - t2,
                      free_dofs=int(m.ndof - len(fixed)), C=C)))
"""


def run_oracle_sample(workload, steps=1):
    """Time the oracle single-threaded (BLAS/OpenMP pinned to 1 thread) on a bounded sample of the
    workload; returns (seconds per pass, info)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    res = []
    for _ in range(steps):
        r = subprocess.run([sys.executable, "-c", oracle_step_script(workload)], capture_output=True, text=True,
                           env=env, timeout=900)
        if r.returncode != 0:
            raise RuntimeError(r.stderr[-2000:])
        res.append(json.loads(r.stdout.strip().splitlines()[-1]))
    return statistics.median(x["seconds"] for x in res), res[-1]


def free_dofs_of(workload):
    import workloads as W
    from oracle import mesh as om
    pr = W.named(workload)
    m = om.DPMesh(pr.nelx, pr.nely, pr.p, pr.d)
    fixed, _ = (om.mbb_bc if pr.load == W.MBB else om.cantilever_bc)(m)
    return int(m.ndof - len(fixed))


def cpu_baseline(workload, steps=1):
    """Oracle on the bounded sample, scaled to the workload by free DOFs (the oracle's cost grows
    at least linearly with the DOFs, so the scaled rate is an upper bound on its full-size rate)."""
    sample = SAMPLE_WORKLOAD.get(workload, workload)
    sec, info = run_oracle_sample(sample, steps)
    scale = info["free_dofs"] / free_dofs_of(workload)
    value = scale / sec
    return dict(value=value, unit=UNIT, cores=1, kind="oracle",
                sample=f"{sample}: one full oracle pass (assemble, equilibrated sparse LU + refinement, "
                       f"sensitivity, indicators, map update) in {sec:.2f} s single-threaded, scaled by free "
                       f"DOFs {info['free_dofs']}/{free_dofs_of(workload)}")


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


def run_oc_loop(args, rank, world, local_rank):
    """One optimization run: args.oc_iters iterations of build, mixed solve (warm-started from the
    previous displacement), FP64 sensitivity and OC update (volume fraction of the initial design,
    move 0.2, eta 0.5), timed as a whole after args.warmup untimed iterations on a copy."""
    import numpy as np
    import torch
    import paper_1811_09821_gb300 as mto
    import workloads as W

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    pr = W.named(args.workload)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    h = mto.Handle(local_rank, stream=stream)
    ndof, dlen = h.setup(pr.nelx, pr.nely, pr.p, pr.d)
    fixed, f = mto.load_case(h, pr.load)
    h.set_supports(fixed)
    mat = mto.material(pr.E0, pr.Emin, pr.nu, pr.q)
    vol = float(np.mean(pr.rho))
    pc = {"schwarz": mto.PREC_SCHWARZ, "jacobi": mto.PREC_JACOBI, "mg": mto.PREC_MG}[args.precond]

    def run(iters):
        rho = torch.tensor(pr.rho, dtype=torch.float64, device=dev)
        rho_new = torch.empty_like(rho)
        u = torch.zeros(ndof, dtype=torch.float64, device=dev)
        dc = torch.zeros(dlen, dtype=torch.float64, device=dev)
        hist, its = [], 0
        for k in range(iters):
            h.build_elements(rho, mat, mto.MTO_MIXED)
            it, _ = h.solve(f, u, precision=mto.MTO_MIXED, rtol=args.rtol, max_iter=400000, check_every=32,
                            precond=pc, mg_degree=args.mg_degree, warm_start=k > 0)
            its += it
            hist.append(h.sensitivity(u, f, rho, mat, dc, precision=mto.MTO_FP64))
            h.oc_update(rho, dc, vol, rho_new, want_lambda=False)
            rho, rho_new = rho_new, rho
        return hist, its

    if args.warmup:
        run(min(args.warmup, 2))
    torch.cuda.synchronize(dev)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        e0.record(stream)
        hist, its = run(args.oc_iters)
        e1.record(stream)
        e1.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    h.close()
    return {
        "metric": METRIC, "value": whole_job_rate(world, args.oc_iters, ms), "unit": UNIT, "n_gpus": world,
        "steps": args.oc_iters, "warmup": args.warmup, "ms_per_step": ms / args.oc_iters, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32x2 split operator (f32 pipes) in inner PCG, f64 vectors/refinement/dots/compliance",
        "data": "synthetic",
        "config": {"workload": args.workload, "nelx": pr.nelx, "nely": pr.nely, "p": int(pr.p[0]), "d": int(pr.d[0]),
                   "design_values": dlen, "rtol": args.rtol, "precond": args.precond, "solve": "mixed",
                   "oc_iterations": args.oc_iters, "volume_fraction": vol, "parallelism": f"replicas x{world}"},
        "pcg_iters_total": its, "compliance_history": hist, "clocks": clk.summary(),
    }


def run_gpu(args, rank, world, local_rank):
    import numpy as np
    import torch
    import paper_1811_09821_gb300 as mto
    import workloads as W

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    pr = W.named(args.workload)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    h = mto.Handle(local_rank, stream=stream)
    ndof, dlen = h.setup(pr.nelx, pr.nely, pr.p, pr.d)
    fixed, f = mto.load_case(h, pr.load)
    h.set_supports(fixed)
    nfree = ndof - len(fixed)
    mat = mto.material(pr.E0, pr.Emin, pr.nu, pr.q)
    rho = torch.tensor(pr.rho, dtype=torch.float64, device=dev)
    u = torch.zeros(ndof, dtype=torch.float64, device=dev)
    dc = torch.zeros(dlen, dtype=torch.float64, device=dev)
    rho_new = torch.zeros(dlen, dtype=torch.float64, device=dev)
    vol = float(np.mean(pr.rho))
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 512 MB > L2

    pc = {"schwarz": mto.PREC_SCHWARZ, "jacobi": mto.PREC_JACOBI, "mg": mto.PREC_MG}[args.precond]

    def step(prec):
        h.build_elements(rho, mat, prec)
        sprec = mto.MTO_FP64 if prec == mto.MTO_FP64 else (mto.MTO_MIXED if args.solve == "mixed" else mto.MTO_MIXED32)
        it, rr = h.solve(f, u, precision=sprec, rtol=args.rtol, max_iter=400000, check_every=32, precond=pc,
                         mg_degree=args.mg_degree)
        h.sensitivity(u, f, rho, mat, dc, precision=mto.MTO_FP64, want_C=False)
        h.indicator(u, rho, mat)
        h.oc_update(rho, dc, vol, rho_new, want_lambda=False)
        return it, rr

    def timed(prec, steps, warmup):
        for _ in range(warmup):
            step(prec)
        torch.cuda.synchronize(dev)
        h.timing_enable("sampled")          # events around one operator launch per chunk of iterations
        l0 = h.launch_count()
        total_ms, iters, rrs = 0.0, 0, []
        for _ in range(steps):
            flush.fill_(1.0)                     # L2 flush outside the timed step
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            it, rr = step(prec)
            e1.record(stream)
            e1.synchronize()
            total_ms += e0.elapsed_time(e1)
            iters += it
            rrs.append(rr)
        tm = h.timing_read()
        h.timing_enable(False)
        return dict(ms=total_ms, iters=iters, relres=max(rrs), launches=h.launch_count() - l0, families=tm)

    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local_rank) as clk:
        wall0 = time.perf_counter()
        mixed = timed(mto.MTO_MIXED, args.steps, args.warmup)
        wall1 = time.perf_counter()
    torch.cuda.synchronize(dev)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    mixed_ms_max = max_over_ranks(mixed["ms"], world, dev)
    C_mixed = h.sensitivity(u, f, rho, mat, dc, precision=mto.MTO_FP64)

    fp64 = None
    if not args.no_fp64:
        fp64 = timed(mto.MTO_FP64, max(1, min(args.steps, 3)), 1)
        C_fp64 = h.sensitivity(u, f, rho, mat, dc, precision=mto.MTO_FP64)

    # end to end through the public API with host buffers: pinned rho and f in, u and dc out
    rho_h = torch.tensor(pr.rho, dtype=torch.float64).pin_memory()
    f_h = f.cpu().pin_memory()
    u_h = torch.empty(ndof, dtype=torch.float64).pin_memory()
    dc_h = torch.empty(dlen, dtype=torch.float64).pin_memory()
    e2e_ms = 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        rho.copy_(rho_h, non_blocking=True)
        f.copy_(f_h, non_blocking=True)
        step(mto.MTO_MIXED)
        u_h.copy_(u, non_blocking=True)
        dc_h.copy_(dc, non_blocking=True)
        torch.cuda.synchronize(dev)
        e2e_ms += (time.perf_counter() - t0) * 1e3

    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    fam = "apply32" if args.solve == "mixed32" else "applydf64"
    n_apply, apply_ms = mixed["families"][fam]
    # algorithmic bytes of one operator launch: the split-precision pair of the element matrix in
    # its circulant-diagonal row ((n_e/2 + 1) n_e entries, 2 x 4 bytes; 544 for Q3) and the node map
    # per element, one read of x and one write of y per DOF (4 bytes FP32, 8 bytes FP64 vectors)
    vb = 4 if args.solve == "mixed32" else 8
    nn = [(int(p) + 1) ** 2 for p in pr.p]
    kbytes = sum(8 * ((2 * n) // 2 + 1) * (2 * n) + 4 * n for n in nn)
    bytes_per_launch = kbytes + 2 * vb * ndof
    ncls = len(set(int(p) for p in pr.p))
    avg_ms = apply_ms / max(n_apply, 1) * ncls     # one apply = ncls class launches
    achieved = bytes_per_launch / (avg_ms * 1e-3) / 1e9 if n_apply else None
    steps = args.steps
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
        "dtype": ("f32x2 split operator (f32 pipes) in inner PCG, f64 vectors/refinement/dots/compliance"
                  if args.solve == "mixed" else "f32 inner PCG + f64 refinement/dots/compliance"),
        "data": "synthetic",
        "config": {"workload": args.workload, "nelx": pr.nelx, "nely": pr.nely, "p": int(pr.p[0]),
                   "d": int(pr.d[0]), "free_dofs": nfree, "design_values": dlen, "rtol": args.rtol,
                   "residual_norm": "l2", "precond": args.precond, "solve": args.solve,
                   "l2_flush": "512 MB write between timed steps",
                   "parallelism": f"replicas x{world}"},
        "mdof_pcg_iter_per_s": nfree * mixed["iters"] / (mixed["ms"] * 1e-3) / 1e6,
        "pcg_iters_per_step": mixed["iters"] / steps,
        "relres": mixed["relres"],
        "sampled_operator_launches": {k: {"launches": v[0], "avg_us": round(1e3 * v[1] / max(v[0], 1), 3)}
                                      for k, v in mixed["families"].items() if v[0]},
        "gpu_launches": mixed["launches"],
        "roofline": {"bound": "hbm",
                     "kernel": (f"ebe_df_pipe_kernel<3,{'float' if vb == 4 else 'double'}> (split-precision element "
                                "operator; ebe_df_tma_kernel for classes above 64 MB of rows)"),
                     "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": (achieved / hbm) if achieved else None,
                     "traffic": MEASURED_TRAFFIC.get(args.workload) if args.solve == "mixed" else None,
                     "bytes_per_launch": bytes_per_launch, "avg_launch_us": avg_ms * 1e3,
                     "note": "peak = measured HBM copy; the element rows stream from DRAM on every launch "
                             "(the multigrid cycle between launches evicts them from L2)"},
        "clocks": clk.summary(),
        "e2e": {"value": world * steps / (e2e_ms * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": 8 * (dlen + ndof), "d2h_bytes_per_step": 8 * (ndof + dlen)},
    }
    if fp64:
        out["fp64_path"] = {"value": fp64["ms"] and (max(1, min(steps, 3)) / (fp64["ms"] * 1e-3)), "unit": UNIT,
                            "ms_per_step": fp64["ms"] / max(1, min(steps, 3)),
                            "mdof_pcg_iter_per_s": nfree * fp64["iters"] / (fp64["ms"] * 1e-3) / 1e6,
                            "pcg_iters_per_step": fp64["iters"] / max(1, min(steps, 3)),
                            "relres": fp64["relres"],
                            "sampled_operator_launches": {k: {"launches": v[0], "avg_us": round(1e3 * v[1] / max(v[0], 1), 3)}
                                                          for k, v in fp64["families"].items() if v[0]}}
        out["speedup_vs_fp64"] = out["value"] / world / out["fp64_path"]["value"]
        out["C_rel_diff_mixed_vs_fp64"] = abs(C_mixed - C_fp64) / abs(C_fp64)
    h.close()
    return out


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return 0
        sample = SAMPLE_WORKLOAD.get(args.workload, args.workload)
        for _ in range(args.warmup):
            run_oracle_sample(sample, 1)
        t0 = time.perf_counter()
        sec, info = run_oracle_sample(sample, args.steps)
        import workloads as W
        pr = W.named(args.workload)
        nfree = free_dofs_of(args.workload)
        scale = info["free_dofs"] / nfree
        value = scale / sec
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "nelx": pr.nelx, "nely": pr.nely, "p": int(pr.p[0]),
                       "d": int(pr.d[0]), "free_dofs": nfree, "design_values": int(len(pr.rho)),
                       "rtol": args.rtol, "residual_norm": "l2", "sample": sample,
                       "parallelism": "rank 0 only (host cores)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{sample}, median of {args.steps} single-threaded oracle passes "
                                       f"({sec:.2f} s each), scaled by free DOFs"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }), flush=True)
        return 0

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if args.oc_iters > 0:
        out = run_oc_loop(args, rank, world, local_rank)
        if rank == 0:
            print(json.dumps(out), flush=True)
        return 0
    out = run_gpu(args, rank, world, local_rank)
    if rank == 0:
        if not args.no_cpu:
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
