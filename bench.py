#!/usr/bin/env python
"""Benchmark: time to the k smallest eigenpairs at backward-stable tol 1e-8.

Workload (default): generalised pencil from a 3D 7-point Dirichlet Laplacian on
a 64^3 grid (n = 262,144, nnz = 1,810,432), diagonal B with entries U[1, 2]
from the seed, Jacobi preconditioner, k = 64 (block width 71), tol 1e-8 in
the backward-stable criterion of Eq. (9), synthetic seeded inputs.

One step = one complete solve through the C ABI (norm estimates, initial
Rayleigh-Ritz, all iterations of Algorithm 8, exit certification).
  value  device-resident inputs (operator already in HBM), CUDA events on the
         solver's stream around K solves; seconds per solve, lower is better.
  e2e    the same through the C ABI with host buffers: the operator and X0 are
         copied from pinned host memory and the eigenpairs read back, per step.
The working set (15 blocks of 262,144 x 72 doubles, 151 MB each) is larger than
the 129 MB L2, so no L2 flush is inserted between steps.

--impl reference times the CPU oracle (plain FP64 numpy) on a bounded sample
of the same workload and extrapolates to a full solve.
Under torchrun (N > 1) every rank solves its own replica (seed = rank); there
is no collective on the data path ("replicas only").
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-k-eigenpairs at backward-stable tol 1e-8; SpMM HBM GB/s; Gram TFLOP/s"
WORKLOAD = "lap3d_64_diagB"
# Iterations the CPU oracle needs to converge on this workload with seed 0
# (measured by running oracle.lobpcg to convergence on the same inputs); used
# to extrapolate the bounded oracle samples to a full solve.
ORACLE_ITERS = {"lap3d_64_diagB": 726, "lap2d_32": 101}
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 (CUDA cores and DMMA), nominal
# DRAM bytes (read + write) of one launch of the dominant kernel, from one ncu
# capture of the same kernel build at the workload's shape
# (profiles/ozaki_update_tc_kernel_n262144_s213_m142.md); None where none is
# taken.
NCU_TRAFFIC = {("lap3d_64_diagB", "update", "ozaki_tc", 6): 448.449280e6 + 263.597312e6}


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "fallback": True}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.file.flush()
        rows = [l.split(",") for l in open(self.file.name) if l.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for name, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(v):
    """Largest value of v over the ranks (v unchanged on a single process).
    NCCL reduces a CUDA tensor, gloo a CPU one."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return v
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def oracle_sample(p, seed, iters):
    """Run the CPU oracle for `iters` iterations; return (seconds, seconds/iteration)."""
    import numpy as np
    import synth
    from oracle import lobpcg as L
    nx = synth.block_width(p.k)
    X0 = synth.normal_block(seed, synth.STREAM_X0, p.n, nx)
    Om = synth.normal_block(seed, synth.STREAM_OMEGA, p.n, 16).T
    pen = L.Pencil(p.n, (p.A.rowptr, p.A.col, p.A.val), p.b_diag, p.kdiag)
    t0 = time.perf_counter()
    L.lobpcg(pen, X0, p.k, p.tol, Om, L.Options(maxit=iters, certify=False))
    dt = time.perf_counter() - t0
    return dt, dt / iters


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import synth
    p = synth.make_problem(args.workload, seed=0)
    sample_iters = args.ref_iters
    full = ORACLE_ITERS.get(args.workload)
    for _ in range(args.warmup):
        oracle_sample(p, 0, 1)
    vals = []
    for _ in range(args.steps):
        _, per_it = oracle_sample(p, 0, sample_iters)
        vals.append(per_it * full)
    v = statistics.median(vals)
    sample = (f"{sample_iters} oracle iterations per step on the full workload, "
              f"extrapolated to the oracle's {full} iterations to convergence")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(args, p),
        "cpu_baseline": {"value": v, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(args, p):
    return {"workload": f"{args.workload}: {p.note}, n={p.n}, nnz={p.A.nnz}, k={p.k}, "
                        f"tol={p.tol}", "n": p.n, "nnz": p.A.nnz, "k": p.k, "tol": p.tol,
            "block_width": None, "gemm_mode": args.mode,
            "dense_eig": "fp64_syevd" if getattr(args, "dense_eig", 0) == 0 else "fp32_refined",
            "ozaki_slices": getattr(args, "slices", 0) or 6,
            "l2": "working set > L2 (15 blocks of n x 72 doubles, 151 MB each); no flush",
            "parallelism": "replicas" if int(os.environ.get("WORLD_SIZE", "1")) > 1 else "1gpu"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="ozaki_tc", choices=["f64", "ozaki", "ozaki_tc"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--ref-iters", type=int, default=6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--maxit", type=int, default=0,
                    help="cap the iterations of every solve (0: the solver's default of 2000); "
                         "a capped run is a bounded profile of the same step, not a bench value")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--slices", type=int, default=0,
                    help="Ozaki slices of the emulated contractions (0: 6; 3..7)")
    ap.add_argument("--dense-eig", type=int, default=0, choices=[0, 1],
                    help="eigensolver of the projected pencils: 0 FP64 syevd, 1 FP32 refined "
                         "to FP64")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import synth
    import paper_1704_07458_gb300 as gb

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    peaks = load_peaks()
    seed = rank
    p = synth.make_problem(args.workload, seed=seed)
    stream = torch.cuda.current_stream()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    A_rp, A_ci, A_v = dev(p.A.rowptr), dev(p.A.col), dev(p.A.val)
    bd = dev(p.b_diag) if p.b_diag is not None else None

    solver = gb.Solver(stream=stream, gemm_mode=args.mode, maxit=args.maxit,
                       dense_eig=args.dense_eig, ozaki_slices=args.slices)
    solver.set_operator(A_rp, A_ci, A_v, b_diag=bd)
    # the seeded starting block, resident in HBM like the operator; the e2e leg
    # below copies the same block from pinned host memory
    nx = synth.block_width(p.k)
    X0h = torch.from_numpy(synth.normal_block(seed, synth.STREAM_X0, p.n, nx)).pin_memory()
    X0d = X0h.cuda()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        lam, X, it, be, rc = solver.solve(p.k, p.tol, X0=X0d, seed=seed, device=True)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tot = {}
    e0.record(stream)
    for _ in range(args.steps):
        lam, X, it, be, rc = solver.solve(p.k, p.tol, X0=X0d, seed=seed, device=True)
        st = solver.stats()
        for key, v in st.items():
            tot[key] = tot.get(key, 0) + v
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms)
    ok = (gb.LOBPCG_OK, gb.LOBPCG_ERR_NOT_CONVERGED) if args.maxit else (gb.LOBPCG_OK,)
    assert rc in ok, f"solve failed: {rc}"
    bemax = float(be.max().item())

    # ---- end to end through the C ABI with host buffers
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_rp, h_ci, h_v = pin(p.A.rowptr), pin(p.A.col), pin(p.A.val)
    h_b = pin(p.b_diag) if p.b_diag is not None else None
    lam_h = torch.empty(p.k, dtype=torch.float64).pin_memory()
    X_h = torch.empty((p.n, p.k), dtype=torch.float64).pin_memory()
    be_h = torch.empty(p.k, dtype=torch.float64).pin_memory()
    h2d = (h_rp.numel() * 4 + h_ci.numel() * 4 + h_v.numel() * 8 +
           (h_b.numel() * 8 if h_b is not None else 0) + X0h.numel() * 8)
    d2h = (lam_h.numel() + X_h.numel() + be_h.numel()) * 8
    e2e_solver = gb.Solver(stream=stream, gemm_mode=args.mode, maxit=args.maxit,
                           dense_eig=args.dense_eig, ozaki_slices=args.slices)
    e2e_steps = 0 if args.no_e2e else max(1, args.steps)
    it_e = None
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        rc_e = gb.lobpcg_set_operator(e2e_solver.h, p.n, h_rp, h_ci, h_v, p.A.nnz, B_diag=h_b,
                                      mem=gb.LOBPCG_MEM_HOST)
        assert rc_e == 0
        rc_e, it_e = gb.lobpcg_solve(e2e_solver.h, p.k, p.tol, X0h, nx, seed, gb.LOBPCG_MEM_HOST,
                                  lam_h, X_h, p.k, gb.LOBPCG_MEM_HOST, be_h)
        assert rc_e in ok, rc_e
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps if e2e_steps else None
    if e2e_s is not None:
        e2e_s = max_over_ranks(e2e_s)

    # ---- roofline of the dominant n-scaled kernel over the timed region
    # FP64 mode: FP64 flops on the CUDA cores ("alu"); emulated modes: the BF16
    # tensor-core flops of the digit products ("tensor").
    f64 = args.mode == "f64"
    phases = {
        "spmm": (tot["ms_spmm"], tot["spmm_bytes"], "hbm"),
        "gram": (tot["ms_gram"], tot["gram_flops"] if f64 else tot["gram_tensor_flops"],
                 "alu" if f64 else "tensor"),
        "update": (tot["ms_update"], tot["update_flops"] if f64 else tot["update_tensor_flops"],
                   "alu" if f64 else "tensor"),
    }
    dom = max(phases, key=lambda k: phases[k][0])
    t_ms, work, bound = phases[dom]
    if bound == "hbm":
        achieved = work / (t_ms * 1e-3) / 1e9
        peak, unit = peaks["hbm_gbs"], "GB/s"
        peak_src = "measured hbm_gbs"
    elif bound == "alu":
        achieved = work / (t_ms * 1e-3) / 1e12
        peak, unit = FP64_NOMINAL_TFLOPS, "TFLOP/s"
        peak_src = "nominal GB300 FP64 rate (no measured FP64 peak)"
    else:
        achieved = work / (t_ms * 1e-3) / 1e12
        peak, unit = peaks["bf16_tflops_sustained"], "TFLOP/s"
        peak_src = "measured bf16_tflops_sustained"
    per_phase = {k: {"ms_per_solve": v[0] / args.steps,
                     "rate": (v[1] / (v[0] * 1e-3) / (1e9 if v[2] == "hbm" else 1e12))
                     if v[0] > 0 else None,
                     "unit": {"hbm": "GB/s", "alu": "FP64 TFLOP/s",
                              "tensor": "BF16 TFLOP/s"}[v[2]]}
                 for k, v in phases.items()}
    for k, key in (("gram", "gram_flops"), ("update", "update_flops")):
        t = phases[k][0]
        per_phase[k]["fp64_equivalent_tflops"] = tot[key] / (t * 1e-3) / 1e12 if t > 0 else None
    traffic = NCU_TRAFFIC.get((args.workload, dom, args.mode, args.slices or 6))
    roofline = {"bound": bound, "kernel": dom, "achieved": achieved, "peak": peak,
                "unit": unit, "frac": achieved / peak, "traffic": traffic,
                "traffic_unit": "bytes per launch (ncu dram read + write)",
                "peak_source": peak_src, "phases": per_phase}

    line = {
        "metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "config": workload_config(args, p),
        "iterations": int(it), "max_backward_error": bemax,
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h),
                "iterations": None if it_e is None else int(it_e)},
        "gpu_launches": int(tot["gpu_launches"]),
        "clocks": clk, "roofline": roofline,
        # per-solve phase times (CUDA events on the solver's stream, exclusive:
        # they add up to the stream time; "total" is the host wall clock)
        "phases_ms_per_solve": {
            k[3:]: tot[k] / args.steps for k in
            ("ms_spmm", "ms_gram", "ms_update", "ms_residual", "ms_small_dense", "ms_ortho",
             "ms_other", "ms_total")},
        "solver": {"flip_iteration": int(st["flip_iteration"]),
                   "ortho_calls": int(st["ortho_calls"]), "svqb_passes": int(st["svqb_passes"]),
                   "dropped_columns": int(st["dropped_columns"]),
                   "eig_calls": int(st["eig_calls"]), "eig_fallbacks": int(st["eig_fallbacks"]),
                   "slice_escalation_iteration": int(st["slice_escalation_iteration"]),
                   "launches_per_solve": int(tot["gpu_launches"]) // max(1, args.steps)},
    }
    line["config"]["block_width"] = int(st["n_x"])
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample_iters = args.ref_iters
        dt, per_it = oracle_sample(p, seed, sample_iters)
        line["cpu_baseline"] = {
            "value": per_it * it, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{sample_iters} oracle iterations ({dt:.1f} s) on the full workload, "
                      f"extrapolated per iteration to this run's {it} iterations"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    solver.close()
    e2e_solver.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
