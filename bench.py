#!/usr/bin/env python
"""Benchmark: time to the k smallest eigenpairs at backward-stable tol 1e-8.

Workload (default): generalised pencil from a 3D 7-point Dirichlet Laplacian on
a 64^3 grid (n = 262,144, nnz = 1,810,432), diagonal B with entries U[1, 2]
from the seed, Jacobi preconditioner, k = 64 (block width 71), tol 1e-8 in
the backward-stable criterion of Eq. (9), synthetic seeded inputs.

One step = one complete solve through the C ABI (norm estimates, initial
Rayleigh-Ritz, all iterations of Algorithm 8, exit certification).
  value     device-resident inputs (operator already in HBM), CUDA events on
            the solver's stream around K solves; seconds per solve, lower is
            better.  Arithmetic form: --mode (default: the n-scaled
            contractions emulated on the tensor cores with 6 BF16 slices,
            dtype "f64-emulated-bf16x6"; everything else FP64).
  e2e       the same through the C ABI with host buffers: the operator and X0
            are copied from pinned host memory and the eigenpairs read back,
            per step.
  fp64_form one solve of the same workload in the plain FP64 form on the same
            GPU (CUDA events), with the largest relative eigenvalue difference
            to the timed form (the mixed-versus-FP64 comparison).
The working set (15 blocks of 262,144 x 72 doubles, 151 MB each) is larger than
the 129 MB L2, so no L2 flush is inserted between steps.

roofline: every n-scaled kernel family is HBM-bound on the method's own
bytes (SpMM: CSR arrays plus the block read and written; Gram: 8 n (p + q);
update: 8 n (s + m) [+ 8 n m]); the one with the largest stream time is
reported against the measured copy bandwidth, the others ride along, and the
BF16 digit-product rate of the emulated contractions is a separate diagnostic.

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
GOLDEN = os.path.join(ROOT, "tests", "golden")
# Iterations the CPU oracle needs to converge on a workload with seed 0, read
# from the stored oracle run (tests/golden/oracle_lambda_<workload>.txt,
# written by a script that calls only the oracle); used to extrapolate the
# bounded oracle samples to a full solve.
ORACLE_ITERS_FALLBACK = {"lap3d_64_diagB": 715, "lap2d_32": 101}
# DRAM bytes (read + write) of one launch of a kernel at the workload's full
# shape, from one ncu capture, keyed by the SHA-256 prefix of the source file
# the kernel was built from: a changed source reports traffic null until it
# is captured again.  (workload, kernel family, mode, slices) ->
# (source file, sha16, bytes per launch)
NCU_TRAFFIC = {
    ("lap3d_64_diagB", "update", "ozaki_tc", 6):
        ("paper_1704_07458_gb300/csrc/ozaki_tc.cu", "8abb673856b2052c", 450.009856e6 + 266.715392e6),
}
# algorithmic bytes of one full-shape launch of each family at the workload
# (the unit the traffic above is compared against)
FULL_SHAPE = {"lap3d_64_diagB": {"n": 262144, "s": 213, "m": 142, "p": 213, "q": 142}}


def oracle_iters(workload):
    path = os.path.join(GOLDEN, f"oracle_lambda_{workload}.txt")
    try:
        for line in open(path):
            if line.startswith("iterations"):
                return int(line.split()[1]), "stored oracle run"
    except OSError:
        pass
    return ORACLE_ITERS_FALLBACK.get(workload), "fallback constant"


def source_sha16(rel):
    import hashlib
    try:
        return hashlib.sha256(open(os.path.join(ROOT, rel), "rb").read()).hexdigest()[:16]
    except OSError:
        return None


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


def oracle_child(args):
    """--oracle-child: time `reps` bounded oracle samples in this process (its
    thread count set by the parent through the environment) and print them."""
    import synth
    p = synth.make_problem(args.workload, seed=0)
    out = [oracle_sample(p, 0, args.ref_iters)[1] for _ in range(args.oracle_reps)]
    print(json.dumps({"per_iter": out}), flush=True)


def oracle_timing(workload, iters, reps, threads):
    """Median seconds per oracle iteration over `reps` bounded samples, run in
    a fresh interpreter with `threads` BLAS/OpenMP threads (None: all cores)."""
    env = dict(os.environ)
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        if threads is None:
            env.pop(var, None)
        else:
            env[var] = str(threads)
    env["CUDA_VISIBLE_DEVICES"] = ""  # the oracle is CPU-only
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-child",
                        "--workload", workload, "--ref-iters", str(iters),
                        "--oracle-reps", str(reps)],
                       capture_output=True, text=True, env=env, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError(f"oracle sample failed: {r.stderr[-2000:]}")
    per = json.loads(r.stdout.strip().splitlines()[-1])["per_iter"]
    return statistics.median(per), per


def cpu_baseline_timing(workload):
    """The oracle on this host's cores, per iteration: all cores (median of 3
    samples of 3 iterations) and one thread (median of 3 samples of 2)."""
    return oracle_timing(workload, 3, 3, None), oracle_timing(workload, 2, 3, 1)


def cpu_baseline_line(timing, iters_to_extrapolate, what):
    """The per-iteration oracle timing extrapolated to a full solve."""
    (all_it, all_s), (one_it, one_s) = timing
    return {
        "value": all_it * iters_to_extrapolate, "unit": "s", "cores": os.cpu_count(),
        "kind": "oracle",
        "single_thread": {"value": one_it * iters_to_extrapolate, "unit": "s", "cores": 1},
        "sample": (f"median of 3 samples of 3 oracle iterations (all {os.cpu_count()} cores; "
                   f"{', '.join(f'{x:.2f}' for x in all_s)} s per iteration) and of 3 samples of "
                   f"2 iterations on one thread ({', '.join(f'{x:.2f}' for x in one_s)} s), "
                   f"full workload, setup included, extrapolated per iteration to {what} "
                   f"({iters_to_extrapolate} iterations)")}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import synth
    p = synth.make_problem(args.workload, seed=0)
    full, src = oracle_iters(args.workload)
    if args.warmup:
        oracle_timing(args.workload, 1, 1, None)
    per_it, samples = oracle_timing(args.workload, args.ref_iters, max(1, args.steps), None)
    v = per_it * full
    sample = (f"median of {len(samples)} samples of {args.ref_iters} oracle iterations on the "
              f"full workload (all {os.cpu_count()} cores), extrapolated to the oracle's {full} "
              f"iterations to convergence ({src})")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(args, p),
        "cpu_baseline": {"value": v, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    line["config"]["block_width"] = synth.block_width(p.k, p.n)
    print(json.dumps(line), flush=True)


def mode_dtype(mode, slices):
    """Arithmetic the timed path computes in: FP64, or FP64 emulated by S exact
    BF16 digits per operand on the tensor cores (the n-scaled contractions;
    the rest of the path is FP64)."""
    return "f64" if mode == "f64" else f"f64-emulated-bf16x{slices or 6}"


def workload_config(args, p):
    return {"workload": f"{args.workload}: {p.note}, n={p.n}, nnz={p.A.nnz}, k={p.k}, "
                        f"tol={p.tol}", "n": p.n, "nnz": p.A.nnz, "k": p.k, "tol": p.tol,
            "block_width": None, "gemm_mode": args.mode,
            "dense_eig": {0: "device_layer_le256_else_fp64_syevd", 1: "fp32_syevd_refined",
                          2: "fp64_syevd"}.get(
                getattr(args, "dense_eig", 0), "?"),
            "ozaki_slices": getattr(args, "slices", 0) or 6,
            "l2": "working set > L2 (15 blocks of n x 72 doubles, 151 MB each); no flush",
            "parallelism": "replicas" if int(os.environ.get("WORLD_SIZE", "1")) > 1 else "1gpu"}


def roofline_report(args, tot, steps, peaks):
    """Per-family HBM rate on the method's own bytes; the family with the
    largest stream time is the headline kernel."""
    fam = {
        "spmm": (tot["ms_spmm"], tot["spmm_bytes"]),
        "gram": (tot["ms_gram"], tot["gram_bytes"]),
        "update": (tot["ms_update"], tot["update_bytes"]),
    }
    peak = peaks["hbm_gbs"]
    per = {}
    for k, (ms, by) in fam.items():
        gbs = by / (ms * 1e-3) / 1e9 if ms > 0 else None
        per[k] = {"ms_per_solve": ms / steps, "bytes_per_solve": by / steps, "gbs": gbs,
                  "frac": gbs / peak if gbs else None}
    for k, key, tkey in (("gram", "gram_flops", "gram_tensor_flops"),
                         ("update", "update_flops", "update_tensor_flops")):
        ms = fam[k][0]
        per[k]["fp64_equivalent_tflops"] = tot[key] / (ms * 1e-3) / 1e12 if ms > 0 else None
        if args.mode != "f64" and ms > 0:
            bf = tot[tkey] / (ms * 1e-3) / 1e12
            per[k]["bf16_digit_tflops"] = bf
            per[k]["bf16_digit_frac_of_sustained"] = bf / peaks["bf16_tflops_sustained"]
    dom = max(fam, key=lambda k: fam[k][0])
    traffic, tsrc = None, "no ncu capture of this kernel family at this shape"
    key = (args.workload, dom, args.mode, args.slices or 6)
    if key in NCU_TRAFFIC:
        rel, sha, by = NCU_TRAFFIC[key]
        if source_sha16(rel) == sha:
            traffic, tsrc = by, f"ncu dram read + write of one full-shape launch ({rel} @ {sha})"
        else:
            tsrc = f"{rel} changed since the ncu capture: traffic not re-measured"
    shape = FULL_SHAPE.get(args.workload)
    algo = None
    if shape and dom == "update":
        algo = 8.0 * shape["n"] * (shape["s"] + shape["m"])
    elif shape and dom == "gram":
        algo = 8.0 * shape["n"] * (shape["p"] + shape["q"])
    return {"bound": "hbm", "kernel": dom, "achieved": per[dom]["gbs"], "peak": peak,
            "unit": "GB/s", "frac": per[dom]["frac"], "traffic": traffic,
            "traffic_unit": "bytes per full-shape launch", "traffic_source": tsrc,
            "algorithmic_bytes_per_full_shape_launch": algo,
            "peak_source": "measured hbm_gbs (MEASURED_PEAKS.json)"
            if not peaks.get("fallback") else "fallback 6.8 TB/s",
            "families": per}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="ozaki_tc", choices=["f64", "ozaki", "ozaki_tc"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--ref-iters", type=int, default=3)
    ap.add_argument("--oracle-child", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--oracle-reps", type=int, default=3, help=argparse.SUPPRESS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-form", action="store_true",
                    help="skip the one-solve FP64-form comparison")
    ap.add_argument("--maxit", type=int, default=0,
                    help="cap the iterations of every solve (0: the solver's default); "
                         "a capped run is a bounded profile of the same step, not a bench value")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--slices", type=int, default=0,
                    help="Ozaki slices of the emulated contractions (0: 6; 3..7)")
    ap.add_argument("--dense-eig", type=int, default=0, choices=[0, 1, 2],
                    help="eigensolver of the projected pencils (the solver's dense_eig option)")
    args = ap.parse_args()
    if args.oracle_child:
        return oracle_child(args)
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import synth
    import paper_1704_07458_gb300 as gb

    rank, world, local = dist_env()
    # the CPU baseline runs first, in interpreters of its own, before this
    # process touches the GPU
    cpu_timing = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_timing = cpu_baseline_timing(args.workload)
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
    lam_h = lam.detach().cpu().numpy().copy()

    # ---- end to end through the C ABI with host buffers
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_rp, h_ci, h_v = pin(p.A.rowptr), pin(p.A.col), pin(p.A.val)
    h_b = pin(p.b_diag) if p.b_diag is not None else None
    lamh = torch.empty(p.k, dtype=torch.float64).pin_memory()
    X_h = torch.empty((p.n, p.k), dtype=torch.float64).pin_memory()
    be_h = torch.empty(p.k, dtype=torch.float64).pin_memory()
    h2d = (h_rp.numel() * 4 + h_ci.numel() * 4 + h_v.numel() * 8 +
           (h_b.numel() * 8 if h_b is not None else 0) + X0h.numel() * 8)
    d2h = (lamh.numel() + X_h.numel() + be_h.numel()) * 8
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
                                     lamh, X_h, p.k, gb.LOBPCG_MEM_HOST, be_h)
        assert rc_e in ok, rc_e
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps if e2e_steps else None
    if e2e_s is not None:
        e2e_s = max_over_ranks(e2e_s)

    # ---- the plain FP64 form of the same solve on the same GPU (one solve)
    fp64_form = None
    if not args.no_fp64_form and args.mode != "f64":
        with gb.Solver(stream=stream, gemm_mode="f64", maxit=args.maxit,
                       dense_eig=args.dense_eig) as s64:
            s64.set_operator(A_rp, A_ci, A_v, b_diag=bd)
            torch.cuda.synchronize()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            lam64, _, it64, be64, rc64 = s64.solve(p.k, p.tol, X0=X0d, seed=seed, device=True)
            f1.record(stream)
            torch.cuda.synchronize()
            st64 = s64.stats()
        l64 = lam64.detach().cpu().numpy()
        fp64_form = {
            "value": f0.elapsed_time(f1) / 1e3, "unit": "s", "dtype": "f64", "status": int(rc64),
            "iterations": int(it64), "max_backward_error": float(be64.max().item()),
            "orth_error": float(st64["orth_error"]),
            "max_rel_lambda_diff_vs_timed_form": float(np.max(np.abs(lam_h - l64) / np.abs(l64))),
            "speedup_of_timed_form": (f0.elapsed_time(f1) / 1e3) / (ms / 1e3),
            "note": "one solve, not warmed up; CUDA events on the same stream"}

    roofline = roofline_report(args, tot, args.steps, peaks)
    line = {
        "metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": mode_dtype(args.mode, args.slices), "data": "synthetic",
        "config": workload_config(args, p),
        "iterations": int(it), "max_backward_error": bemax,
        "orth_error": float(st["orth_error"]),
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h),
                "iterations": None if it_e is None else int(it_e)},
        "gpu_launches": int(tot["gpu_launches"]),
        "clocks": clk, "roofline": roofline,
        "fp64_form": fp64_form,
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
                   "eig_check_failures": {k: int(st[f"eig_check_{k}"]) for k in
                                          ("orthogonality", "wide_cluster", "nonfinite")},
                   "slice_escalation_iteration": int(st["slice_escalation_iteration"]),
                   "host_syncs_per_solve": int(tot["host_syncs"]) // max(1, args.steps),
                   "launches_per_solve": int(tot["gpu_launches"]) // max(1, args.steps)},
    }
    line["config"]["block_width"] = int(st["n_x"])
    if cpu_timing is not None:
        line["cpu_baseline"] = cpu_baseline_line(cpu_timing, int(it),
                                                 "this run's iteration count")
    if rank == 0:
        print(json.dumps(line), flush=True)
    solver.close()
    e2e_solver.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
