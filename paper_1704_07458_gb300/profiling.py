"""Profiling helpers: single-kernel timing through the C ABI and ncu launch lists.

  python -m paper_1704_07458_gb300.profiling kernel update [--mode ozaki_tc] [--slices 6]
      times lobpcg_update (or gram / spmm) on the shapes one iteration of the
      k = 64 solve on the 64^3 pencil uses (n = 262,144 rows, n_s = 213 basis
      columns, 2 n_x = 142 output columns), CUDA events on the launching
      stream, inputs larger than L2; prints one JSON line.  This is also the
      small, self-contained command to capture under ncu (-k, -c 1..3).
  python -m paper_1704_07458_gb300.profiling launches launches.csv
      summarises an ncu launch list (--metrics gpu__time_duration.sum --csv):
      launches, total device time and share per kernel.
  python -m paper_1704_07458_gb300.profiling forms [--workload lap3d_64_diagB]
      one timed solve per arithmetic form (FP64, mma.sync emulation, tcgen05
      emulation with 7, 6, 5 slices): seconds, iterations, backward error and
      the largest relative eigenvalue difference from the FP64 form.
  python -m paper_1704_07458_gb300.profiling versions [--workload ...] [--N 32 --k 32]
      the component breakdown of the implementation versions of Sec. 6.2
      (Fig. 2 methodology) on a synthetic workload: CHL, AHL, Algorithm 8's
      basis selection with orthogonalisation on every iteration and only
      identity (12), the same with orthogonalisation skipped while cond(R)
      allows, and Algorithm 8; per version the time, iterations, per-phase
      times, svqb passes per orthogonalisation call and the eigenvalue
      difference from Algorithm 8.
  python -m paper_1704_07458_gb300.profiling ksweep [--workload ...] [--ks 16,32,64,128]
      time to k eigenpairs against k on one operator (Fig. 4 methodology).
"""
import argparse
import collections
import csv
import json
import os
import sys

SCALE = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3}

# digit pairs (s, t) with s + t <= S + 1: the BF16 products of one emulated FP64 product
def pairs(slices):
    return sum(L - 1 for L in range(2, slices + 2)) if slices > 0 else 0


def kernel_name(raw):
    s = raw.replace("void ", "").replace("(anonymous namespace)::", "").replace("<unnamed>::", "")
    s = s.split("(")[0]
    return s.split("<")[0].strip()


def summarize_launches(path, out=sys.stdout):
    rows = list(csv.reader(open(path)))
    hi = next(i for i, r in enumerate(rows) if r and r[0] == "ID")
    hdr = rows[hi]
    ki, mi, vi, ui = (hdr.index("Kernel Name"), hdr.index("Metric Name"),
                      hdr.index("Metric Value"), hdr.index("Metric Unit"))
    tot = collections.defaultdict(float)
    cnt = collections.Counter()
    for r in rows[hi + 1:]:
        if len(r) <= vi or r[mi] != "gpu__time_duration.sum":
            continue
        name = kernel_name(r[ki])
        tot[name] += float(r[vi].replace(",", "")) * SCALE.get(r[ui], 1.0)
        cnt[name] += 1
    T = sum(tot.values())
    print(f"{'kernel':44s} {'launches':>8s} {'total_us':>11s} {'share':>7s}", file=out)
    for k, v in sorted(tot.items(), key=lambda x: -x[1]):
        print(f"{k[:44]:44s} {cnt[k]:8d} {v:11.1f} {100 * v / T:6.1f}%", file=out)
    print(f"{'total':44s} {sum(cnt.values()):8d} {T:11.1f}", file=out)
    return tot, cnt


def time_kernel(which, mode, slices, reps, warmup, n, s, m):
    import numpy as np
    import torch
    from . import _native as nat
    mode_id = {"f64": nat.LOBPCG_GEMM_F64, "ozaki": nat.LOBPCG_GEMM_OZAKI,
               "ozaki_tc": nat.LOBPCG_GEMM_OZAKI_TC}[mode]
    g = torch.Generator(device="cuda")
    g.manual_seed(1)
    st = torch.cuda.current_stream()
    dev = dict(dtype=torch.float64, device="cuda")
    if which == "update":
        S = torch.randn(n, s, generator=g, **dev)
        C = torch.randn(m * s, generator=g, **dev)
        ldy = (m + 7) // 8 * 8  # the solver's blocks: leading dimension rounded up to 8 doubles
        Y = torch.empty(n, ldy, **dev)

        def run():
            rc = nat.lobpcg_update(n, S, s, s, C, s, m, 1.0, 0.0, None, 0, Y, ldy, mode_id,
                                   slices, st)
            assert rc == 0, rc
        flops = 2.0 * n * s * m
        tensor = 2.0 * n * s * m * pairs(slices) if mode != "f64" else 0.0
        bytes_ = 8.0 * n * (s + m)
    elif which == "gram":
        U = torch.randn(n, s, generator=g, **dev)
        V = torch.randn(n, m, generator=g, **dev)
        G = torch.empty(s * m, **dev)
        wb = nat.lobpcg_gram_workspace(n, s, m, mode_id, slices)
        W = torch.empty(max(wb, 8), dtype=torch.uint8, device="cuda")

        def run():
            rc = nat.lobpcg_gram(n, U, s, s, V, m, m, G, s, mode_id, slices, W, wb, st)
            assert rc == 0, rc
        flops = 2.0 * n * s * m
        tensor = 2.0 * n * s * m * pairs(slices) if mode != "f64" else 0.0
        bytes_ = 8.0 * n * (s + m)
    elif which == "spmm":
        # the solver's shape: A W with the diagonal-B product fused, blocks
        # with the leading dimension rounded up to 8 doubles
        import synth
        A = synth.laplacian_3d_dirichlet(64)
        n = A.n
        ld = (m + 7) // 8 * 8
        rp = torch.from_numpy(A.rowptr).cuda()
        ci = torch.from_numpy(A.col).cuda()
        va = torch.from_numpy(A.val).cuda()
        b = torch.rand(n, generator=g, **dev) + 1.0
        X = torch.randn(n, ld, generator=g, **dev)
        Y = torch.empty(n, ld, **dev)
        BY = torch.empty(n, ld, **dev)

        def run():
            rc = nat.lobpcg_spmm(n, rp, ci, va, X, ld, m, Y, ld, b, BY, ld, st)
            assert rc == 0, rc
        flops = 2.0 * A.nnz * m
        tensor = 0.0
        bytes_ = 12.0 * A.nnz + 4.0 * (n + 1) + 16.0 * n * m + 8.0 * n + 16.0 * n * m
    elif which == "residual":
        # R = AX - BX diag(theta), W = R / kdiag, Eq. (9) norms; diagonal B
        ld = (m + 7) // 8 * 8
        X = torch.randn(n, ld, generator=g, **dev)
        AX = torch.randn(n, ld, generator=g, **dev)
        BX = torch.randn(n, ld, generator=g, **dev)
        W = torch.empty(n, ld, **dev)
        th = torch.rand(m, generator=g, **dev)
        kd = torch.rand(n, generator=g, **dev) + 1.0
        be = torch.empty(m, **dev)

        def run():
            rc = nat.lobpcg_residual(n, X, AX, BX, ld, m, 0, th, kd, W, ld, 12.0, 2.0, be, st)
            assert rc == 0, rc
        flops = 0.0
        tensor = 0.0
        bytes_ = 8.0 * n * m * 4 + 8.0 * n
    else:
        raise ValueError(which)
    for _ in range(warmup):
        run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        run()
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(reps, 1)
    return {"kernel": which, "mode": mode, "slices": slices, "n": n, "s": s, "m": m,
            "ms": ms, "fp64_equivalent_tflops": flops / (ms * 1e-3) / 1e12,
            "bf16_tensor_tflops": tensor / (ms * 1e-3) / 1e12 if tensor else None,
            "gbs": bytes_ / (ms * 1e-3) / 1e9}


def compare_forms(workload, forms):
    """Time one solve of `workload` per arithmetic form and compare its
    eigenvalues with the FP64 form's (the first form listed must be f64)."""
    import time
    import numpy as np
    import torch
    import synth
    from . import Solver
    p = synth.make_problem(workload, seed=0)
    nx = synth.block_width(p.k)
    X0 = torch.from_numpy(synth.normal_block(0, synth.STREAM_X0, p.n, nx)).cuda()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    A = (dev(p.A.rowptr), dev(p.A.col), dev(p.A.val))
    bd = dev(p.b_diag) if p.b_diag is not None else None
    ref = None
    for mode, slices in forms:
        s = Solver(stream=torch.cuda.current_stream(), gemm_mode=mode, ozaki_slices=slices)
        s.set_operator(*A, b_diag=bd)
        s.solve(p.k, p.tol, X0=X0, device=True)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lam, X, it, be, rc = s.solve(p.k, p.tol, X0=X0, device=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        lam = lam.cpu().numpy()
        if ref is None:
            ref = lam
        out = {"workload": workload, "mode": mode, "slices": slices or 6, "status": rc,
               "seconds": dt, "iterations": it, "max_backward_error": float(be.max().item()),
               "max_rel_lambda_diff_vs_f64": float(np.max(np.abs(lam - ref) / np.abs(ref)))}
        print(json.dumps(out), flush=True)
        s.close()


# (label, solver options) of the versions of Sec. 6.2, Fig. 2; the blockwise
# basis update that separates versions 1/2 and 3/4 there is this library's
# tiled update in every version
VERSIONS = [
    ("1-2 CHL", dict(basis=1)),
    ("3-4 AHL", dict(basis=2)),
    ("5 robust ortho every it, (12) only", dict(basis=0, gram_blocks=1, tau_skip=1.0)),
    ("6 + skip ortho", dict(basis=0, gram_blocks=1)),
    ("7 Algorithm 8", dict(basis=0)),
]


def _solve_once(p, opts, X0, warm=True):
    """One timed solve (CUDA events on the solver's stream) -> (lam, stats dict)."""
    import numpy as np
    import torch
    from . import Solver
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    st_ = torch.cuda.current_stream()
    s = Solver(stream=st_, **opts)
    s.set_operator(dev(p.A.rowptr), dev(p.A.col), dev(p.A.val),
                   b_diag=None if p.b_diag is None else dev(p.b_diag))
    if warm:
        s.solve(p.k, p.tol, X0=X0, device=True, raise_on_error=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st_)
    lam, X, it, be, rc = s.solve(p.k, p.tol, X0=X0, device=True, raise_on_error=False)
    e1.record(st_)
    torch.cuda.synchronize()
    st = s.stats()
    s.close()
    st["seconds"] = e0.elapsed_time(e1) / 1e3
    st["status"] = rc
    st["max_backward_error"] = float(be.max().item())
    return lam.cpu().numpy(), st


def versions(workload, mode, kw):
    import numpy as np
    import torch
    import synth
    p = synth.make_problem(workload, seed=0, **kw)
    nx = synth.block_width(p.k, p.n)
    X0 = torch.from_numpy(synth.normal_block(0, synth.STREAM_X0, p.n, nx)).cuda()
    rows, ref = [], None
    for label, opts in reversed(VERSIONS):
        lam, st = _solve_once(p, dict(gemm_mode=mode, maxit=6000, **opts), X0)
        if ref is None:
            ref = lam
        rows.append((label, st, float(np.max(np.abs(lam - ref) / np.abs(ref)))))
    rows.reverse()
    out = {"workload": workload, "n": p.n, "k": p.k, "mode": mode, "versions": []}
    for label, st, dl in rows:
        out["versions"].append({
            "version": label, "status": st["status"], "seconds": st["seconds"],
            "iterations": st["iterations"], "max_backward_error": st["max_backward_error"],
            "ms": {k[3:]: st[k] for k in ("ms_spmm", "ms_gram", "ms_update", "ms_residual",
                                          "ms_small_dense", "ms_ortho", "ms_other")},
            "ortho_calls": st["ortho_calls"],
            "svqb_passes_per_ortho_call": st["svqb_passes"] / max(1, st["ortho_calls"]),
            "flip_iteration": st["flip_iteration"], "dropped_columns": st["dropped_columns"],
            "max_rel_lambda_diff_vs_algorithm8": dl})
    print(json.dumps(out), flush=True)
    return out


def ksweep(workload, mode, ks, kw):
    import torch
    import synth
    out = {"workload": workload, "mode": mode, "points": []}
    for k in ks:
        p = synth.make_problem(workload, seed=0, k=k, **kw)
        nx = synth.block_width(p.k, p.n)
        X0 = torch.from_numpy(synth.normal_block(0, synth.STREAM_X0, p.n, nx)).cuda()
        lam, st = _solve_once(p, dict(gemm_mode=mode, maxit=6000), X0, warm=True)
        out["points"].append({
            "k": k, "n_x": nx, "status": st["status"], "seconds": st["seconds"],
            "iterations": st["iterations"], "max_backward_error": st["max_backward_error"],
            "ms_per_iteration": 1e3 * st["seconds"] / max(1, st["iterations"]),
            "ms": {kk[3:]: st[kk] for kk in ("ms_spmm", "ms_gram", "ms_update", "ms_residual",
                                             "ms_small_dense", "ms_ortho", "ms_other")}})
        print(json.dumps(out["points"][-1]), flush=True)
    print(json.dumps(out), flush=True)
    return out


def mma_rate():
    """Build and run the standalone tcgen05.mma rate probe
    (csrc/probes/tcgen05_mma_rate.cu): cycles per M = 128, K = 16 MMA against
    N, operand layout and issuing thread.  Needs a GB300; prints its lines."""
    import subprocess
    from . import build as b
    src = os.path.join(os.path.dirname(__file__), "csrc", "probes", "tcgen05_mma_rate.cu")
    exe = os.path.join(b.OUT, "tcgen05_mma_rate")
    os.makedirs(b.OUT, exist_ok=True)
    subprocess.run([b._nvcc(), *b.ARCH, "-O3", "-o", exe, src], check=True)
    return subprocess.run([exe], check=True).returncode


def main(argv=None):
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    k = sub.add_parser("kernel")
    k.add_argument("which", choices=["update", "gram", "spmm", "residual"])
    k.add_argument("--mode", default="ozaki_tc", choices=["f64", "ozaki", "ozaki_tc"])
    k.add_argument("--slices", type=int, default=6)
    k.add_argument("--reps", type=int, default=5)
    k.add_argument("--warmup", type=int, default=3)
    k.add_argument("--n", type=int, default=262144)
    k.add_argument("--s", type=int, default=213)
    k.add_argument("--m", type=int, default=142)
    l = sub.add_parser("launches")
    l.add_argument("csv")
    f = sub.add_parser("forms")
    f.add_argument("--workload", default="lap3d_64_diagB")
    v = sub.add_parser("versions")
    v.add_argument("--workload", default="lap3d_64_diagB")
    v.add_argument("--mode", default="f64", choices=["f64", "ozaki", "ozaki_tc"])
    v.add_argument("--N", type=int, default=0)
    v.add_argument("--k", type=int, default=0)
    ks = sub.add_parser("ksweep")
    ks.add_argument("--workload", default="lap3d_64_diagB")
    ks.add_argument("--mode", default="ozaki_tc", choices=["f64", "ozaki", "ozaki_tc"])
    ks.add_argument("--ks", default="16,32,64,128")
    ks.add_argument("--N", type=int, default=0)
    sub.add_parser("mma-rate")
    a = ap.parse_args(argv)
    if a.cmd == "mma-rate":
        return mma_rate()
    if a.cmd == "versions":
        kw = {kk: vv for kk, vv in (("N", a.N), ("k", a.k)) if vv}
        return versions(a.workload, a.mode, kw)
    if a.cmd == "ksweep":
        kw = {"N": a.N} if a.N else {}
        return ksweep(a.workload, a.mode, [int(x) for x in a.ks.split(",")], kw)
    if a.cmd == "launches":
        summarize_launches(a.csv)
    elif a.cmd == "forms":
        compare_forms(a.workload, [("f64", 0), ("ozaki", 6), ("ozaki_tc", 7), ("ozaki_tc", 6),
                                   ("ozaki_tc", 5)])
    else:
        print(json.dumps(time_kernel(a.which, a.mode, a.slices, a.reps, a.warmup, a.n, a.s,
                                     a.m)), flush=True)


if __name__ == "__main__":
    main()
