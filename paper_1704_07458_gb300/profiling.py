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
"""
import argparse
import collections
import csv
import json
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
        Y = torch.empty(n, m, **dev)

        def run():
            rc = nat.lobpcg_update(n, S, s, s, C, s, m, 1.0, 0.0, None, 0, Y, m, mode_id,
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
    a = ap.parse_args(argv)
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
