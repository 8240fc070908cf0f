"""Write the CPU oracle's eigenvalues of a full-size workload to a text fixture.

The stored values come from the plain FP64 oracle (Algorithm 8 of Duersch,
Shao, Yang, Gu, 2018, as restated in oracle/lobpcg.py) run to convergence on
the seeded synthetic inputs of synth/, with the same starting block X0
(Philox stream 1), the same Gaussian sketch Omega (stream 5) and the same
tolerance as the GPU solve.  Nothing here calls the CUDA library.

    python tests/golden/make_oracle_lambda.py lap3d_64_diagB
    python tests/golden/make_oracle_lambda.py lap2d_512_V --maxit 6000

writes tests/golden/oracle_lambda_<workload>.txt.
"""
import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import lobpcg as L  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--maxit", type=int, default=2000)
    args = ap.parse_args()
    p = synth.make_problem(args.workload, seed=args.seed)
    nx = synth.block_width(p.k, p.n)
    X0 = synth.normal_block(args.seed, synth.STREAM_X0, p.n, nx)
    Om = synth.normal_block(args.seed, synth.STREAM_OMEGA, p.n, 16).T
    pen = L.Pencil(p.n, (p.A.rowptr, p.A.col, p.A.val), p.b_diag, p.kdiag)
    t0 = time.perf_counter()
    r = L.lobpcg(pen, X0, p.k, p.tol, Om, L.Options(maxit=args.maxit))
    dt = time.perf_counter() - t0
    if r.status != L.OK:
        raise SystemExit(f"oracle did not converge (status {r.status}, {r.iters} iterations)")
    out = os.path.join(HERE, f"oracle_lambda_{args.workload}.txt")
    with open(out, "w") as f:
        f.write(f"# CPU oracle (plain FP64 Algorithm 8, oracle/lobpcg.py) eigenvalues of the\n"
                f"# workload {args.workload}: {p.note}, n={p.n}, k={p.k}, tol={p.tol},\n"
                f"# seed {args.seed} (X0 = Philox stream 1, Omega = stream 5), block width {nx}.\n"
                f"# Written by tests/golden/make_oracle_lambda.py; the oracle converged in\n"
                f"# {r.iters} iterations ({dt:.0f} s on {os.cpu_count()} host cores), max backward\n"
                f"# error (Eq. 9) {float(np.max(r.be)):.3e}, flip to orthogonalisation at iteration\n"
                f"# {r.stats['flip_iter']}.\n")
        f.write(f"iterations {r.iters}\n")
        f.write(f"norm_a {float(r.normA)!r}\n")
        f.write(f"norm_b {float(r.normB)!r}\n")
        for i, (lam, be) in enumerate(zip(r.lam, r.be)):
            f.write(f"lambda {i} {float(lam)!r} {float(be)!r}\n")
    print(out, r.iters, "iterations", f"{dt:.0f} s")


if __name__ == "__main__":
    main()
