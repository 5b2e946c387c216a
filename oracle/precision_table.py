"""Error of reduced-precision contraction operands against FP64 (oracle only).

The shared-matrix products of the iteration -- the evaluations P c, Pdot c,
Pddot c and the transposed products with F -- are what tensor cores would
run.  This script solves seeded scenes with the FP64 oracle twice: exact,
and with those operands rounded to bfloat16 (8 significant bits) or TF32
(11), alone or as a hi + lo pair, or to float32 (24), the KKT inverses and
all arithmetic staying FP64; it prints the position error of each against
the exact solve after 100 iterations.  The oracle takes the direct form of
the QP step (rho F^T g + lambda through K11), so the rounding of F multiplies
the large F^T g: the table measures the dtype in that form.  The GPU kernel
contracts residuals (the increment form), where the same rounding multiplies
small quantities; its own error table comes from the kernel's precision
modes, measured against this oracle by the GPU tests.

    python oracle/precision_table.py [--sample 16]

TEST INFRASTRUCTURE: it runs the oracle only.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
from paper_2109_10392_gb300 import scenes  # noqa: E402

DTYPES = [("bf16", 8, 0), ("bf16 hi+lo", 8, 1), ("tf32", 11, 0), ("tf32 hi+lo", 11, 1), ("fp32", 24, 0)]


def positions(p, coef):
    x, y, _ = oracle.positions(p, coef)
    return x, y


def table(sample: int = 16, threads: int | None = None):
    threads = threads or (os.cpu_count() or 1)
    f = lambda a: np.asarray(a, np.float32).astype(np.float64)  # noqa: E731
    rows = []
    for name, sc, stride in [("N=200 n=16 m=30", scenes.scene_custom(31, 16384, 30, N=200, n=16), 16384 // sample),
                             ("N=100 n=12 m=50", scenes.scene_large(0), 1024 // sample)]:
        kw = dict(sc.params)
        kw.update(tol=0.0, iters=100)
        idx = np.arange(0, len(sc.goals), stride)
        exact = oracle.solve(oracle.params(**kw), f(sc.ego), f(sc.obst), f(sc.goals)[idx], nthreads=threads)
        xe, ye = positions(oracle.params(**kw), exact["coef"])
        for dname, bits, split in DTYPES:
            pk = oracle.params(**kw, basis_bits=bits, basis_split=split)
            r = oracle.solve(pk, f(sc.ego), f(sc.obst), f(sc.goals)[idx], nthreads=threads)
            x, y = positions(oracle.params(**kw), r["coef"])
            err = np.max(np.hypot(x - xe, y - ye), axis=1)
            rows.append((name, dname, float(np.median(err)), float(err.max()), float(np.mean(err <= 1e-3))))
    return rows


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--sample", type=int, default=16)
    a = ap.parse_args()
    print("| workload | operands | median error [m] | max error [m] | share <= 1e-3 m |")
    print("|---|---|---|---|---|")
    for r in table(a.sample):
        print(f"| {r[0]} | {r[1]} | {r[2]:.1e} | {r[3]:.1e} | {r[4]:.2f} |")
