"""Writes the oracle's own rounding spread of whole solves in the headline regime.

The headline workload (3D variable-coefficient Poisson, eta = 10^(3 g) with g a
smoothed Gaussian field, contrast 1e6, preconditioner = 4 inner Jacobi-PCG
iterations, PIPEFCG / PIPEGCR with nu_max = 30, rtol 1e-8 with residual
replacement) reaches 1e-8 only through repeated replacement restarts: the
pipelined recurrences drift from B(r) under this nonlinear preconditioner, the
true residual stalls, and the restarts fire at points that depend on rounding.
So the iteration count of one correct FP64 implementation is not a sharp
number.  This script measures how far it moves when nothing but the summation
order of the inner products (and, for the "rowsum" order, the operator's
evaluation form) changes, running only the oracle: each order is one full
solve to convergence.

Output: one JSON file per (size, method), a list of runs with the order name,
status, iterations, restarts, breakdowns, true relative residual and CPU time.
The GPU tests read the files to check that the GPU's iteration count lies in
the oracle's own range.  Orders:

  numpy     the oracle as it stands (numpy.dot),
  pairwise  numpy.sum of the products (pairwise summation),
  reversed  numpy.dot over the reversed vectors,
  fsum      exactly rounded sums (math.fsum) -- slow, small sizes only,
  fma       every vector update y + a v evaluated as a fused multiply-add,
  rowsum    the operator as its assembled CSR (d_i u_i - sum K u_nbr).

Usage: python tests/golden/make_oracle_spread.py --n 64 --ell 4 --methods pipefcg,pipegcr
       [--orders numpy,pairwise,reversed,fsum,rowsum] [--workers 5]
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))

ALL_ORDERS = ("numpy", "pairwise", "reversed", "fsum", "fma", "rowsum")


def spread_path(n: int, method: str) -> str:
    return os.path.join(HERE, f"oracle_spread_{method}_{n}cube.json")


def _dot_of(order: str):
    import numpy as np
    if order == "pairwise":
        return lambda a, b: float(np.sum(np.asarray(a, dtype=np.float64) * np.asarray(b, dtype=np.float64)))
    if order == "reversed":
        return lambda a, b: float(np.dot(np.asarray(a, dtype=np.float64)[::-1], np.asarray(b, dtype=np.float64)[::-1]))
    if order == "fsum":
        return lambda a, b: float(math.fsum(np.asarray(a, dtype=np.float64) * np.asarray(b, dtype=np.float64)))
    return None


def one_run(job: dict) -> dict:
    sys.path.insert(0, ROOT)
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    import workloads as W
    from oracle import krylov as K
    from oracle import operators as O
    from oracle import preconditioners as PC
    c = W.poisson3d_gaussian(n=job["n"], ell=job["ell"], log_contrast=job["log_contrast"])
    A = O.StencilOperator(c["dims"], c["eta"])
    f = _dot_of(job["order"])
    if f is not None:
        K.dot = f
        PC._dot = f
    if job["order"] == "fma":
        from tests._parity import fma_axpy
        K.axpy = fma_axpy
        PC._axpy = fma_axpy
    op = A.to_csr() if job["order"] == "rowsum" else A
    prm = K.Params(mmax=30, rtol=1e-8, maxit=job["maxit"], max_restarts=job["max_restarts"])
    t0 = time.perf_counter()
    res = K.solve(job["method"], op, PC.InnerPCG(op, 4), c["b"], prm=prm)
    return {"order": job["order"], "status": res.status, "iterations": int(res.iterations),
            "restarts": int(res.restarts), "breakdowns": int(res.breakdowns),
            "replacements": int(res.replacements),
            "true_rel_residual": float(res.rnorm_true / res.bnorm), "cpu_s": time.perf_counter() - t0}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, required=True)
    ap.add_argument("--ell", type=float, required=True)
    ap.add_argument("--log-contrast", type=float, default=3.0)
    ap.add_argument("--methods", default="pipefcg")
    ap.add_argument("--orders", default=",".join(ALL_ORDERS))
    ap.add_argument("--maxit", type=int, default=20000)
    ap.add_argument("--max-restarts", type=int, default=200)
    ap.add_argument("--workers", type=int, default=5)
    args = ap.parse_args()
    jobs = [dict(n=args.n, ell=args.ell, log_contrast=args.log_contrast, method=m, order=o, maxit=args.maxit,
                 max_restarts=args.max_restarts)
            for m in args.methods.split(",") for o in args.orders.split(",")]
    with mp.get_context("spawn").Pool(args.workers) as pool:
        runs = pool.map(one_run, jobs, chunksize=1)
    for m in args.methods.split(","):
        mine = [r for j, r in zip(jobs, runs) if j["method"] == m]
        its = [r["iterations"] for r in mine if r["status"] == "converged"]
        doc = {"workload": f"3D {args.n}^3 Poisson, eta = 10^({args.log_contrast:g} g), Gaussian field "
                           f"ell = {args.ell:g} cells, 4 inner Jacobi-PCG (FP64), {m} nu_max = 30, rtol 1e-8, "
                           f"at most {args.max_restarts} residual-replacement restarts",
               "n": args.n, "ell": args.ell, "log_contrast": args.log_contrast, "method": m,
               "max_restarts": args.max_restarts, "maxit": args.maxit,
               "generator": "tests/golden/make_oracle_spread.py (oracle/ only)",
               "runs": mine,
               "converged_iterations": {"min": min(its), "max": max(its)} if its else None}
        with open(spread_path(args.n, m), "w") as fh:
            json.dump(doc, fh, indent=1)
            fh.write("\n")
        print(json.dumps({"method": m, "runs": [(r["order"], r["status"], r["iterations"], r["restarts"])
                                                 for r in mine]}))


if __name__ == "__main__":
    main()
