"""Writes the oracle's own rounding spread of whole solves in the headline regime.

The headline workload (3D variable-coefficient Poisson, eta = 10^(3 g) with g a
smoothed Gaussian field, contrast 1e6, preconditioner = 4 inner Jacobi-PCG
iterations, PIPEFCG / PIPEGCR with nu_max = 30, rtol 1e-8 with residual
replacement) reaches 1e-8 only through repeated replacement restarts: the
pipelined recurrences drift from B(r) under this nonlinear preconditioner, the
true residual stalls, and the restarts fire at points that depend on rounding.
So the iteration count of one correct FP64 implementation is not a sharp
number.  This script measures how far it moves when only the rounding of the
same statements changes, running only the oracle (through the job runner of
tests/_oracle_pool.py, the same one the GPU tests use): each order is one full
solve to convergence.

Orders:
  numpy     the oracle as it stands (numpy.dot),
  pairwise  numpy.sum of the products (pairwise summation),
  reversed  numpy.dot over the reversed vectors,
  fsum      exactly rounded inner products (math.fsum) -- slow, small sizes,
  fma       every vector update y + a v evaluated as a fused multiply-add,
  rowsum    the operator as its assembled CSR (d_i u_i - sum K u_nbr).

Output: tests/golden/oracle_spread_<method>_<n>cube.json with the sha256 of
the inputs and per run the order, status, iteration / restart / breakdown
counts and the true relative residual.  tests/test_gpu_headline.py checks the
GPU's iteration count against the range when its inputs hash the same.

Usage: python tests/golden/make_oracle_spread.py --n 64 --methods pipefcg
       [--orders numpy,pairwise,reversed,fsum,fma,rowsum] [--workers 6] [--suffix _x]
(the correlation length is scaled with the grid: ell = 8 n / 128 cells)
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from tests import _oracle_pool as P  # noqa: E402
from tests._headline_cases import field  # noqa: E402

ALL_ORDERS = ("numpy", "pairwise", "reversed", "fsum", "fma", "rowsum")


def spread_path(n: int, method: str) -> str:
    return os.path.join(HERE, f"oracle_spread_{method}_{n}cube.json")


def timed_run(job: dict) -> dict:
    t0 = time.perf_counter()
    r = P._run(job)
    r.pop("rho_hist", None)
    r.pop("x_sample", None)
    r["cpu_s"] = time.perf_counter() - t0
    r["true_rel_residual"] = r["rnorm_true"] / r["bnorm"]
    return r


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, required=True)
    ap.add_argument("--methods", default="pipefcg")
    ap.add_argument("--orders", default=",".join(ALL_ORDERS))
    ap.add_argument("--maxit", type=int, default=20000)
    ap.add_argument("--max-restarts", type=int, default=200)
    ap.add_argument("--workers", type=int, default=6)
    ap.add_argument("--suffix", default="", help="appended to the output file name")
    args = ap.parse_args()
    spec = field(args.n)
    prm = dict(mmax=30, rtol=1e-8, maxit=args.maxit, max_restarts=args.max_restarts)
    jobs = [dict(problem=spec, method=m, pc=("inner_pcg", {"k": 4}), prm=prm, order=o, sample=[])
            for m in args.methods.split(",") for o in args.orders.split(",")]
    with mp.get_context("spawn").Pool(args.workers) as pool:
        runs = pool.map(timed_run, jobs, chunksize=1)
    h = P.input_hash(P.problem(spec))
    for m in args.methods.split(","):
        mine = [r for j, r in zip(jobs, runs) if j["method"] == m]
        its = [r["iterations"] for r in mine if r["status"] == "converged"]
        doc = {"workload": f"3D {args.n}^3 Poisson, eta = 10^(3 g), field ell = {spec['kw']['ell']:g} cells, "
                           f"4 inner Jacobi-PCG (FP64), {m} nu_max = 30, rtol 1e-8, at most "
                           f"{args.max_restarts} residual-replacement restarts",
               "problem": spec, "method": m, "prm": prm, "inputs_sha256": h,
               "generator": "tests/golden/make_oracle_spread.py (oracle/ only)",
               "runs": mine,
               "converged_iterations": {"min": min(its), "max": max(its)} if its else None}
        with open(spread_path(args.n, m)[:-5] + args.suffix + ".json", "w") as fh:
            json.dump(doc, fh, indent=1)
            fh.write("\n")
        print(json.dumps({"method": m, "runs": [(r["order"], r["status"], r["iterations"], r["restarts"])
                                                 for r in mine]}), flush=True)


if __name__ == "__main__":
    main()
