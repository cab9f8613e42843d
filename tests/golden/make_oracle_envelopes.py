"""Writes the stored oracle envelopes of the headline-regime parity tests.

Each case of tests/_headline_cases.py is run by the oracle once per summation
order (numpy.dot, pairwise, reversed, exactly rounded, and the operator in
row-sum form; the full-size cases use the first three), exactly as the GPU
tests would run it inline, and stored as tests/golden/envelope_<case>.json:
the sha256 of the inputs, and per run the order, status, iteration / restart /
breakdown counts, true residual and the rho history.  The history is cut a few
entries after the runs' relative spread first exceeds 1e-4 (the protocol of
tests/_parity.py checks nothing beyond that point).  A GPU test uses a stored
file only when its own inputs hash to the same value; otherwise it runs the
oracle itself.  Only oracle/ and the input generators of workloads/ run here.

Usage: python tests/golden/make_oracle_envelopes.py [case ...] [--workers N]
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from tests import _oracle_pool as P  # noqa: E402
from tests._headline_cases import CASES  # noqa: E402

DECORRELATED = 1e-4
KEEP_AFTER = 5


def cut(runs):
    k = min(len(r["rho_hist"]) for r in runs)
    ref = np.asarray(runs[0]["rho_hist"][:k])
    env = np.zeros(k)
    for r in runs[1:]:
        a = np.asarray(r["rho_hist"][:k])
        with np.errstate(divide="ignore", invalid="ignore"):
            env = np.maximum(env, np.abs(a - ref) / np.abs(ref))
    env = np.maximum.accumulate(np.nan_to_num(env, nan=np.inf))
    over = np.where(env > DECORRELATED)[0]
    end = (int(over[0]) + KEEP_AFTER) if over.size else k
    for r in runs:
        r["rho_len_full"] = len(r["rho_hist"])
        r["rho_hist"] = r["rho_hist"][:end]
    return runs


def _tagged(job):
    name, j = job
    return name, P._run(j)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("cases", nargs="*")
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    args = ap.parse_args()
    names = args.cases or list(CASES)
    jobs = []
    for name in names:
        cs = CASES[name]
        for o in cs["orders"]:
            jobs.append((name, dict(problem=cs["problem"], method=cs["method"], pc=cs["pc"], prm=cs["prm"],
                                    order=o, sample=[])))
    # the longest jobs first; each case's file is written as soon as its runs are in
    jobs.sort(key=lambda j: (not CASES[j[0]]["big"], j[1]["order"] not in ("fsum", "fma", "rowsum")))
    done = {name: [] for name in names}
    with mp.get_context("spawn").Pool(args.workers) as pool:
        for name, r in pool.imap_unordered(_tagged, jobs, chunksize=1):
            done[name].append(r)
            cs = CASES[name]
            if len(done[name]) < len(cs["orders"]):
                continue
            runs = sorted(done[name], key=lambda rr: cs["orders"].index(rr["order"]))
            for rr in runs:
                rr.pop("x_sample", None)
            doc = {"case": name, "generator": "tests/golden/make_oracle_envelopes.py (oracle/ only)",
                   "problem": cs["problem"], "method": cs["method"], "pc": cs["pc"], "prm": cs["prm"],
                   "inputs_sha256": P.input_hash(P.problem(cs["problem"])), "runs": cut(runs)}
            with open(P.stored_path(name), "w") as fh:
                json.dump(doc, fh)
                fh.write("\n")
            print(name, [(rr["order"], rr["status"], rr["iterations"], rr["restarts"], len(rr["rho_hist"]))
                         for rr in runs], flush=True)


if __name__ == "__main__":
    main()
