"""Oracle runs in worker processes, for the GPU tests' expensive envelopes.

The envelope of a whole-solve parity check needs the oracle several times over
(its own summation order and the alternative ones, see tests/_parity.py); at
the headline sizes each run takes seconds to minutes.  The runs are independent,
so they go to a pool of worker processes started with "spawn" (never forked
from a process that has touched the GPU).  A job names its problem by the
workload generator and its arguments, so each worker builds the same inputs
itself; the result carries what the parity protocol reads (rho history,
status, iteration and restart counts) and a few sampled iterate entries.
"""
from __future__ import annotations

import math
import multiprocessing as mp
import os
import sys
from concurrent.futures import ProcessPoolExecutor

# one BLAS thread per worker process (set before numpy loads its BLAS)
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_pools = {}


def _avail_gb() -> float:
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 2 ** 20
    except OSError:
        pass
    return 16.0


def pool(kind: str = "small") -> ProcessPoolExecutor:
    """Worker pools: "small" jobs (a few hundred MB each) get up to one worker
    per spare core; "big" jobs (full-size problems, several GB each) get as
    many workers as about a quarter of the available host memory allows at
    ~8 GB per job."""
    if kind not in _pools:
        cores = max(1, (os.cpu_count() or 2) - 1)
        n = cores if kind == "small" else max(1, min(cores, 6, int(_avail_gb() / 4 / 8)))
        _pools[kind] = ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn"))
    return _pools[kind]


class Lite:
    """The part of an oracle Result the parity protocol reads."""

    def __init__(self, d: dict):
        self.__dict__.update(d)

    def rho(self) -> np.ndarray:
        return np.asarray(self.rho_hist)


def _dot(order: str):
    if order == "pairwise":
        return lambda a, b: float(np.sum(np.asarray(a, dtype=np.float64) * np.asarray(b, dtype=np.float64)))
    if order == "reversed":
        return lambda a, b: float(np.dot(np.asarray(a, dtype=np.float64)[::-1], np.asarray(b, dtype=np.float64)[::-1]))
    if order == "fsum":
        return lambda a, b: float(math.fsum(np.asarray(a, dtype=np.float64) * np.asarray(b, dtype=np.float64)))
    return None


def problem(spec: dict) -> dict:
    sys.path.insert(0, ROOT)
    import workloads as W
    return getattr(W, spec["gen"])(**spec.get("kw", {}))


def input_hash(c: dict) -> str:
    """sha256 of a problem's inputs (dims, eta, velocity, b), to tell whether a
    stored oracle run was made from bitwise the same inputs."""
    import hashlib
    h = hashlib.sha256()
    h.update(np.asarray(c["dims"], dtype=np.int64).tobytes())
    h.update(np.ascontiguousarray(c["eta"], dtype=np.float64).tobytes())
    h.update(np.asarray(c.get("vel", (0.0, 0.0, 0.0)), dtype=np.float64).tobytes())
    h.update(np.ascontiguousarray(c["b"], dtype=np.float64).tobytes())
    return h.hexdigest()


def _run(job: dict) -> dict:
    sys.path.insert(0, ROOT)
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    from oracle import krylov as K
    from oracle import operators as O
    from oracle import preconditioners as PC
    c = problem(job["problem"])
    A = O.StencilOperator(c["dims"], c["eta"], c.get("vel", (0.0, 0.0, 0.0)))
    f = _dot(job["order"])
    if f is not None:
        K.dot = f
        PC._dot = f
    if job["order"] == "fma":
        from tests._parity import fma_axpy
        K.axpy = fma_axpy
        PC._axpy = fma_axpy
    kind, args = job["pc"]
    lo, hi = PC.chebyshev_bounds(A) if kind == "chebyshev" else (None, None)
    if job["order"] == "rowsum":
        A = A.to_csr()
    if kind == "inner_pcg":
        B = PC.InnerPCG(A, args.get("k", 4), precision=args.get("precision", "fp64"))
    elif kind == "chebyshev":
        B = PC.Chebyshev(A, args.get("k", 8), lo, hi, precision=args.get("precision", "fp64"))
    else:
        B = PC.JacobiPC(A)
    res = K.solve(job["method"], A, B, c["b"], prm=K.Params(**job["prm"]))
    idx = np.asarray(job.get("sample", []), dtype=np.int64)
    return {"order": job["order"], "rho_hist": [float(h["rho"]) for h in res.history], "status": res.status,
            "iterations": int(res.iterations), "restarts": int(res.restarts), "breakdowns": int(res.breakdowns),
            "rnorm_true": float(res.rnorm_true), "bnorm": float(res.bnorm),
            "x_sample": res.x[idx].tolist() if idx.size else [],
            "x_norm": float(np.linalg.norm(res.x))}


def envelope_runs(problem_spec: dict, method: str, pc: tuple, prm: dict, orders=("numpy", "pairwise", "reversed"),
                  sample=(), big: bool = False, stored: str | None = None):
    """One oracle run per summation order; returns a function that waits and
    gives (reference, [alternatives]) as Lite results (the first order is the
    reference).  big: full-size problem (memory-bounded pool).  stored: name of
    a tests/golden/envelope_<name>.json written by
    tests/golden/make_oracle_envelopes.py for the same job; it is used when its
    input hash equals this machine's inputs (bitwise), otherwise the runs are
    submitted to the pool."""
    if stored is not None:
        doc = load_stored(stored)
        if doc is not None and doc["inputs_sha256"] == input_hash(problem(problem_spec)):
            runs = [Lite(r) for r in doc["runs"]]
            return lambda: (runs[0], runs[1:])
    jobs = [dict(problem=problem_spec, method=method, pc=pc, prm=prm, order=o, sample=list(sample)) for o in orders]
    futs = [pool("big" if big else "small").submit(_run, j) for j in jobs]

    def wait():
        res = [Lite(f.result()) for f in futs]
        return res[0], res[1:]
    return wait


GOLDEN = os.path.join(ROOT, "tests", "golden")


def stored_path(name: str) -> str:
    return os.path.join(GOLDEN, f"envelope_{name}.json")


def load_stored(name: str):
    import json
    try:
        with open(stored_path(name)) as fh:
            return json.load(fh)
    except OSError:
        return None
