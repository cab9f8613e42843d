"""Parity protocol for whole Krylov solves (GPU vs oracle), shared by the GPU tests.

Krylov recurrences amplify rounding: two correct FP64 implementations that
differ only in summation order drift apart by a factor of roughly 10 every few
iterations, so agreement to 1e-10 on *every* iteration of a long solve is not a
property any implementation has.  The oracle itself, re-run with a different
summation order of its inner products, shows the size of that drift.  The
protocol is therefore:

1. Envelope: the oracle is re-run with three other summation orders of every
   inner product (pairwise, reversed, exactly rounded via math.fsum), once
   with every vector update y + a v evaluated as a fused multiply-add (the
   product kept exact, one rounding: how the GPU kernels evaluate their AXPYs
   and MAXPYs, and what sets the gap between the recurred and the true
   residual, hence when a residual replacement fires) and, for a stencil
   operator, once more with the operator applied in row-sum form (its
   assembled CSR: d_i u_i - sum K u_nbr, the form the GPU evaluates) instead
   of the flux form sum K (u_i - u_nbr); env_i is the running maximum over
   those runs of |rho_alt - rho| / rho at entry i.
2. Strict prefix: on every entry where env_i <= 1e-11 the GPU must agree with
   the oracle to 1e-10 relative.
3. Envelope region: while env_i <= 1e-4 (the trajectories are still
   correlated) the GPU must stay within max(1e-10, 100 env_i).
4. Convergence level: same status; the GPU's iteration count within
   2 * (largest alt-vs-oracle spread) + 5 % + 2 of the oracle's; true residual
   within the tolerance.

A wrong scalar, sign, window index or dropped term shows up as a departure of
1e-6 or more within a few iterations, where the envelope is still ~1e-14.
"""
from __future__ import annotations

import math

import numpy as np

from oracle import krylov as K
from oracle import preconditioners as PC

STRICT = 1e-10
PREFIX_ENV = 1e-11
DECORRELATED = 1e-4
FACTOR = 100.0


def _alt_dots():
    def pairwise(a, b):
        return float(np.sum(np.asarray(a, dtype=np.float64) * np.asarray(b, dtype=np.float64)))

    def reversed_(a, b):
        a = np.asarray(a, dtype=np.float64)
        b = np.asarray(b, dtype=np.float64)
        return float(np.dot(a[::-1], b[::-1]))

    def exact(a, b):
        return float(math.fsum(np.asarray(a, dtype=np.float64) * np.asarray(b, dtype=np.float64)))

    return [pairwise, reversed_, exact]


_SPLIT = 134217729.0   # 2^27 + 1: Dekker's splitting constant for float64


def fma_axpy(y, a, v):
    """y + a v with the product kept exact before the addition (Dekker's
    TwoProduct and Knuth's TwoSum, then one final rounding): the fused
    multiply-add evaluation of an update, up to a rare double rounding.  Float32
    arrays keep the plain evaluation."""
    y = np.asarray(y)
    v = np.asarray(v)
    if y.dtype != np.float64 or v.dtype != np.float64:
        return y + a * v
    a = np.float64(a)
    p = a * v
    c = _SPLIT * a
    ah = c - (c - a)
    al = a - ah
    c = _SPLIT * v
    vh = c - (c - v)
    vl = v - vh
    e = ((ah * vh - p) + ah * vl + al * vh) + al * vl
    s_ = p + y
    bb = s_ - p
    t = (p - (s_ - bb)) + (y - bb)
    return s_ + (t + e)


def oracle_with_envelope(method, A, make_B, b, prm, x0=None):
    """(reference result, [alternative results]): three other summation orders
    of every inner product, every vector update evaluated as a fused
    multiply-add (as the GPU kernels evaluate theirs), and, for a stencil, the
    operator in row-sum form."""
    ref = K.solve(method, A, make_B(), b, x0=x0, prm=prm)
    alts = []
    saved = (K.dot, PC._dot, K.axpy, PC._axpy)
    try:
        for f in _alt_dots():
            K.dot = f
            PC._dot = f
            alts.append(K.solve(method, A, make_B(), b, x0=x0, prm=prm))
        K.dot, PC._dot = saved[0], saved[1]
        K.axpy = fma_axpy
        PC._axpy = fma_axpy
        alts.append(K.solve(method, A, make_B(), b, x0=x0, prm=prm))
    finally:
        K.dot, PC._dot, K.axpy, PC._axpy = saved
    if hasattr(A, "to_csr"):
        alts.append(K.solve(method, A.to_csr(), make_B(), b, x0=x0, prm=prm))
    return ref, alts


def envelope(ref, alts) -> np.ndarray:
    r = ref.rho()
    env = np.zeros(len(r))
    for a in alts:
        ra = a.rho()
        k = min(len(ra), len(r))
        d = np.full(len(r), np.inf)
        d[:k] = np.abs(ra[:k] - r[:k]) / np.abs(r[:k])
        env = np.maximum(env, d)
    return np.maximum.accumulate(env)


def check_solve(hist, info, ref, alts, rtol=None, min_prefix=3, check_status=True, check_restarts=False):
    """Applies the protocol; returns a summary dict (asserts on failure).

    check_restarts: also require the GPU's restart count within
    2 * (largest alt-vs-oracle restart spread) + 2 of the oracle's (same
    condition as the iteration band: the alternative runs agree on the status).
    """
    r = ref.rho()
    env = envelope(ref, alts)
    g = hist[:, 0]
    k = min(len(g), len(r))
    prefix = int(np.sum(env[:k] <= PREFIX_ENV))
    assert prefix >= min(min_prefix, k), f"envelope already above {PREFIX_ENV} at entry {prefix}"
    d = np.abs(g[:k] - r[:k]) / np.abs(r[:k])
    assert np.all(d[:prefix] <= STRICT), (int(np.argmax(d[:prefix])), float(d[:prefix].max()))
    corr = env[:k] <= DECORRELATED
    bound = np.maximum(STRICT, FACTOR * env[:k])
    bad = np.where(corr & (d > bound))[0]
    assert bad.size == 0, (int(bad[0]), float(d[bad[0]]), float(env[bad[0]]))
    # convergence level: only where the oracle's own alternative-order runs agree
    # on the outcome (a stagnating method, e.g. Alg. 7 with a nonlinear
    # preconditioner, can end either way depending on rounding alone)
    spread = max(abs(a.iterations - ref.iterations) for a in alts)
    if check_status and all(a.status == ref.status for a in alts):
        status = {"converged": 0, "maxit": -5, "stagnated": -5, "breakdown": -4}[ref.status]
        assert info["status"] == status, (info["status"], ref.status)
        band = 2 * spread + 0.05 * ref.iterations + 2
        assert abs(info["iterations"] - ref.iterations) <= band, (info["iterations"], ref.iterations, band)
        if check_restarts:
            rspread = max(abs(a.restarts - ref.restarts) for a in alts)
            assert abs(info["restarts"] - ref.restarts) <= 2 * rspread + 2, (info["restarts"], ref.restarts, rspread)
    if rtol is not None and ref.status == "converged" and (check_status or info["status"] == 0):
        assert info["rnorm_true"] <= rtol * info["bnorm"] * (1 + 1e-12)
    return dict(prefix=prefix, correlated=int(corr.sum()), max_strict=float(d[:prefix].max()) if prefix else 0.0,
                iterations=(info["iterations"], ref.iterations, spread),
                restarts=(info.get("restarts"), getattr(ref, "restarts", None)))
