"""The paper's Krylov methods, step by step, in plain NumPy float64.

Every function takes the operator ``A`` (callable v -> A v), the preconditioner
``B`` (callable, possibly nonlinear), ``b``, ``x0`` and a ``Params`` record, and
returns a ``Result`` with the iterate, the status and a per-iteration history.
The loop bodies follow the listings' statement order and notation; the comments
name the quantities, not listing lines.

Readings taken where the paper is ambiguous or garbled (each listed in the
design notes with its reason):

* Alg. 8 initialisation uses m_0 = B(w_0) as printed (equal to
  u_0 + B(w_0 - r_0) for a linear B); its "u_0" in the first dot products is
  the tilde-u_0 computed just before.
* Truncation: standard nu_i = min(i, nu_max) (default, as in Sec. 6);
  restart-style nu_i = ((i - 1) mod nu_max) + 1, i counted since the last
  (re)start, which gives one direction right after a restart.
* Alg. 9 (GCR) uses gamma_i = <r_i, s_i> (Eisenstat's minimal-residual step);
  ``gcr_literal_gamma`` keeps the printed <u_i, s_i>.
* Alg. 11/12: p_0 = tilde-u_0; gamma_0 = <r_0, s_0> (``gcr_literal_init``
  keeps the printed <r_0, A r_0>); eta_0 = <s_0, s_0> (squared, consistent
  with delta_i = <w_i, w_i>); one vector tilde-u throughout.  Alg. 12 needs
  w_0, which it never defines: w_0 = A tilde-u_0 = s_0.
* Alg. 15: h_{j,i-1} = hbar_{j,i-1} for j < i-1; the initial wbar_0 = A qbar_0;
  u_0 = B(p_0) is the first column of tilde-U; constant shift sigma, so the
  zbar update takes the simplified form of eq. (pipefgmresz).
* Convergence: the natural norm sqrt|gamma_i| (CG- and CR-type) or the
  recurred ||r_i||_2 (``norm='unpreconditioned'``), relative to its value at
  the first fill; for the GMRES family the least-squares residual estimate.
  At convergence the true residual ||b - A x||_2 must be <= rtol ||b||_2,
  otherwise the solver restarts from x with its target tightened by
  0.5 rtol ||b|| / ||b - A x|| (residual replacement).  When the true
  residual still misses the goal after ``max_restarts`` restarts the solve
  ends with status "stagnated" (x is the last iterate).
* Norm breakdown (eta_i <= 0, or t < 0 for the GMRES family) restarts the
  method from the current x, flushing the pipeline (Sec. 5).  A breakdown in a
  fill, or in the first iteration after a breakdown restart, or more than
  ``max_restarts`` restarts, ends the solve with status "breakdown".
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Params:
    mmax: int = 30               # nu_max for FCG/GCR types, restart length m for FGMRES types
    truncation: str = "standard"  # "standard" | "restart"
    rtol: float = 1e-8
    atol: float = 0.0
    maxit: int = 10000
    norm: str = "natural"        # "natural" | "unpreconditioned"
    sigma: float = 0.0           # constant shift of CGFGMRES / PIPEFGMRES
    max_restarts: int = 20
    true_residual_check: bool = True
    gcr_literal_init: bool = False
    gcr_literal_gamma: bool = False
    trace: bool = False          # keep copies of the iteration vectors (tests only)


@dataclass
class Result:
    x: np.ndarray
    status: str = "running"      # converged | maxit | breakdown | stagnated
    iterations: int = 0
    restarts: int = 0
    breakdowns: int = 0
    replacements: int = 0
    cycles: int = 0              # GMRES-type restart cycles (not counted in restarts)
    sigma: float = float("nan")  # shift used by CGFGMRES / PIPEFGMRES
    rho0: float = float("nan")
    rnorm_true: float = float("nan")
    bnorm: float = float("nan")
    stagnated: bool = False
    history: list = field(default_factory=list)
    trace: list = field(default_factory=list)

    def rho(self) -> np.ndarray:
        return np.array([h["rho"] for h in self.history])


def dot(a, b) -> float:
    return float(np.dot(a, b))


def nu_window(i: int, prm: Params) -> int:
    if prm.truncation == "standard":
        return min(i, prm.mmax)
    if prm.truncation == "restart":
        return ((i - 1) % prm.mmax) + 1
    raise ValueError(prm.truncation)


class _Monitor:
    """Convergence bookkeeping shared by all methods (not part of any listing)."""

    def __init__(self, A, b, prm: Params, res: Result):
        self.A, self.b, self.prm, self.res = A, b, prm, res
        res.bnorm = float(np.linalg.norm(b))
        self.target = None

    def rho(self, gamma: float, r: np.ndarray) -> float:
        if self.prm.norm == "natural":
            return float(np.sqrt(abs(gamma)))
        return float(np.sqrt(dot(r, r)))

    def record(self, rho: float, **scalars) -> bool:
        if self.target is None:
            self.res.rho0 = rho
            self.target = max(self.prm.rtol * rho, self.prm.atol)
        entry = dict(it=self.res.iterations, rho=rho)
        entry.update(scalars)
        self.res.history.append(entry)
        return rho <= self.target

    def accept(self, x: np.ndarray) -> bool:
        """True-residual test at convergence; tightens the target when it fails."""
        rt = float(np.linalg.norm(self.b - self.A(x)))
        self.res.rnorm_true = rt
        if not self.prm.true_residual_check:
            return True
        goal = max(self.prm.rtol * self.res.bnorm, self.prm.atol)
        if rt <= goal:
            return True
        if self.res.restarts >= self.prm.max_restarts:
            self.res.stagnated = True
            return True
        self.res.replacements += 1
        self.res.restarts += 1
        self.target *= 0.5 * goal / rt
        return False

    def finish(self, x, status):
        self.res.x = x
        if status == "converged" and self.res.stagnated:
            status = "stagnated"
        self.res.status = status
        if np.isnan(self.res.rnorm_true) or status != "converged":
            self.res.rnorm_true = float(np.linalg.norm(self.b - self.A(x)))
        return self.res

    def breakdown(self, i_since_restart: int, after_breakdown: bool) -> bool:
        """Count a norm breakdown; True if the solve must stop."""
        self.res.breakdowns += 1
        if i_since_restart <= 1 and after_breakdown:
            return True
        if self.res.restarts >= self.prm.max_restarts:
            return True
        self.res.restarts += 1
        return False


def axpy(y: np.ndarray, a: float, v: np.ndarray) -> np.ndarray:
    """y + a v (every vector update of the methods goes through here)."""
    return y + a * v


def _maxpy(base: np.ndarray, beta: dict, hist: dict) -> np.ndarray:
    """base + sum_k beta_k hist_k, k ascending."""
    out = base.copy()
    for k in sorted(beta):
        out = axpy(out, beta[k], hist[k])
    return out


# ---------------------------------------------------------------------------
# Conjugate-gradient family (Sec. 3)
# ---------------------------------------------------------------------------

def pcg(A, M, b, x0, prm: Params) -> Result:
    """Preconditioned CG, Alg. 3 (M linear)."""
    res = Result(x=x0.copy())
    mon = _Monitor(A, b, prm, res)
    x = np.array(x0, dtype=np.float64)
    after_bd = False
    while True:
        r = b - A(x)
        u = M(r)
        p = u.copy()
        s = A(p)
        gamma = dot(u, r)
        eta = dot(s, p)
        conv = mon.record(mon.rho(gamma, r), gamma=gamma, eta=eta)
        if conv:
            if mon.accept(x):
                return mon.finish(x, "converged")
            continue
        if eta <= 0.0:
            return mon.finish(x, "breakdown")
        alpha = gamma / eta
        i = 0
        restart = False
        while True:
            if res.iterations >= prm.maxit:
                return mon.finish(x, "maxit")
            i += 1
            x = axpy(x, alpha, p)
            r = axpy(r, -alpha, s)
            res.iterations += 1
            u = M(r)
            gamma_new = dot(u, r)
            conv = mon.record(mon.rho(gamma_new, r), gamma=gamma_new)
            if conv:
                if mon.accept(x):
                    return mon.finish(x, "converged")
                restart = True
                after_bd = False
                break
            beta = gamma_new / gamma
            gamma = gamma_new
            p = axpy(u, beta, p)
            s = A(p)
            eta = dot(s, p)
            res.history[-1].update(eta=eta, beta=beta)
            if eta <= 0.0:
                if mon.breakdown(i, after_bd):
                    return mon.finish(x, "breakdown")
                after_bd = True
                restart = True
                break
            after_bd = False
            alpha = gamma / eta
        if restart:
            continue


def fcg(A, B, b, x0, prm: Params) -> Result:
    """Flexible CG with truncated Gram-Schmidt, Alg. 2 (Notay)."""
    res = Result(x=x0.copy())
    mon = _Monitor(A, b, prm, res)
    x = np.array(x0, dtype=np.float64)
    after_bd = False
    while True:
        r = b - A(x)
        u = B(r)
        P = {0: u.copy()}
        S = {0: A(P[0])}
        gamma = dot(u, r)
        eta = {0: dot(P[0], S[0])}
        conv = mon.record(mon.rho(gamma, r), gamma=gamma, eta=eta[0])
        if conv:
            if mon.accept(x):
                return mon.finish(x, "converged")
            continue
        if eta[0] <= 0.0:
            return mon.finish(x, "breakdown")
        alpha = gamma / eta[0]
        i = 0
        while True:
            if res.iterations >= prm.maxit:
                return mon.finish(x, "maxit")
            i += 1
            x = axpy(x, alpha, P[i - 1])
            r = axpy(r, -alpha, S[i - 1])
            res.iterations += 1
            u = B(r)
            gamma = dot(u, r)
            conv = mon.record(mon.rho(gamma, r), gamma=gamma)
            if conv:
                if mon.accept(x):
                    return mon.finish(x, "converged")
                after_bd = False
                break
            nu = nu_window(i, prm)
            beta = {k: -dot(u, S[k]) / eta[k] for k in range(i - nu, i)}
            P[i] = _maxpy(u, beta, P)
            S[i] = A(P[i])
            eta[i] = dot(P[i], S[i])
            res.history[-1].update(eta=eta[i], nu=nu)
            if prm.trace:
                res.trace.append(dict(i=i, x=x.copy(), r=r.copy(), u=u.copy(), p=P[i].copy(),
                                      s=S[i].copy(), eta=eta[i], window=dict(P), beta=beta))
            for k in [k for k in P if k < i - prm.mmax]:
                del P[k], S[k], eta[k]
            if eta[i] <= 0.0:
                if mon.breakdown(i, after_bd):
                    return mon.finish(x, "breakdown")
                after_bd = True
                break
            after_bd = False
            alpha = gamma / eta[i]


def cgfcg(A, B, b, x0, prm: Params) -> Result:
    """Single-reduction FCG, Alg. 6 (w_0 = A u_0 since p_0 = u_0)."""
    res = Result(x=x0.copy())
    mon = _Monitor(A, b, prm, res)
    x = np.array(x0, dtype=np.float64)
    after_bd = False
    while True:
        r = b - A(x)
        u = B(r)
        w = A(u)
        gamma = dot(u, r)
        delta = dot(u, w)
        P = {0: u.copy()}
        S = {0: w.copy()}
        eta = {0: delta}
        conv = mon.record(mon.rho(gamma, r), gamma=gamma, delta=delta, eta=delta)
        if conv:
            if mon.accept(x):
                return mon.finish(x, "converged")
            continue
        if eta[0] <= 0.0:
            return mon.finish(x, "breakdown")
        alpha = gamma / eta[0]
        i = 0
        while True:
            if res.iterations >= prm.maxit:
                return mon.finish(x, "maxit")
            i += 1
            x = axpy(x, alpha, P[i - 1])
            r = axpy(r, -alpha, S[i - 1])
            res.iterations += 1
            u = B(r)
            w = A(u)
            gamma = dot(u, r)
            nu = nu_window(i, prm)
            beta = {k: -dot(u, S[k]) / eta[k] for k in range(i - nu, i)}
            delta = dot(u, w)
            conv = mon.record(mon.rho(gamma, r), gamma=gamma, delta=delta)
            if conv:
                if mon.accept(x):
                    return mon.finish(x, "converged")
                after_bd = False
                break
            P[i] = _maxpy(u, beta, P)
            S[i] = _maxpy(w, beta, S)
            eta[i] = delta - sum(beta[k] ** 2 * eta[k] for k in sorted(beta))
            res.history[-1].update(eta=eta[i], nu=nu)
            if prm.trace:
                res.trace.append(dict(i=i, x=x.copy(), r=r.copy(), u=u.copy(), w=w.copy(),
                                      p=P[i].copy(), s=S[i].copy(), eta=eta[i], window=dict(P)))
            for k in [k for k in P if k < i - prm.mmax]:
                del P[k], S[k], eta[k]
            if eta[i] <= 0.0:
                if mon.breakdown(i, after_bd):
                    return mon.finish(x, "breakdown")
                after_bd = True
                break
            after_bd = False
            alpha = gamma / eta[i]


def pipefcg(A, B, b, x0, prm: Params, naive: bool = False, theta: bool = False) -> Result:
    """Pipelined FCG, Alg. 8; ``naive=True`` gives Alg. 7 (m_i = B(w_i)).

    The only difference between the two is the pipelined preconditioner input:
    Alg. 8 applies B to w_i - r_i and adds tilde-u_i back (eq. BwMinusR).
    ``theta=True`` is the projection repair of eq. (proj) in Alg. 8's
    indexing: m_i = theta_i tilde-u_i + B(w_i - theta_i r_i) with
    theta_i = <r_i, w_i> / <r_i, r_i>; theta = 1 gives Alg. 8, theta = 0 Alg. 7.
    """
    res = Result(x=x0.copy())
    mon = _Monitor(A, b, prm, res)
    x = np.array(x0, dtype=np.float64)
    after_bd = False
    while True:
        # pipeline fill
        r = b - A(x)
        u = B(r)                 # tilde-u_0
        P = {0: u.copy()}        # p_0
        w = A(P[0])              # w_0
        m = B(w)                 # m_0
        n = A(m)                 # n_0
        gamma = dot(u, r)
        delta = dot(u, w)
        S = {0: w.copy()}
        Q = {0: m.copy()}
        Z = {0: n.copy()}
        eta = {0: delta}
        alpha = gamma / eta[0] if eta[0] != 0.0 else float("nan")
        conv = mon.record(mon.rho(gamma, r), gamma=gamma, delta=delta, eta=eta[0], alpha=alpha)
        if conv:
            if mon.accept(x):
                return mon.finish(x, "converged")
            continue
        if eta[0] <= 0.0:
            return mon.finish(x, "breakdown")
        i = 0
        while True:
            if res.iterations >= prm.maxit:
                return mon.finish(x, "maxit")
            i += 1
            x = axpy(x, alpha, P[i - 1])
            r = axpy(r, -alpha, S[i - 1])
            u = axpy(u, -alpha, Q[i - 1])
            w = axpy(w, -alpha, Z[i - 1])
            res.iterations += 1
            gamma = dot(u, r)
            nu = nu_window(i, prm)
            beta = {k: -dot(u, S[k]) / eta[k] for k in range(i - nu, i)}
            delta = dot(u, w)
            conv = mon.record(mon.rho(gamma, r), gamma=gamma, delta=delta, nu=nu,
                              rnorm=float(np.sqrt(dot(r, r))))
            if conv:
                if mon.accept(x):
                    return mon.finish(x, "converged")
                after_bd = False
                break
            if naive:
                m = B(w)
            elif theta:
                th = dot(r, w) / dot(r, r)
                m = axpy(B(axpy(w, -th, r)), th, u)
            else:
                m = u + B(w - r)
            n = A(m)
            P[i] = _maxpy(u, beta, P)
            S[i] = _maxpy(w, beta, S)
            Q[i] = _maxpy(m, beta, Q)
            Z[i] = _maxpy(n, beta, Z)
            eta[i] = delta - sum(beta[k] ** 2 * eta[k] for k in sorted(beta))
            alpha = gamma / eta[i] if eta[i] != 0.0 else float("nan")
            res.history[-1].update(eta=eta[i], alpha=alpha)
            if prm.trace:
                res.trace.append(dict(i=i, x=x.copy(), r=r.copy(), u=u.copy(), w=w.copy(),
                                      m=m.copy(), n=n.copy(), p=P[i].copy(), s=S[i].copy(),
                                      q=Q[i].copy(), z=Z[i].copy(), eta=eta[i], gamma=gamma,
                                      delta=delta, window=dict(P)))
            for k in [k for k in P if k < i - prm.mmax]:
                del P[k], S[k], Q[k], Z[k], eta[k]
            if eta[i] <= 0.0:
                if mon.breakdown(i, after_bd):
                    return mon.finish(x, "breakdown")
                after_bd = True
                break
            after_bd = False


# ---------------------------------------------------------------------------
# Conjugate-residual family (Sec. 4)
# ---------------------------------------------------------------------------

def gcr(A, B, b, x0, prm: Params) -> Result:
    """Generalized conjugate residuals, Alg. 9 (Eisenstat)."""
    res = Result(x=x0.copy())
    mon = _Monitor(A, b, prm, res)
    x = np.array(x0, dtype=np.float64)
    after_bd = False
    while True:
        r = b - A(x)
        u = B(r)
        P = {0: u.copy()}
        S = {0: A(P[0])}
        gamma = dot(u, S[0]) if prm.gcr_literal_gamma else dot(r, S[0])
        eta = {0: dot(S[0], S[0])}
        conv = mon.record(mon.rho(gamma, r), gamma=gamma, eta=eta[0])
        if conv:
            if mon.accept(x):
                return mon.finish(x, "converged")
            continue
        if eta[0] <= 0.0:
            return mon.finish(x, "breakdown")
        alpha = gamma / eta[0]
        i = 0
        while True:
            if res.iterations >= prm.maxit:
                return mon.finish(x, "maxit")
            i += 1
            x = axpy(x, alpha, P[i - 1])
            r = axpy(r, -alpha, S[i - 1])
            res.iterations += 1
            u = B(r)
            au = A(u)
            nu = nu_window(i, prm)
            beta = {k: -dot(au, S[k]) / eta[k] for k in range(i - nu, i)}
            P[i] = _maxpy(u, beta, P)
            S[i] = A(P[i])
            gamma = dot(u, S[i]) if prm.gcr_literal_gamma else dot(r, S[i])
            eta[i] = dot(S[i], S[i])
            conv = mon.record(mon.rho(gamma, r), gamma=gamma, eta=eta[i], nu=nu)
            if conv:
                if mon.accept(x):
                    return mon.finish(x, "converged")
                after_bd = False
                break
            for k in [k for k in P if k < i - prm.mmax]:
                del P[k], S[k], eta[k]
            if eta[i] <= 0.0:
                if mon.breakdown(i, after_bd):
                    return mon.finish(x, "breakdown")
                after_bd = True
                break
            after_bd = False
            alpha = gamma / eta[i]


def _pipegcr(A, B, b, x0, prm: Params, w_recurred: bool) -> Result:
    res = Result(x=x0.copy())
    mon = _Monitor(A, b, prm, res)
    x = np.array(x0, dtype=np.float64)
    after_bd = False
    while True:
        r = b - A(x)
        u = B(r)                 # tilde-u_0
        P = {0: u.copy()}        # p_0 = tilde-u_0
        S = {0: A(P[0])}         # s_0
        Q = {0: B(S[0])}         # q_0
        Z = {}
        if w_recurred:
            Z[0] = A(Q[0])       # z_0
            w = S[0].copy()      # w_0 = A tilde-u_0 = s_0
        gamma = dot(r, A(r)) if prm.gcr_literal_init else dot(r, S[0])
        eta = {0: dot(S[0], S[0])}
        alpha = gamma / eta[0] if eta[0] != 0.0 else float("nan")
        conv = mon.record(mon.rho(gamma, r), gamma=gamma, eta=eta[0], alpha=alpha)
        if conv:
            if mon.accept(x):
                return mon.finish(x, "converged")
            continue
        if eta[0] <= 0.0:
            return mon.finish(x, "breakdown")
        i = 0
        while True:
            if res.iterations >= prm.maxit:
                return mon.finish(x, "maxit")
            i += 1
            x = axpy(x, alpha, P[i - 1])
            r = axpy(r, -alpha, S[i - 1])
            u = axpy(u, -alpha, Q[i - 1])
            if w_recurred:
                w = axpy(w, -alpha, Z[i - 1])
            else:
                w = A(u)
            res.iterations += 1
            gamma = dot(r, w)
            delta = dot(w, w)
            nu = nu_window(i, prm)
            beta = {k: -dot(w, S[k]) / eta[k] for k in range(i - nu, i)}
            conv = mon.record(mon.rho(gamma, r), gamma=gamma, delta=delta, nu=nu,
                              rnorm=float(np.sqrt(dot(r, r))))
            if conv:
                if mon.accept(x):
                    return mon.finish(x, "converged")
                after_bd = False
                break
            m = B(w - r) + u
            P[i] = _maxpy(u, beta, P)
            S[i] = _maxpy(w, beta, S)
            Q[i] = _maxpy(m, beta, Q)
            if w_recurred:
                n = A(m)
                Z[i] = _maxpy(n, beta, Z)
            eta[i] = delta - sum(beta[k] ** 2 * eta[k] for k in sorted(beta))
            alpha = gamma / eta[i] if eta[i] != 0.0 else float("nan")
            res.history[-1].update(eta=eta[i], alpha=alpha)
            if prm.trace:
                res.trace.append(dict(i=i, x=x.copy(), r=r.copy(), u=u.copy(), w=w.copy(),
                                      m=m.copy(), p=P[i].copy(), s=S[i].copy(), q=Q[i].copy(),
                                      z=Z[i].copy() if w_recurred else None, eta=eta[i],
                                      window_s=dict(S)))
            for k in [k for k in P if k < i - prm.mmax]:
                del P[k], S[k], Q[k], eta[k]
                Z.pop(k, None)
            if eta[i] <= 0.0:
                if mon.breakdown(i, after_bd):
                    return mon.finish(x, "breakdown")
                after_bd = True
                break
            after_bd = False


def pipegcr(A, B, b, x0, prm: Params) -> Result:
    """Pipelined GCR with explicit w_i = A tilde-u_i, Alg. 11."""
    return _pipegcr(A, B, b, x0, prm, w_recurred=False)


def pipegcr_w(A, B, b, x0, prm: Params) -> Result:
    """Pipelined GCR with recurred w and a z history, Alg. 12."""
    return _pipegcr(A, B, b, x0, prm, w_recurred=True)


# ---------------------------------------------------------------------------
# Flexible GMRES family (Sec. 5)
# ---------------------------------------------------------------------------

def _lsq(H: np.ndarray, beta0: float):
    """y = argmin ||H y - beta0 e_0||_2 and the residual norm (library lstsq)."""
    rhs = np.zeros(H.shape[0])
    rhs[0] = beta0
    if H.shape[1] == 0:
        return np.zeros(0), abs(beta0)
    y = np.linalg.lstsq(H, rhs, rcond=None)[0]
    return y, float(np.linalg.norm(H @ y - rhs))


def fgmres(A, B, b, x0, prm: Params) -> Result:
    """Flexible GMRES(m), Alg. 13 (classical Gram-Schmidt as printed), restarted."""
    res = Result(x=x0.copy())
    mon = _Monitor(A, b, prm, res)
    x = np.array(x0, dtype=np.float64)
    m = prm.mmax
    while True:
        r0 = b - A(x)
        beta0 = float(np.linalg.norm(r0))
        conv = mon.record(beta0)
        if conv:
            if mon.accept(x):
                return mon.finish(x, "converged")
            continue
        P = [r0 / beta0]
        U = [B(P[0])]
        z = A(U[0])
        H = np.zeros((m + 1, m))
        done = None
        ncols = 0
        for i in range(1, m + 1):
            if res.iterations >= prm.maxit:
                done = "maxit"
                break
            for j in range(i):
                H[j, i - 1] = dot(P[j], z)
            pbar = z.copy()
            for j in range(i):
                pbar = axpy(pbar, -H[j, i - 1], P[j])
            H[i, i - 1] = float(np.linalg.norm(pbar))
            res.iterations += 1
            ncols = i
            _, est = _lsq(H[:i + 1, :i], beta0)
            if mon.record(est) or H[i, i - 1] == 0.0:
                done = "converged"
                break
            if i == m:
                break
            P.append(pbar / H[i, i - 1])
            U.append(B(P[i]))
            z = A(U[i])
        y, _ = _lsq(H[:ncols + 1, :ncols], beta0)
        if prm.trace and ncols:
            res.trace.append(dict(x0=x.copy(), P=[v.copy() for v in P], U=[v.copy() for v in U],
                                  H=H[:ncols + 1, :ncols].copy(), ncols=ncols, y=y))
        x = x + np.column_stack(U[:ncols]) @ y if ncols else x
        if done == "maxit":
            return mon.finish(x, "maxit")
        if done == "converged" and mon.accept(x):
            return mon.finish(x, "converged")
        res.cycles += 1


def estimate_sigma(A, B, b, iters: int = 10) -> float:
    """Shift for CGFGMRES / PIPEFGMRES when none is given: an estimate of the
    largest eigenvalue of the preconditioned operator (Sec. 5.3), by power
    iteration on v -> A B(v) from v = b / ||b||; returns ||A B(v)|| of the last
    step (||v|| = 1)."""
    v = np.asarray(b, dtype=np.float64) / np.linalg.norm(b)
    nrm = 0.0
    for _ in range(iters):
        y = A(B(v))
        nrm = float(np.linalg.norm(y))
        v = y / nrm
    return nrm


def _fgmres_single_reduction(A, B, b, x0, prm: Params, pipelined: bool) -> Result:
    res = Result(x=x0.copy())
    mon = _Monitor(A, b, prm, res)
    x = np.array(x0, dtype=np.float64)
    m = prm.mmax
    sigma = prm.sigma if not np.isnan(prm.sigma) else estimate_sigma(A, B, b)
    res.sigma = sigma
    after_bd = False
    while True:
        r0 = b - A(x)
        beta0 = float(np.linalg.norm(r0))
        conv = mon.record(beta0)
        if conv:
            if mon.accept(x):
                return mon.finish(x, "converged")
            continue
        P = [r0 / beta0]                  # p_0
        U = [B(P[0])]                     # u_0 (first column of tilde-U)
        Zb = [axpy(A(U[0]), -sigma, P[0])]     # zbar_0
        if pipelined:
            qb = B(Zb[0])                 # qbar_0
            wb = A(qb)                    # wbar_0
        H = np.zeros((m + 1, m))
        Hb = np.zeros((m + 1, m))
        status = None
        ncols = 0
        for i in range(1, m + 1):
            if res.iterations >= prm.maxit:
                status = "maxit"
                break
            for j in range(i - 1):
                Hb[j, i - 1] = dot(P[j], Zb[i - 1])
                H[j, i - 1] = Hb[j, i - 1]
            Hb[i - 1, i - 1] = dot(P[i - 1], Zb[i - 1])
            H[i - 1, i - 1] = Hb[i - 1, i - 1] + sigma
            t = dot(Zb[i - 1], Zb[i - 1]) - sum(Hb[k, i - 1] ** 2 for k in range(i))
            if t < 0.0:
                status = "breakdown"
                break
            Hb[i, i - 1] = float(np.sqrt(t))
            H[i, i - 1] = Hb[i, i - 1]
            res.iterations += 1
            ncols = i
            _, est = _lsq(H[:i + 1, :i], beta0)
            if mon.record(est, t=t) or t == 0.0:
                status = "converged"
                break
            if i == m:
                break
            hb = Hb[i, i - 1]
            pi = Zb[i - 1].copy()
            for k in range(i):
                pi = axpy(pi, -Hb[k, i - 1], P[k])
            P.append(pi / hb)
            if pipelined:
                ui = qb.copy()
                for k in range(i):
                    ui = axpy(ui, -Hb[k, i - 1], U[k])
                U.append(ui / hb)
                zi = wb.copy()
                for k in range(i):
                    zi = axpy(zi, -H[k, i - 1], Zb[k])
                Zb.append(zi / H[i, i - 1])
                qb = B(Zb[i])
                wb = A(qb)
            else:
                U.append(B(P[i]))
                Zb.append(axpy(A(U[i]), -sigma, P[i]))
        if ncols:
            y, _ = _lsq(H[:ncols + 1, :ncols], beta0)
            if prm.trace:
                res.trace.append(dict(x0=x.copy(), P=[v.copy() for v in P], U=[v.copy() for v in U],
                                      Zb=[v.copy() for v in Zb], H=H[:ncols + 1, :ncols].copy(),
                                      Hb=Hb[:ncols + 1, :ncols].copy(), ncols=ncols, y=y))
            x = x + np.column_stack(U[:ncols]) @ y
        if status == "maxit":
            return mon.finish(x, "maxit")
        if status == "breakdown":
            if mon.breakdown(ncols + 1, after_bd):
                return mon.finish(x, "breakdown")
            after_bd = True
            continue
        after_bd = False
        if status == "converged" and mon.accept(x):
            return mon.finish(x, "converged")
        res.cycles += 1


def cgfgmres(A, B, b, x0, prm: Params) -> Result:
    """Single-reduction FGMRES with constant shift sigma, Alg. 14."""
    return _fgmres_single_reduction(A, B, b, x0, prm, pipelined=False)


def pipefgmres(A, B, b, x0, prm: Params) -> Result:
    """Pipelined FGMRES with constant shift sigma, Alg. 15 with eq. (pipefgmresz)."""
    return _fgmres_single_reduction(A, B, b, x0, prm, pipelined=True)


METHODS = {
    "pcg": pcg, "fcg": fcg, "cgfcg": cgfcg, "pipefcg": pipefcg,
    "pipefcg_naive": lambda A, B, b, x0, prm: pipefcg(A, B, b, x0, prm, naive=True),
    "pipefcg_theta": lambda A, B, b, x0, prm: pipefcg(A, B, b, x0, prm, theta=True),
    "gcr": gcr, "pipegcr": pipegcr, "pipegcr_w": pipegcr_w,
    "fgmres": fgmres, "cgfgmres": cgfgmres, "pipefgmres": pipefgmres,
}


def solve(method: str, A, B, b, x0=None, prm: Params = None) -> Result:
    if x0 is None:
        x0 = np.zeros_like(np.asarray(b, dtype=np.float64))
    return METHODS[method](A, B, np.asarray(b, dtype=np.float64), np.asarray(x0, dtype=np.float64),
                           prm or Params())
