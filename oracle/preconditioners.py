"""Preconditioners B for the oracle.

The flexible methods accept any, possibly nonlinear, map v -> B(v)
(Sec. 2 and the notation table of Sec. 3).  The ones used here:

* ``IdentityPC``      -- B(v) = v.
* ``JacobiPC``        -- B(v) = D^-1 v, D = diag(A) (the block-Jacobi limit
                         of one cell per block, Sec. 6).
* ``InnerPCG``        -- k iterations of Jacobi-preconditioned CG (Alg. 3 with
                         M^-1 = D^-1), zero initial guess, no tolerance test.
                         Sec. 6 uses 5 such inner iterations per block; this is
                         nonlinear in v, hence a flexible preconditioner.
* ``Chebyshev``       -- k Chebyshev-Jacobi sweeps on D^-1 A over [lo, hi]
                         (Saad, Iterative Methods for Sparse Linear Systems,
                         2nd ed., Alg. 12.1), zero initial guess.
* ``NoisyPC``         -- B(r) = r + eta ||r|| xi / ||xi|| with Gaussian xi,
                         the pathological preconditioner of Fig. FCGtoy.
* ``DensePC``         -- B(v) = M v for a given matrix (e.g. A^-1).
* ``BlockUpperPC``    -- the right preconditioner of the nested Stokes
                         experiment (Sec. 6, ex43): B = [K_hat B^T; 0 S_hat]^-1
                         with S_hat diagonal and K_hat^-1 an inexact inner
                         flexible Krylov solve of the viscous block.

Reduced-precision copies (``precision='fp32'`` / ``'bf16'``) emulate the
mixed-precision preconditioners: the preconditioner's copy of A stores the
diagonal, the interior face coefficients and D^-1, each rounded
FP64 -> FP32 (-> BF16, round to nearest even); constant advection weights stay
FP32; vector arithmetic is FP32; inner products are accumulated in FP64 from
the FP32 values.  The paper fixes no reduced-precision arithmetic; this
rounding model is the reading, pinned by its properties (format
representability and unit-roundoff bounds of the copies, the copy's operator
error bound, the Chebyshev closed form with the rounded D^-1, the one-cell
inner PCG).
"""
from __future__ import annotations

import numpy as np

from .operators import StencilOperator, _shift


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round FP32 values to BF16 (round to nearest, ties to even), returned as FP32.

    Works on the bit pattern: add 0x7FFF plus the lowest kept bit, then clear the
    16 low bits.  NaN stays NaN.
    """
    f = np.asarray(x, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    r = ((bits + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).copy()
    nan = np.isnan(f)
    out[nan] = np.float32(np.nan)
    return out


def round_coefficients(x64: np.ndarray, precision: str) -> np.ndarray:
    x32 = np.asarray(x64, dtype=np.float64).astype(np.float32)
    if precision == "fp32":
        return x32
    if precision == "bf16":
        return bf16_round(x32)
    raise ValueError(precision)


class RoundedStencil:
    """The preconditioner's reduced-precision copy of a stencil operator.

    y = d u - sum_interior K_f u_nbr - sum_d a_d u_up, with d, K_f rounded per
    ``precision`` and a_d = h |v_d| in FP32; arithmetic in FP32.
    """

    def __init__(self, op: StencilOperator, precision: str):
        self.op = op
        self.shape = op.shape
        self.d = round_coefficients(op.diagonal(), precision).reshape(op.shape)
        self.dinv = round_coefficients(1.0 / op.diagonal(), precision).reshape(op.shape)
        self.K = {}
        for key, k in op.K.items():
            dd, s = key
            inside = _shift(np.ones(op.shape), op.axes[dd], s) > 0
            self.K[key] = np.where(inside, round_coefficients(k, precision).reshape(op.shape),
                                   np.float32(0.0)).astype(np.float32)
        self.adv = [np.float32(a) for a in op.adv]

    def apply(self, u32: np.ndarray) -> np.ndarray:
        u = np.asarray(u32, dtype=np.float32).reshape(self.shape)
        y = self.d * u
        for (dd, s), k in self.K.items():
            y = y - k * _shift(u, self.op.axes[dd], s)
        for dd, ax in enumerate(self.op.axes):
            v = self.op.vel[dd]
            if v != 0.0:
                up = -1 if v > 0 else +1
                y = y - self.adv[dd] * _shift(u, ax, up)
        return y.reshape(-1).astype(np.float32)


def _dot(a, b) -> float:
    return float(np.dot(np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)))


def _axpy(y, a, v):
    """y + a v (the vector updates of the inner iterations go through here)."""
    return y + a * v


class IdentityPC:
    linear = True

    def __call__(self, v):
        return np.array(v, dtype=np.float64, copy=True)


class JacobiPC:
    linear = True

    def __init__(self, A):
        self.dinv = 1.0 / A.diagonal()

    def __call__(self, v):
        return self.dinv * np.asarray(v, dtype=np.float64)


class DensePC:
    linear = True

    def __init__(self, m):
        self.m = np.asarray(m, dtype=np.float64)

    def __call__(self, v):
        return self.m @ np.asarray(v, dtype=np.float64)


class NoisyPC:
    """B(r) = r + eta ||r|| xi_j / ||xi_j||, xi_j the j-th row of a noise bank."""

    linear = False

    def __init__(self, eta: float, bank: np.ndarray):
        self.eta = float(eta)
        self.bank = np.asarray(bank, dtype=np.float64)
        self.calls = 0

    def __call__(self, r):
        xi = self.bank[self.calls % len(self.bank)]
        self.calls += 1
        r = np.asarray(r, dtype=np.float64)
        return r + self.eta * np.linalg.norm(r) * xi / np.linalg.norm(xi)


class InnerPCG:
    """B(v) = x_k, k iterations of Alg. 3 (PCG, M^-1 = D^-1) on A x = v from x_0 = 0.

    Loop body as in Alg. 3: x_i = x_{i-1} + alpha p; r_i = r_{i-1} - alpha s;
    u_i = M^-1 r_i; gamma_i = <u_i, r_i>; beta_i = gamma_i / gamma_{i-1};
    p_i = u_i + beta_i p_{i-1}; s_i = A p_i; eta_i = <s_i, p_i>;
    alpha_i = gamma_i / eta_i.  After the k-th update of x the remaining
    statements of that iteration are not needed and are skipped.
    Guards: if gamma or eta is exactly zero, the current x is returned.
    """

    linear = False

    def __init__(self, A, k: int, precision: str = "fp64"):
        self.A = A
        self.k = int(k)
        self.precision = precision
        if precision == "fp64":
            self.apply_A = A.apply
            self.dinv = 1.0 / A.diagonal()
            self.dt = np.float64
        else:
            rs = RoundedStencil(A, precision)
            self.apply_A = rs.apply
            self.dinv = rs.dinv.reshape(-1)
            self.dt = np.float32

    def __call__(self, v):
        dt = self.dt
        v = np.asarray(v, dtype=np.float64).astype(dt)
        x = np.zeros_like(v)
        r = v.copy()                      # r_0 = v - A x_0, x_0 = 0
        u = (self.dinv * r).astype(dt)    # u_0 = M^-1 r_0
        p = u.copy()                      # p_0 = u_0
        s = self.apply_A(p).astype(dt)    # s_0 = A p_0
        gamma = _dot(u, r)
        eta = _dot(s, p)
        if gamma == 0.0 or eta == 0.0:
            return x.astype(np.float64)
        alpha = gamma / eta
        for i in range(1, self.k + 1):
            x = _axpy(x, dt(alpha), p).astype(dt)
            if i == self.k:
                break
            r = _axpy(r, -dt(alpha), s).astype(dt)
            u = (self.dinv * r).astype(dt)
            gamma_new = _dot(u, r)
            if gamma_new == 0.0:
                break
            beta = gamma_new / gamma
            gamma = gamma_new
            p = _axpy(u, dt(beta), p).astype(dt)
            s = self.apply_A(p).astype(dt)
            eta = _dot(s, p)
            if eta == 0.0:
                break
            alpha = gamma / eta
        return x.astype(np.float64)


def chebyshev_bounds(A) -> tuple:
    """[0.1 lam, 1.1 lam] with lam the Gershgorin bound max_i sum_j |a_ij| / a_ii."""
    lam = A.gershgorin_jacobi_bound()
    return 0.1 * lam, 1.1 * lam


class Chebyshev:
    """k Chebyshev sweeps for D^-1 A x = D^-1 v from x_0 = 0 over [lo, hi].

    theta = (hi + lo)/2, delta = (hi - lo)/2, sigma_1 = theta/delta,
    rho_0 = 1/sigma_1, r_0 = v, d_0 = D^-1 r_0 / theta; for j = 0..k-1:
    x_{j+1} = x_j + d_j; if j+1 < k: r_{j+1} = r_j - A d_j,
    rho_{j+1} = 1/(2 sigma_1 - rho_j),
    d_{j+1} = rho_{j+1} rho_j d_j + (2 rho_{j+1}/delta) D^-1 r_{j+1}.
    Returns x_k (k - 1 operator applications).
    """

    linear = True

    def __init__(self, A, k: int, lo: float = None, hi: float = None, precision: str = "fp64"):
        if lo is None or hi is None:
            lo, hi = chebyshev_bounds(A)
        self.lo, self.hi = float(lo), float(hi)
        self.k = int(k)
        self.precision = precision
        if precision == "fp64":
            self.apply_A = A.apply
            self.dinv = 1.0 / A.diagonal()
            self.dt = np.float64
        else:
            rs = RoundedStencil(A, precision)
            self.apply_A = rs.apply
            self.dinv = rs.dinv.reshape(-1)
            self.dt = np.float32

    def __call__(self, v):
        dt = self.dt
        theta = (self.hi + self.lo) / 2.0
        delta = (self.hi - self.lo) / 2.0
        sigma1 = theta / delta
        rho = 1.0 / sigma1
        r = np.asarray(v, dtype=np.float64).astype(dt)
        x = np.zeros_like(r)
        d = (self.dinv * r / dt(theta)).astype(dt)
        for j in range(self.k):
            x = (x + d).astype(dt)
            if j + 1 == self.k:
                break
            r = (r - self.apply_A(d)).astype(dt)
            rho_new = 1.0 / (2.0 * sigma1 - rho)
            d = _axpy(dt(2.0 * rho_new / delta) * (self.dinv * r), dt(rho_new * rho), d).astype(dt)
            rho = rho_new
        return x.astype(np.float64)


class BlockUpperPC:
    """B(v) = [K_hat B^T; 0 S_hat]^-1 v for v = (v_u, v_p), the block
    upper-triangular preconditioner of Sec. 6 (ex43):

        y_p = S_hat^-1 v_p,  y_u = K_hat^-1 (v_u - B^T y_p),

    S_hat a diagonal (``schur_diag``), K_hat^-1 an inner solve of K y_u = t
    with ``inner_method`` from zero, Jacobi-preconditioned, ending at the
    inner tolerance (natural norm), at ``inner_maxit`` iterations or at a norm
    breakdown (no restarts, no true-residual check).  ``Bt`` acts on the full
    vector (zero rows for the pressure block).  Nonlinear through the inner
    solve: a flexible outer method is required.
    """

    linear = False

    def __init__(self, K, Bt, schur_diag, nu: int, inner_method: str = "pipefcg", inner_mmax: int = 30,
                 inner_rtol: float = 1e-3, inner_maxit: int = 100):
        from . import krylov
        self.K, self.Bt, self.nu = K, Bt, int(nu)
        self.sinv = 1.0 / np.asarray(schur_diag, dtype=np.float64)
        self.method = inner_method
        self.prm = krylov.Params(mmax=inner_mmax, rtol=inner_rtol, maxit=inner_maxit, max_restarts=0,
                                 true_residual_check=False)
        self.inner_iterations = []

    def __call__(self, v):
        from . import krylov
        v = np.asarray(v, dtype=np.float64)
        y = np.zeros_like(v)
        y[self.nu:] = self.sinv * v[self.nu:]
        t = v[:self.nu] - self.Bt(y)[:self.nu]
        r = krylov.solve(self.method, self.K, JacobiPC(self.K), t, prm=self.prm)
        self.inner_iterations.append(r.iterations)
        y[:self.nu] = r.x
        return y
