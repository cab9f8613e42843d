"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This module only draws random numbers and lays out arrays.  It holds none of
the Krylov methods' arithmetic, no operator application and no preconditioner:
both the oracle and the GPU library receive the same arrays from here and
compute everything else on their own.

Seeds: ``numpy.random.default_rng([config_id, item_id, 151107226])``.

Workloads (stand-ins for the paper's pTatin3D viscous sinker and PETSc ex43
Stokes problems, which are not available; they keep the traits the paper
stresses in Sec. 6: heterogeneous viscosity, sharp inclusions, high contrast):

* ``poisson2d_inclusions``  -- 64x64 cells, eta = 1e3 inside 8 random squares
  (side U{4..12}), 1 elsewhere; f ~ U(-1, 1).
* ``poisson3d_gaussian``    -- n^3 cells, eta = 10^(3 g), g a (almost-)Gaussian
  random field with correlation length 8 cells, clipped to [-1, 1] (contrast
  1e6).  Generated from IEEE additions, multiplications and divisions only, so
  the arrays are bitwise the same on every platform.
* ``poisson3d_two_phase``   -- n^3 cells, eta = 1 with 1e4 spheres covering
  >= 20 % of the volume, constant advection velocity with global Peclet 10.
* ``batched2d``             -- many 2D systems, sides U[32, 256], eta = 10^(2 g).
* ``request_stream``        -- Poisson arrivals of 3D solves for serving.
* ``toy_diagonal``          -- the diagonal toy system of the FCG noise study
  (Sec. 3.2.1, Fig. FCGtoy): n = 100, condition number 5.

Right-hand sides are returned already scaled as b = h^2 f with h = 1/nx, the
cell-centred finite-volume scaling in which the operator carries no h.
"""
from __future__ import annotations

import numpy as np

SEED_SALT = 151107226


def rng(config_id: int, item_id: int = 0) -> np.random.Generator:
    return np.random.default_rng([int(config_id), int(item_id), SEED_SALT])


# exp(x) from IEEE additions and multiplications only (the library exp and the
# FFT differ in their last bits between platforms, and the inputs must be
# bitwise the same on every machine that generates them): Cody-Waite reduction
# x = k ln2 + r with the two-part ln2 of fdlibm, |r| <= ln2 / 2, a degree-13
# Taylor polynomial of e^r by Horner's rule (truncation error < 1e-17), and an
# exact scaling by 2^k.  Relative error ~1e-15.
_LN2_HI = 6.93147180369123816490e-01
_LN2_LO = 1.90821492927058770002e-10
_INV_LN2 = 1.44269504088896338700e+00
_LN10 = 2.30258509299404568402e+00


def _exp_coefficients(deg: int = 13) -> list:
    from fractions import Fraction
    from math import factorial
    return [float(Fraction(1, factorial(j))) for j in range(deg + 1)]


_EXP_C = _exp_coefficients()


def portable_exp(x) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    k = np.rint(x * _INV_LN2)
    r = (x - k * _LN2_HI) - k * _LN2_LO
    p = np.full_like(r, _EXP_C[-1])
    for c in reversed(_EXP_C[:-1]):
        p = p * r + c
    return np.ldexp(p, k.astype(np.int32))


def portable_pow10(x) -> np.ndarray:
    """10^x = exp(x ln 10) with portable_exp."""
    return portable_exp(np.asarray(x, dtype=np.float64) * _LN10)


def box_widths(sigma: float, passes: int = 4) -> list:
    """Odd widths of `passes` box filters whose repeated application has
    (close to) the variance sigma^2 of a Gaussian kernel: Kovesi's rule (Fast
    almost-Gaussian filtering, 2010) -- m passes of width wl and the rest of
    width wl + 2, wl the largest odd width not above the ideal one."""
    ideal = np.sqrt(12.0 * sigma * sigma / passes + 1.0)
    wl = int(np.floor(ideal))
    if wl % 2 == 0:
        wl -= 1
    wl = max(wl, 1)
    wu = wl + 2
    m = int(round((12.0 * sigma * sigma - passes * wl * wl - 4 * passes * wl - 3 * passes) / (-4.0 * wl - 4.0)))
    m = min(max(m, 0), passes)
    return [wl] * m + [wu] * (passes - m)


def _box_periodic(f: np.ndarray, axis: int, width: int) -> np.ndarray:
    """Periodic moving average of odd `width` along `axis`, from a running sum
    (numpy.cumsum adds strictly in order, so the result is the same on every
    platform)."""
    if width <= 1:
        return f
    half = width // 2
    n = f.shape[axis]
    idx = np.arange(-half - 1, n + half) % n
    padded = np.take(f, idx, axis=axis)
    cs = np.cumsum(padded, axis=axis)
    hi = np.take(cs, np.arange(width, width + n), axis=axis)
    lo = np.take(cs, np.arange(0, n), axis=axis)
    return (hi - lo) / float(width)


def gaussian_field(shape, ell: float, g: np.random.Generator) -> np.ndarray:
    """White N(0,1) noise smoothed by an almost-Gaussian periodic filter.

    Covariance exp(-r^2 / (2 ell^2)) needs a kernel of std ell/sqrt(2); the
    kernel is approximated by four passes of periodic box filters per axis
    whose combined variance is (close to) ell^2 / 2 (box_widths).  The field is
    then normalised to zero mean and unit sample std and clipped to [-1, 1].
    Every step is additions, multiplications and divisions in a fixed order,
    so the field is bitwise the same on every platform.
    """
    w = g.standard_normal(shape)
    s = ell / np.sqrt(2.0)
    f = w
    for ax in range(len(shape)):
        for width in box_widths(s):
            f = _box_periodic(f, ax, width)
    f = f - f.mean()
    sd = f.std()
    if sd > 0:
        f = f / sd
    return np.clip(f, -1.0, 1.0)


def _rhs(shape, g: np.random.Generator, nx: int) -> np.ndarray:
    h = 1.0 / nx
    f = g.uniform(-1.0, 1.0, size=shape)
    return (h * h) * f.reshape(-1)


def poisson2d_inclusions(nx: int = 64, ny: int = 64, n_incl: int = 8, contrast: float = 1e3,
                         config_id: int = 1, item_id: int = 0) -> dict:
    g = rng(config_id, item_id)
    eta = np.ones((ny, nx))
    for _ in range(n_incl):
        side = int(g.integers(4, 13))
        side = min(side, nx, ny)
        i0 = int(g.integers(0, nx - side + 1))
        j0 = int(g.integers(0, ny - side + 1))
        eta[j0:j0 + side, i0:i0 + side] = contrast
    b = _rhs((ny, nx), g, nx)
    return dict(dims=(nx, ny, 1), eta=eta.reshape(-1).copy(), b=b, vel=(0.0, 0.0, 0.0))


def poisson3d_gaussian(n: int = 128, ell: float = 8.0, log_contrast: float = 3.0,
                       config_id: int = 2, item_id: int = 0, dims=None) -> dict:
    nx, ny, nz = dims if dims is not None else (n, n, n)
    g = rng(config_id, item_id)
    field = gaussian_field((nz, ny, nx), ell, g)
    eta = portable_pow10(log_contrast * field)
    b = _rhs((nz, ny, nx), g, nx)
    return dict(dims=(nx, ny, nz), eta=eta.reshape(-1).copy(), b=b, vel=(0.0, 0.0, 0.0))


def poisson3d_two_phase(n: int = 256, eta_hi: float = 1e4, vol_frac: float = 0.2,
                        r_lo: float = 8.0, r_hi: float = 24.0, peclet: float = 10.0,
                        config_id: int = 3, item_id: int = 0) -> dict:
    g = rng(config_id, item_id)
    inside = np.zeros((n, n, n), dtype=bool)
    scale = n / 256.0
    target = vol_frac * n ** 3
    count = 0
    while count < target:
        r = g.uniform(r_lo, r_hi) * scale
        c = g.uniform(0.0, n, size=3)
        lo = np.maximum(np.floor(c - r).astype(int), 0)
        hi = np.minimum(np.ceil(c + r).astype(int) + 1, n)
        zz, yy, xx = np.meshgrid(np.arange(lo[2], hi[2]) + 0.5, np.arange(lo[1], hi[1]) + 0.5,
                                 np.arange(lo[0], hi[0]) + 0.5, indexing="ij")
        m = (xx - c[0]) ** 2 + (yy - c[1]) ** 2 + (zz - c[2]) ** 2 <= r * r
        sub = inside[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        sub |= m
        count = int(inside.sum())
    eta = np.where(inside, eta_hi, 1.0)
    v = peclet / np.sqrt(3.0)
    b = _rhs((n, n, n), g, n)
    return dict(dims=(n, n, n), eta=eta.reshape(-1).copy(), b=b, vel=(v, v, v))


def batched2d_sides(count: int = 512, lo: int = 32, hi: int = 256, config_id: int = 4) -> np.ndarray:
    g = rng(config_id, 1_000_000)
    return g.integers(lo, hi + 1, size=count)


def batched2d_system(index: int, side: int, ell: float = 8.0, log_contrast: float = 2.0,
                     config_id: int = 4) -> dict:
    g = rng(config_id, index)
    field = gaussian_field((side, side), ell, g)
    eta = portable_pow10(log_contrast * field)
    b = _rhs((side, side), g, side)
    return dict(dims=(side, side, 1), eta=eta.reshape(-1).copy(), b=b, vel=(0.0, 0.0, 0.0))


def request_stream(count: int = 2000, rate: float = 200.0, side_lo: int = 32, side_hi: int = 160,
                   config_id: int = 5) -> list:
    """Arrival time, side, log10 contrast and method index of each request."""
    g = rng(config_id, 1_000_000)
    gaps = g.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps)
    sides = g.integers(side_lo, side_hi + 1, size=count)
    logc = g.uniform(2.0, 6.0, size=count)
    meth = g.integers(0, 3, size=count)
    return [dict(t=float(t[i]), side=int(sides[i]), log_contrast=float(logc[i]), method=int(meth[i]),
                 item_id=i) for i in range(count)]


def request_problem(req: dict, ell: float = 8.0, config_id: int = 5) -> dict:
    n = req["side"]
    return poisson3d_gaussian(n=n, ell=ell, log_contrast=req["log_contrast"] / 2.0,
                              config_id=config_id, item_id=req["item_id"])


def toy_diagonal(n: int = 100, kappa: float = 5.0) -> dict:
    lam = np.linspace(1.0, kappa, n)
    b = np.full(n, 1.0 / np.sqrt(n))
    return dict(diag=lam, b=b)


def noise_bank(n: int, count: int, seed_item: int = 0, config_id: int = 101) -> np.ndarray:
    """Gaussian vectors for the noisy preconditioner of the toy study (one per call)."""
    return rng(config_id, seed_item).standard_normal((count, n))


def random_spd(n: int, cond: float = 100.0, item_id: int = 0, config_id: int = 102) -> np.ndarray:
    g = rng(config_id, item_id)
    q, _ = np.linalg.qr(g.standard_normal((n, n)))
    lam = np.geomspace(1.0, cond, n)
    a = (q * lam) @ q.T
    return 0.5 * (a + a.T)


def random_nonsym(n: int, shift: float = 3.0, item_id: int = 0, config_id: int = 103) -> np.ndarray:
    g = rng(config_id, item_id)
    return shift * np.eye(n) + g.standard_normal((n, n)) / np.sqrt(n)


def random_vector(n: int, item_id: int = 0, config_id: int = 104) -> np.ndarray:
    return rng(config_id, item_id).standard_normal(n)


def random_csr(n: int, per_row: int = 7, item_id: int = 0, config_id: int = 105):
    """Random diagonally dominant CSR matrix (int32 indices, sorted columns)."""
    g = rng(config_id, item_id)
    rowptr = [0]
    cols, vals = [], []
    for i in range(n):
        k = int(g.integers(0, per_row))
        c = set(int(v) for v in g.integers(0, n, size=k))
        c.add(i)
        c = sorted(c)
        v = g.uniform(-1.0, 1.0, size=len(c))
        v[c.index(i)] = float(len(c)) + 1.0
        cols.extend(c)
        vals.extend(v.tolist())
        rowptr.append(len(cols))
    return (np.asarray(rowptr, dtype=np.int32), np.asarray(cols, dtype=np.int32),
            np.asarray(vals, dtype=np.float64))
