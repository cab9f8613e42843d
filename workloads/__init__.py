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
* ``poisson3d_gaussian``    -- n^3 cells, eta = 10^(3 g), g a Gaussian random
  field with correlation length 8 cells, clipped to [-1, 1] (contrast 1e6).
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


def gaussian_field(shape, ell: float, g: np.random.Generator) -> np.ndarray:
    """White N(0,1) noise filtered by a periodic Gaussian kernel.

    Covariance exp(-r^2 / (2 ell^2)) needs a kernel of std ell/sqrt(2); the
    filter is applied in Fourier space, then the field is normalised to zero
    mean and unit sample std and clipped to [-1, 1].
    """
    w = g.standard_normal(shape)
    s = ell / np.sqrt(2.0)
    fw = np.fft.fftn(w)
    for ax, n in enumerate(shape):
        k = 2.0 * np.pi * np.fft.fftfreq(n)
        filt = np.exp(-0.5 * (k * s) ** 2)
        bshape = [1] * len(shape)
        bshape[ax] = n
        fw *= filt.reshape(bshape)
    f = np.real(np.fft.ifftn(fw))
    f -= f.mean()
    sd = f.std()
    if sd > 0:
        f /= sd
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
    eta = np.power(10.0, log_contrast * field)
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
    eta = np.power(10.0, log_contrast * field)
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
