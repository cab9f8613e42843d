"""Operators A for the oracle, written from their definitions.

Variable-coefficient Poisson problem -div(eta grad u) = f on the unit square or
cube, cell-centred finite volumes, homogeneous Dirichlet boundary, scaled so the
operator carries no h (the right-hand side is h^2 f):

    (A u)_i = sum over the faces f of cell i of K_f (u_i - u_nbr(f))

* interior face between cells i and j: K_f = 2 eta_i eta_j / (eta_i + eta_j)
  (harmonic mean of the two cell viscosities);
* boundary face: K_f = 2 eta_i and u_nbr = 0 (the Dirichlet value, mirrored).

Optional constant advection velocity v (nonsymmetric case), first-order upwind
of v . grad u in the same scaling: + h |v_d| (u_i - u_up) for each direction d,
where u_up is the neighbour at -e_d if v_d > 0 and at +e_d if v_d < 0, and the
upwind ghost outside the domain is 0.  h = 1/nx.

Cell ordering: index = i + nx (j + ny k), i.e. arrays of shape (nz, ny, nx) in
C order.  The paper's operators are SpMVs with n_z = 7 nonzeros per row in 3D
(Sec. 8, performance model); this is the matrix-free form of such a stencil.
"""
from __future__ import annotations

import numpy as np


def _shift(u: np.ndarray, axis: int, step: int) -> np.ndarray:
    """v[idx] = u[idx + step along axis], zero outside the domain."""
    v = np.zeros_like(u)
    n = u.shape[axis]
    src = [slice(None)] * u.ndim
    dst = [slice(None)] * u.ndim
    if step > 0:
        src[axis] = slice(step, n)
        dst[axis] = slice(0, n - step)
    else:
        src[axis] = slice(0, n + step)
        dst[axis] = slice(-step, n)
    v[tuple(dst)] = u[tuple(src)]
    return v


class StencilOperator:
    """5-point (2D) / 7-point (3D) finite-volume operator, matrix-free."""

    def __init__(self, dims, eta, vel=(0.0, 0.0, 0.0)):
        nx, ny, nz = (tuple(dims) + (1, 1))[:3]
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.ndim = 3 if self.nz > 1 else 2
        self.shape = (self.nz, self.ny, self.nx) if self.ndim == 3 else (self.ny, self.nx)
        self.n = self.nx * self.ny * self.nz
        self.eta = np.asarray(eta, dtype=np.float64).reshape(self.shape)
        self.vel = tuple(float(v) for v in (tuple(vel) + (0.0, 0.0, 0.0))[:3])
        self.h = 1.0 / self.nx
        # axis of the array for each direction d = x, y, z
        self.axes = [self.ndim - 1, self.ndim - 2] + ([0] if self.ndim == 3 else [])
        # K[(d, s)] = coefficient of the face of each cell on side s (-1 or +1) in direction d
        self.K = {}
        for d, ax in enumerate(self.axes):
            for s in (-1, +1):
                nb = _shift(self.eta, ax, s)
                inside = _shift(np.ones_like(self.eta), ax, s) > 0
                e = self.eta
                harm = np.zeros_like(e)
                harm[inside] = 2.0 * e[inside] * nb[inside] / (e[inside] + nb[inside])
                bnd = 2.0 * e
                self.K[(d, s)] = np.where(inside, harm, bnd)
        self.adv = [self.h * abs(self.vel[d]) for d in range(self.ndim)]

    def apply(self, u: np.ndarray) -> np.ndarray:
        u = np.asarray(u, dtype=np.float64).reshape(self.shape)
        y = np.zeros_like(u)
        for d, ax in enumerate(self.axes):
            for s in (-1, +1):
                y += self.K[(d, s)] * (u - _shift(u, ax, s))
        for d, ax in enumerate(self.axes):
            v = self.vel[d]
            if v != 0.0:
                up = -1 if v > 0 else +1
                y += self.adv[d] * (u - _shift(u, ax, up))
        return y.reshape(-1)

    __call__ = apply

    def diagonal(self) -> np.ndarray:
        dg = np.zeros(self.shape)
        for key in self.K:
            dg += self.K[key]
        for d in range(self.ndim):
            dg += self.adv[d]
        return dg.reshape(-1)

    def to_dense(self) -> np.ndarray:
        """Column-by-column application to unit vectors (small grids only)."""
        a = np.zeros((self.n, self.n))
        e = np.zeros(self.n)
        for j in range(self.n):
            e[j] = 1.0
            a[:, j] = self.apply(e)
            e[j] = 0.0
        return a

    def to_csr(self):
        """Assemble the same operator as CSR (int32 indices, ascending columns)."""
        idx = np.arange(self.n).reshape(self.shape)
        rows = [idx.reshape(-1)]
        cols = [idx.reshape(-1)]
        vals = [self.diagonal()]
        for d, ax in enumerate(self.axes):
            for s in (-1, +1):
                inside = _shift(np.ones(self.shape), ax, s) > 0
                nbr = _shift(idx.astype(np.float64) + 1.0, ax, s) - 1.0
                coef = -self.K[(d, s)]
                v = self.vel[d]
                if v != 0.0 and s == (-1 if v > 0 else +1):
                    coef = coef - self.adv[d]
                rows.append(idx[inside])
                cols.append(nbr[inside].astype(np.int64))
                vals.append(coef[inside])
        r = np.concatenate(rows)
        c = np.concatenate(cols)
        v = np.concatenate(vals)
        order = np.lexsort((c, r))
        r, c, v = r[order], c[order], v[order]
        rowptr = np.zeros(self.n + 1, dtype=np.int64)
        np.add.at(rowptr, r + 1, 1)
        rowptr = np.cumsum(rowptr)
        return CsrOperator(rowptr.astype(np.int32), c.astype(np.int32), v)

    def gershgorin_jacobi_bound(self) -> float:
        """max_i sum_j |a_ij| / a_ii: Gershgorin bound on the spectrum of D^-1 A."""
        dg = self.diagonal().reshape(self.shape)
        s = dg.copy()
        for key in self.K:
            d, side = key
            inside = _shift(np.ones(self.shape), self.axes[d], side) > 0
            off = np.where(inside, self.K[key], 0.0)
            v = self.vel[d]
            if v != 0.0 and side == (-1 if v > 0 else +1):
                off = np.where(inside, off + self.adv[d], 0.0)
            s = s + off
        return float(np.max(s / dg))


class CsrOperator:
    """y_i = sum_j a_ij x_j over the stored entries of row i, in column order."""

    def __init__(self, rowptr, colidx, vals):
        self.rowptr = np.asarray(rowptr, dtype=np.int64)
        self.colidx = np.asarray(colidx, dtype=np.int64)
        self.vals = np.asarray(vals, dtype=np.float64)
        self.n = len(self.rowptr) - 1
        self._rowid = np.repeat(np.arange(self.n), np.diff(self.rowptr))

    def apply(self, x: np.ndarray) -> np.ndarray:
        x = np.asarray(x, dtype=np.float64)
        prod = self.vals * x[self.colidx]
        y = np.zeros(self.n)
        np.add.at(y, self._rowid, prod)
        return y

    __call__ = apply

    def diagonal(self) -> np.ndarray:
        dg = np.zeros(self.n)
        m = self.colidx == self._rowid
        dg[self._rowid[m]] = self.vals[m]
        return dg

    def to_dense(self) -> np.ndarray:
        a = np.zeros((self.n, self.n))
        a[self._rowid, self.colidx] = self.vals
        return a


class DenseOperator:
    def __init__(self, a):
        self.a = np.asarray(a, dtype=np.float64)
        self.n = self.a.shape[0]

    def apply(self, x):
        return self.a @ np.asarray(x, dtype=np.float64)

    __call__ = apply

    def diagonal(self):
        return np.diag(self.a).copy()

    def to_dense(self):
        return self.a.copy()


class DiagonalOperator:
    def __init__(self, d):
        self.d = np.asarray(d, dtype=np.float64)
        self.n = len(self.d)

    def apply(self, x):
        return self.d * np.asarray(x, dtype=np.float64)

    __call__ = apply

    def diagonal(self):
        return self.d.copy()

    def to_dense(self):
        return np.diag(self.d)
