"""Seeded 2D Stokes-like saddle-point system (stand-in for the PETSc ex43
viscous-sinker problem of Sec. 6, which is not available).

This module lays out the input arrays only (matrices in CSR form, right-hand
side, the Schur-complement diagonal); it holds none of the Krylov methods'
arithmetic.  Both the oracle and the GPU library receive these arrays.

Discretisation (MAC staggered grid on the unit square, n x n cells, h = 1/n,
all-Dirichlet velocity: no slip on every wall):

* unknowns: x-velocity on the (n-1) x n interior vertical faces, y-velocity on
  the n x (n-1) interior horizontal faces, pressure in the n x n cells;
  ordering [u_x (face i + (n-1) j), u_y (face i + n (j-1)), p (cell i + n j)];
* viscous block K = diag(K_x, K_y), K_x u = sum over the four neighbours of
  eta_f (u - u_nbr): across a cell eta of that cell, across a grid node the
  mean of the four cells around it; a neighbour face on a wall is u = 0, a
  wall half a cell away takes the ghost -u (coefficient 2 eta, eta the mean of
  the two cells along the wall);
* B = h (-div), B^T = h grad: (B^T p) on the face between cells L and R is
  h (p_R - p_L), so the system [K B^T; B 0] is symmetric (indefinite);
* rhs: buoyancy of a circular sinker, h^2 (0, -drho) on the faces inside it,
  zero divergence rhs;
* Schur diagonal S_hat = -h^2 / eta_cell (pressure mass scaled by the inverse
  viscosity, with the sign of -B K^-1 B^T).

The pressure is determined up to a constant (enclosed flow): the system is
singular but consistent (the divergence rhs is zero).
"""
from __future__ import annotations

import numpy as np

from . import rng


def sinker_viscosity(n: int, contrast: float = 25.0, radius: float = 0.15, config_id: int = 6,
                     item_id: int = 0):
    """eta = contrast inside a circle (centre jittered by the seed), 1 outside; and the mask."""
    g = rng(config_id, item_id)
    cx, cy = 0.5 + g.uniform(-0.1, 0.1, size=2)
    xc = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(xc, xc, indexing="xy")          # [j, i]
    inside = (X - cx) ** 2 + (Y - cy) ** 2 <= radius ** 2
    eta = np.where(inside, contrast, 1.0)
    return eta, inside


def _csr_from_coo(rows, cols, vals, nrows):
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(nrows + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    return np.cumsum(rowptr), cols.astype(np.int64), vals.astype(np.float64)


def stokes2d(n: int = 64, contrast: float = 25.0, drho: float = 1.0, config_id: int = 6, item_id: int = 0) -> dict:
    h = 1.0 / n
    eta, inside = sinker_viscosity(n, contrast, config_id=config_id, item_id=item_id)   # eta[j, i]
    nux, nuy, npr = (n - 1) * n, n * (n - 1), n * n
    nu = nux + nuy
    N = nu + npr
    # node viscosity enode[J, I]: mean of the four cells around interior node (I, J), I, J = 1..n-1
    enode = np.zeros((n + 1, n + 1))
    enode[1:n, 1:n] = 0.25 * (eta[:-1, :-1] + eta[:-1, 1:] + eta[1:, :-1] + eta[1:, 1:])
    rows, cols, vals = [], [], []

    def emit(r, c, v):
        rows.append(np.asarray(r).ravel()); cols.append(np.asarray(c).ravel()); vals.append(np.asarray(v).ravel())

    # ---- K_x on faces (i, j), i = 1..n-1, j = 0..n-1; index (i-1) + (n-1) j ----
    J, I = np.meshgrid(np.arange(n), np.arange(1, n), indexing="ij")
    ux = (I - 1) + (n - 1) * J
    eL, eR = eta[J, I - 1], eta[J, I]                     # cells left / right of the face
    dg = eL + eR
    m = I - 1 >= 1
    emit(ux[m], ux[m] - 1, -eL[m])
    m = I + 1 <= n - 1
    emit(ux[m], ux[m] + 1, -eR[m])
    wall = 0.5 * (eL + eR)
    for dj in (-1, 1):
        jj = J + dj
        m = (jj >= 0) & (jj <= n - 1)
        en = np.where(m, enode[np.maximum(J, jj).clip(0, n), I], 0.0)
        dg = dg + np.where(m, en, 2.0 * wall)
        emit(ux[m], ux[m] + dj * (n - 1), -en[m])
    emit(ux, ux, dg)
    # ---- K_y on faces (i, j), j = 1..n-1, i = 0..n-1; index nux + i + n (j-1) ----
    J, I = np.meshgrid(np.arange(1, n), np.arange(n), indexing="ij")
    uy = nux + I + n * (J - 1)
    eB, eT = eta[J - 1, I], eta[J, I]                     # cells below / above the face
    dg = eB + eT
    m = J - 1 >= 1
    emit(uy[m], uy[m] - n, -eB[m])
    m = J + 1 <= n - 1
    emit(uy[m], uy[m] + n, -eT[m])
    wall = 0.5 * (eB + eT)
    for di in (-1, 1):
        ii = I + di
        m = (ii >= 0) & (ii <= n - 1)
        en = np.where(m, enode[J, np.maximum(I, ii).clip(0, n)], 0.0)
        dg = dg + np.where(m, en, 2.0 * wall)
        emit(uy[m], uy[m] + di, -en[m])
    emit(uy, uy, dg)
    kr, kc, kv = np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)

    # ---- B^T = h grad on velocity rows ----
    J, I = np.meshgrid(np.arange(n), np.arange(1, n), indexing="ij")
    fx = ((I - 1) + (n - 1) * J).ravel()
    pR, pL = (nu + I + n * J).ravel(), (nu + (I - 1) + n * J).ravel()
    J, I = np.meshgrid(np.arange(1, n), np.arange(n), indexing="ij")
    fy = (nux + I + n * (J - 1)).ravel()
    pT, pB = (nu + I + n * J).ravel(), (nu + I + n * (J - 1)).ravel()
    br = np.concatenate([fx, fx, fy, fy])
    bc = np.concatenate([pR, pL, pT, pB])
    bv = np.concatenate([np.full(fx.size, h), np.full(fx.size, -h), np.full(fy.size, h), np.full(fy.size, -h)])

    K = _csr_from_coo(kr, kc, kv, nu)
    Bt = _csr_from_coo(br, bc, bv, N)                        # N x N, velocity rows only
    full = _csr_from_coo(np.concatenate([kr, br, bc]), np.concatenate([kc, bc, br]),
                         np.concatenate([kv, bv, bv]), N)    # [K B^T; B 0]

    b = np.zeros(N)
    J, I = np.meshgrid(np.arange(1, n), np.arange(n), indexing="ij")
    m = inside[J - 1, I] & inside[J, I]
    b[(nux + I + n * (J - 1))[m]] = -h * h * drho
    schur = -(h * h) / eta.reshape(-1)
    return dict(n=n, h=h, N=N, nu=nu, npr=npr, eta=eta, K=K, Bt=Bt, A=full, b=b, schur_diag=schur)
