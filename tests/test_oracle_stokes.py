"""Pins of the Stokes-like saddle-point inputs (workloads/stokes.py) and of the
oracle's block upper-triangular preconditioner (Sec. 6, ex43 nesting).

The discretisation is checked against what the mathematics fixes: symmetry of
[K B^T; B 0], K symmetric positive definite, the constant-viscosity K_x as a
Kronecker sum of 1-D Dirichlet Laplacians, div(curl psi) = 0 and grad(const) =
0 on the MAC grid.  The preconditioner is checked as the block triangular
solve it defines, and the nested solve against a dense solution."""
import numpy as np
import pytest

from oracle import krylov as K
from oracle import operators as O
from oracle import preconditioners as PC
from workloads import stokes as S


def _dense(csr, ncols=None):
    rp, ci, va = csr
    n = len(rp) - 1
    a = np.zeros((n, ncols or n))
    for r in range(n):
        for p in range(rp[r], rp[r + 1]):
            a[r, ci[p]] += va[p]
    return a


@pytest.fixture(scope="module")
def small():
    return S.stokes2d(n=8, item_id=1)


def test_saddle_matrix_symmetric_and_k_spd(small):
    a = _dense(small["A"])
    assert np.allclose(a, a.T, rtol=0, atol=1e-15)
    k = _dense(small["K"])
    assert np.allclose(k, k.T, rtol=0, atol=1e-15)
    assert np.linalg.eigvalsh(k).min() > 0.0
    nu = small["nu"]
    assert np.array_equal(a[:nu, :nu], k)
    assert np.all(a[nu:, nu:] == 0.0)


def test_constant_viscosity_kx_is_kronecker_sum():
    n = 6
    d = S.stokes2d(n=n, contrast=1.0)
    k = _dense(d["K"])
    nux = (n - 1) * n
    tx = 2 * np.eye(n - 1) - np.eye(n - 1, k=1) - np.eye(n - 1, k=-1)       # faces on walls are u = 0
    ty = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    ty[0, 0] = ty[-1, -1] = 3.0                                            # ghost -u half a cell away
    kx = np.kron(np.eye(n), tx) + np.kron(ty, np.eye(n - 1))
    assert np.allclose(k[:nux, :nux], kx, rtol=0, atol=1e-14)


def test_div_curl_and_grad_const_vanish(small):
    n, h, nu = small["n"], small["h"], small["nu"]
    nux = (n - 1) * n
    g = np.random.default_rng(5)
    psi = np.zeros((n + 1, n + 1))                      # stream function on nodes [J, I], zero on walls
    psi[1:n, 1:n] = g.standard_normal((n - 1, n - 1))
    u = np.zeros(small["N"])
    for j in range(n):
        for i in range(1, n):
            u[(i - 1) + (n - 1) * j] = (psi[j + 1, i] - psi[j, i]) / h          # u_x = d psi / dy
    for j in range(1, n):
        for i in range(n):
            u[nux + i + n * (j - 1)] = -(psi[j, i + 1] - psi[j, i]) / h         # u_y = -d psi / dx
    a = _dense(small["A"])
    div = a[nu:, :] @ u
    assert np.abs(div).max() <= 1e-13 * np.abs(u).max()
    p = np.zeros(small["N"])
    p[nu:] = 1.0
    assert np.abs(a[:nu, :] @ p).max() <= 1e-15


def test_block_upper_pc_is_the_block_triangular_solve(small):
    nu = small["nu"]
    Kop = O.CsrOperator(*small["K"])
    Bt = O.CsrOperator(*small["Bt"])
    B = PC.BlockUpperPC(Kop, Bt, small["schur_diag"], nu, inner_method="pipefcg", inner_mmax=30,
                        inner_rtol=1e-14, inner_maxit=500)
    v = np.random.default_rng(6).standard_normal(small["N"])
    y = B(v)
    k = _dense(small["K"])
    bt = _dense(small["Bt"])[:nu, nu:]
    assert np.allclose(small["schur_diag"] * y[nu:], v[nu:], rtol=1e-14, atol=0)
    res = k @ y[:nu] + bt @ y[nu:] - v[:nu]
    assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(v[:nu])
    # a wrong sign of the B^T term or of the Schur block breaks the identity
    assert np.linalg.norm(k @ y[:nu] - bt @ y[nu:] - v[:nu]) > 1e-3 * np.linalg.norm(v[:nu])


@pytest.mark.parametrize("outer", ["fgmres", "pipefgmres"])
@pytest.mark.parametrize("inner", ["fcg", "pipefcg", "pipegcr"])
def test_nested_solve_matches_dense_solution(outer, inner):
    d = S.stokes2d(n=12, item_id=2)
    nu, N = d["nu"], d["N"]
    A = O.CsrOperator(*d["A"])
    B = PC.BlockUpperPC(O.CsrOperator(*d["K"]), O.CsrOperator(*d["Bt"]), d["schur_diag"], nu,
                        inner_method=inner, inner_rtol=1e-4, inner_maxit=100)
    r = K.solve(outer, A, B, d["b"], prm=K.Params(mmax=30, rtol=1e-8, norm="unpreconditioned", sigma=1.0,
                                                  maxit=300))
    assert r.status == "converged"
    a = _dense(d["A"])
    x = np.linalg.lstsq(a, d["b"], rcond=None)[0]     # minimum-norm solution (pressure mean 0)
    u_ref, u = x[:nu], r.x[:nu]
    assert np.linalg.norm(u - u_ref) <= 1e-6 * np.linalg.norm(u_ref)
    p_ref, p = x[nu:] - x[nu:].mean(), r.x[nu:] - r.x[nu:].mean()
    assert np.linalg.norm(p - p_ref) <= 1e-5 * np.linalg.norm(p_ref)
    assert max(B.inner_iterations) <= 100


def _loop_assembly(n, contrast=25.0, item_id=0):
    """Entry-by-entry statement of the discretisation (reference for the
    vectorised generator): [K B^T; B 0] as a dense matrix."""
    h = 1.0 / n
    eta, _ = S.sinker_viscosity(n, contrast, item_id=item_id)
    nux = (n - 1) * n
    nu = nux + n * (n - 1)
    N = nu + n * n
    a = np.zeros((N, N))
    ux = lambda i, j: (i - 1) + (n - 1) * j
    uy = lambda i, j: nux + i + n * (j - 1)
    pc = lambda i, j: nu + i + n * j
    node = lambda i, j: 0.25 * (eta[j - 1, i - 1] + eta[j - 1, i] + eta[j, i - 1] + eta[j, i])
    for j in range(n):
        for i in range(1, n):
            r = ux(i, j)
            for ii, ec in ((i - 1, eta[j, i - 1]), (i + 1, eta[j, i])):
                a[r, r] += ec
                if 1 <= ii <= n - 1:
                    a[r, ux(ii, j)] -= ec
            for jj in (j - 1, j + 1):
                if 0 <= jj <= n - 1:
                    en = node(i, max(j, jj))
                    a[r, r] += en
                    a[r, ux(i, jj)] -= en
                else:
                    a[r, r] += eta[j, i - 1] + eta[j, i]
            a[r, pc(i, j)] += h
            a[r, pc(i - 1, j)] -= h
    for j in range(1, n):
        for i in range(n):
            r = uy(i, j)
            for jj, ec in ((j - 1, eta[j - 1, i]), (j + 1, eta[j, i])):
                a[r, r] += ec
                if 1 <= jj <= n - 1:
                    a[r, uy(i, jj)] -= ec
            for ii in (i - 1, i + 1):
                if 0 <= ii <= n - 1:
                    en = node(max(i, ii), j)
                    a[r, r] += en
                    a[r, uy(ii, j)] -= en
                else:
                    a[r, r] += eta[j - 1, i] + eta[j, i]
            a[r, pc(i, j)] += h
            a[r, pc(i, j - 1)] -= h
    a[nu:, :nu] = a[:nu, nu:].T
    return a


@pytest.mark.parametrize("n,item", [(5, 0), (8, 3), (11, 4)])
def test_vectorised_assembly_equals_entrywise_statement(n, item):
    d = S.stokes2d(n=n, item_id=item)
    assert np.allclose(_dense(d["A"]), _loop_assembly(n, item_id=item), rtol=0, atol=1e-15)
