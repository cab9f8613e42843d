"""Pins for the oracle's operators and preconditioners (CPU only).

Each check compares the oracle with something fixed independently of its own
code: textbook matrices, an energy identity with series conductances, closed
forms of the upwind difference and of Chebyshev error polynomials, Krylov
minimisation by brute force, and a library BF16 conversion.
"""
import numpy as np
import pytest

import workloads as W
from oracle import operators as O
from oracle import preconditioners as PC


def _t1d(n):
    t = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    t[0, 0] = t[-1, -1] = 3.0       # boundary face 2*eta plus one interior face
    return t


def test_constant_coefficient_2d_is_kronecker_laplacian():
    nx, ny = 5, 4
    op = O.StencilOperator((nx, ny, 1), np.ones(nx * ny))
    a = op.to_dense()
    ref = np.kron(np.eye(ny), _t1d(nx)) + np.kron(_t1d(ny), np.eye(nx))
    assert np.array_equal(a, ref)


def test_constant_coefficient_3d_is_kronecker_laplacian():
    nx, ny, nz = 4, 3, 5
    op = O.StencilOperator((nx, ny, nz), 2.5 * np.ones(nx * ny * nz))
    a = op.to_dense()
    ix, iy, iz = np.eye(nx), np.eye(ny), np.eye(nz)
    ref = (np.kron(iz, np.kron(iy, _t1d(nx))) + np.kron(iz, np.kron(_t1d(ny), ix))
           + np.kron(_t1d(nz), np.kron(iy, ix)))
    assert np.allclose(a, 2.5 * ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("dims", [(6, 5, 1), (4, 3, 5)])
def test_energy_identity_series_conductance(dims):
    """u^T A u = sum_faces (u_i-u_j)^2 / (1/(2 eta_i) + 1/(2 eta_j)) + sum_bfaces 2 eta_i u_i^2."""
    nx, ny, nz = dims
    g = W.rng(900, 1)
    eta = 10.0 ** g.uniform(-3, 3, size=nx * ny * nz)
    op = O.StencilOperator(dims, eta)
    u = g.standard_normal(nx * ny * nz)
    shape = (nz, ny, nx)
    e = eta.reshape(shape)
    uu = u.reshape(shape)
    energy = 0.0
    for ax in range(3):
        n = shape[ax]
        if n == 1 and ax == 0:
            continue
        for k in range(n):
            sl = [slice(None)] * 3
            sl[ax] = k
            if k + 1 < n:
                sl2 = list(sl)
                sl2[ax] = k + 1
                c = 1.0 / (1.0 / (2 * e[tuple(sl)]) + 1.0 / (2 * e[tuple(sl2)]))
                energy += np.sum(c * (uu[tuple(sl)] - uu[tuple(sl2)]) ** 2)
            if k == 0 or k == n - 1:
                mult = 2 if n == 1 else 1
                energy += mult * np.sum(2 * e[tuple(sl)] * uu[tuple(sl)] ** 2)
    assert np.isclose(u @ op.apply(u), energy, rtol=1e-12)
    a = op.to_dense()
    assert np.allclose(a, a.T, rtol=0, atol=1e-12 * np.abs(a).max())


def test_upwind_advection_closed_form():
    """Pure upwind part A(v) - A(0) on linear functions, one velocity component at a time."""
    nx, ny, nz = 7, 4, 3
    eta = W.rng(900, 2).uniform(1, 2, size=nx * ny * nz)
    a_dif = O.StencilOperator((nx, ny, nz), eta)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    h = 1.0 / nx
    # v_x = 3 > 0, u = x index: h v_x (u_i - u_{i-1}) = h v_x inside, 0 at i = 0 (u_0 = 0, ghost 0)
    a_adv = O.StencilOperator((nx, ny, nz), eta, (3.0, 0.0, 0.0))
    d = (a_adv.apply(i.astype(float).reshape(-1)) - a_dif.apply(i.astype(float).reshape(-1)))
    assert np.allclose(d.reshape(nz, ny, nx), np.where(i == 0, 0.0, h * 3.0), atol=1e-13)
    # v_y = -2 < 0, u = y index: upwind at +y: -h|v_y| inside, h|v_y| (ny-1) against the ghost
    a_adv = O.StencilOperator((nx, ny, nz), eta, (0.0, -2.0, 0.0))
    d = (a_adv.apply(j.astype(float).reshape(-1)) - a_dif.apply(j.astype(float).reshape(-1)))
    assert np.allclose(d.reshape(nz, ny, nx), np.where(j == ny - 1, h * 2.0 * (ny - 1), -h * 2.0),
                       atol=1e-13)
    # v_z = 0.5 > 0 on a constant: zero except the first layer, which sees the zero ghost
    a_adv = O.StencilOperator((nx, ny, nz), eta, (0.0, 0.0, 0.5))
    one = np.ones(nx * ny * nz)
    d = a_adv.apply(one) - a_dif.apply(one)
    assert np.allclose(d.reshape(nz, ny, nx), np.where(k == 0, h * 0.5, 0.0), atol=1e-13)


def test_csr_assembly_matches_dense_and_config1_nnz():
    for dims, vel in [((6, 5, 1), (0, 0, 0)), ((4, 3, 5), (1.0, -2.0, 3.0))]:
        eta = W.rng(900, 3).uniform(0.5, 5, size=int(np.prod(dims)))
        op = O.StencilOperator(dims, eta, vel)
        csr = op.to_csr()
        assert np.allclose(csr.to_dense(), op.to_dense(), rtol=0, atol=1e-13)
        x = W.random_vector(op.n, 7)
        assert np.allclose(csr.apply(x), op.apply(x), rtol=1e-13, atol=1e-13)
    c1 = W.poisson2d_inclusions()
    csr = O.StencilOperator(c1["dims"], c1["eta"]).to_csr()
    assert csr.n == 4096 and len(csr.vals) == 20224


def test_gershgorin_bound_covers_spectrum():
    dims = (6, 5, 4)
    eta = 10.0 ** W.rng(900, 4).uniform(-2, 2, size=120)
    op = O.StencilOperator(dims, eta)
    a = op.to_dense()
    d = np.diag(a)
    lam = np.linalg.eigvals(a / d[:, None]).real
    assert lam.max() <= op.gershgorin_jacobi_bound() + 1e-12
    assert op.gershgorin_jacobi_bound() <= 2.0 + 1e-12


def test_bf16_rounding_matches_library():
    torch = pytest.importorskip("torch")
    g = W.rng(900, 5)
    x = np.concatenate([g.standard_normal(20000).astype(np.float32) * 10.0 ** g.integers(-30, 30, 20000),
                        np.array([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8), 3.0e38, 1e-40],
                                 dtype=np.float32)]).astype(np.float32)
    ours = PC.bf16_round(x)
    lib = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(ours.view(np.uint32), lib.view(np.uint32))


def _hadamard(n):
    h = np.array([[1.0]])
    while h.shape[0] < n:
        h = np.block([[h, h], [h, -h]])
    return h / np.sqrt(n)


def test_chebyshev_error_polynomial_closed_form():
    """x_k = (I - P_k(D^-1 A)) A^-1 v with P_k(l) = T_k((theta-l)/delta) / T_k(theta/delta)."""
    n = 16
    q = _hadamard(n)
    lam = np.linspace(0.3, 1.7, n)                     # mean 1 -> diag(Q L Q^T) = 1
    g = W.rng(900, 6)
    dvec = 10.0 ** g.uniform(-1, 1, n)
    dh = np.sqrt(dvec)
    a = (dh[:, None] * (q * lam) @ q.T) * dh[None, :]
    assert np.allclose(np.diag(a), dvec)
    A = O.DenseOperator(a)
    v = g.standard_normal(n)
    lo, hi = 0.2, 1.9
    theta, delta = (hi + lo) / 2, (hi - lo) / 2
    vmat = q / dh[:, None]                              # eigenvectors of D^-1 A: D^-1/2 Q
    for k in (1, 2, 3, 6):
        cheb = PC.Chebyshev(A, k, lo=lo, hi=hi)
        ck = np.zeros(k + 1)
        ck[k] = 1.0
        pk = np.polynomial.chebyshev.chebval((theta - lam) / delta, ck) / \
            np.polynomial.chebyshev.chebval(theta / delta, ck)
        xstar = np.linalg.solve(a, v)
        coef = np.linalg.solve(vmat, xstar)
        exp = xstar - vmat @ (pk * coef)
        assert np.allclose(cheb(v), exp, rtol=1e-11, atol=1e-12 * np.abs(xstar).max())


def _krylov_basis(op_mat, v, k):
    """Orthonormal basis of span(v, M v, ..., M^{k-1} v) by repeated Gram-Schmidt."""
    vs = []
    w = v.copy()
    for _ in range(k):
        for _ in range(2):
            for b in vs:
                w = w - (b @ w) * b
        nrm = np.linalg.norm(w)
        vs.append(w / nrm)
        w = op_mat @ vs[-1]
    return np.column_stack(vs)


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_inner_pcg_is_a_norm_minimiser(k):
    """k steps of Jacobi-PCG from 0 minimise ||x - A^-1 v||_A over K_k(D^-1 A, D^-1 v)."""
    dims = (5, 4, 3)
    eta = 10.0 ** W.rng(900, 7).uniform(-1, 1, size=60)
    op = O.StencilOperator(dims, eta)
    a = op.to_dense()
    dinv = 1.0 / np.diag(a)
    v = W.random_vector(60, 8)
    V = _krylov_basis(dinv[:, None] * a, dinv * v, k)
    y = np.linalg.solve(V.T @ a @ V, V.T @ v)
    assert np.allclose(PC.InnerPCG(op, k)(v), V @ y, rtol=1e-9, atol=1e-12)


def test_inner_pcg_finite_termination_and_zero_guard():
    op = O.StencilOperator((3, 3, 1), W.rng(900, 9).uniform(1, 3, size=9))
    v = W.random_vector(9, 10)
    assert np.allclose(PC.InnerPCG(op, 9)(v), np.linalg.solve(op.to_dense(), v), rtol=1e-10)
    assert np.array_equal(PC.InnerPCG(op, 4)(np.zeros(9)), np.zeros(9))


def test_jacobi_and_noisy_pc():
    op = O.StencilOperator((4, 4, 1), W.rng(900, 11).uniform(1, 3, size=16))
    v = W.random_vector(16, 12)
    assert np.allclose(PC.JacobiPC(op)(v), v / np.diag(op.to_dense()))
    bank = W.noise_bank(16, 3)
    npc = PC.NoisyPC(1e-2, bank)
    out = npc(v)
    assert np.isclose(np.linalg.norm(out - v), 1e-2 * np.linalg.norm(v))
    assert np.allclose((out - v) / np.linalg.norm(out - v), bank[0] / np.linalg.norm(bank[0]))


_UNIT = {"fp32": 2.0 ** -24, "bf16": 2.0 ** -8}   # unit roundoff of the coefficient format


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_rounded_stencil_coefficients_and_error_bound(precision):
    """The preconditioner's reduced-precision operator copy: every stored
    coefficient is a number of the target format (rounding is idempotent)
    within its unit roundoff of the FP64 value; y = A~ u on an FP32 vector is
    within the bound of a 7-term FP32 sum plus the coefficient rounding of the
    FP64 product sum |a_ij| |u_j|, and (BF16) far enough from it that the
    coefficient rounding shows."""
    c = W.poisson3d_gaussian(dims=(7, 6, 5), log_contrast=2.0, config_id=900, item_id=31)
    op = O.StencilOperator(c["dims"], c["eta"], (1.5, -0.5, 0.8))
    rs = PC.RoundedStencil(op, precision)
    u = _UNIT[precision]
    d64 = op.diagonal().reshape(op.shape)
    for got, ref in [(rs.d, d64), (rs.dinv, 1.0 / d64)]:
        assert got.dtype == np.float32
        if precision == "bf16":
            assert np.array_equal(PC.bf16_round(got), got)
        assert np.all(np.abs(got.astype(np.float64) - ref) <= u * np.abs(ref))
    a = op.to_dense()
    x = W.random_vector(op.n, 32).astype(np.float32)
    y = rs.apply(x).astype(np.float64)
    scale = np.abs(a) @ np.abs(x.astype(np.float64))
    rel = np.abs(y - a @ x.astype(np.float64)) / scale
    assert rel.max() <= u + 8 * 2.0 ** -24, rel.max()
    if precision == "bf16":
        assert rel.max() >= 0.1 * u


def _cheb_closed_form(a, dinv, v, k, lo, hi):
    """x_k = (I - P_k(M)) A^-1 v, M = diag(dinv) A, from the eigenvectors of the
    symmetric diag(dinv)^1/2 A diag(dinv)^1/2."""
    theta, delta = (hi + lo) / 2, (hi - lo) / 2
    gh = np.sqrt(dinv)
    mu, q = np.linalg.eigh(gh[:, None] * a * gh[None, :])
    ck = np.zeros(k + 1)
    ck[k] = 1.0
    pk = np.polynomial.chebyshev.chebval((theta - mu) / delta, ck) / \
        np.polynomial.chebyshev.chebval(theta / delta, ck)
    xstar = np.linalg.solve(a, v)
    return xstar - (gh[:, None] * q) @ (pk * (q.T @ (xstar / gh))), xstar


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("k", [1, 3, 6])
def test_reduced_precision_chebyshev_closed_form(precision, k):
    """Constant eta (every face and diagonal coefficient an integer, exact in
    both formats): the reduced-precision Chebyshev sweeps give the closed-form
    error polynomial of M = D~^-1 A with D~^-1 the diagonal's inverse rounded to
    the format, to FP32 accuracy -- and (BF16) not that of the exact D^-1."""
    op = O.StencilOperator((6, 5, 4), np.ones(120))
    a = op.to_dense()
    d = np.diag(a)
    assert np.array_equal(d, np.round(d))
    dinv = (1.0 / d).astype(np.float32)
    if precision == "bf16":
        dinv = PC.bf16_round(dinv)
    v = W.random_vector(120, 21)
    lo, hi = 0.05, 2.0
    x = PC.Chebyshev(op, k, lo=lo, hi=hi, precision=precision)(v)
    assert np.array_equal(x, x.astype(np.float32).astype(np.float64))
    exp, xstar = _cheb_closed_form(a, dinv.astype(np.float64), v, k, lo, hi)
    assert np.linalg.norm(x - exp) <= 1e-6 * np.linalg.norm(xstar)
    if precision == "bf16":
        exact, _ = _cheb_closed_form(a, 1.0 / d, v, k, lo, hi)
        assert np.linalg.norm(x - exact) >= 1e-4 * np.linalg.norm(xstar)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("k", [1, 3])
def test_reduced_precision_inner_pcg_one_cell(precision, k):
    """One cell: Jacobi-PCG converges in one step to v / d~, d~ the diagonal as
    the preconditioner's copy stores it (the format's rounding of d), to FP32
    accuracy; the result is an FP32 number."""
    op = O.StencilOperator((1, 1, 1), np.array([2.7]))
    d = op.diagonal()[0]
    dr = np.float32(d)
    if precision == "bf16":
        dr = PC.bf16_round(np.array([dr]))[0]
    v = np.array([0.37])
    x = PC.InnerPCG(op, k, precision=precision)(v)
    assert x[0] == np.float64(np.float32(x[0]))
    assert abs(x[0] - 0.37 / float(dr)) <= 4 * 2.0 ** -24 * abs(x[0])
    if precision == "bf16":
        assert abs(x[0] - 0.37 / d) >= 1e-4 * abs(x[0])


@pytest.mark.parametrize("precision,tol", [("fp32", 3e-6), ("bf16", 2e-2)])
def test_reduced_precision_preconditioners_close_to_fp64(precision, tol):
    """On a variable-coefficient problem with advection the reduced-precision
    forms stay close to the FP64 ones (the pins above fix their rounding)."""
    c = W.poisson3d_gaussian(dims=(12, 10, 8), log_contrast=1.0, config_id=900, item_id=13)
    op = O.StencilOperator(c["dims"], c["eta"], (2.0, 1.0, -1.0))
    v = W.random_vector(op.n, 14)
    ref = PC.Chebyshev(op, 6)(v)
    got = PC.Chebyshev(op, 6, precision=precision)(v)
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)
    op2 = O.StencilOperator(c["dims"], c["eta"])
    ref = PC.InnerPCG(op2, 4)(v)
    got = PC.InnerPCG(op2, 4, precision=precision)(v)
    assert np.linalg.norm(got - ref) <= 10 * tol * np.linalg.norm(ref)
