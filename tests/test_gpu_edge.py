"""Edge and degenerate cases of the solve path on the GPU, each against what
the method or the oracle fixes: b = 0, one-cell and one-row grids, an exact
preconditioner (B = A^-1 gives one step with alpha_0 = 1), nu_max = 1 (IPCG,
Sec. 5 truncation remark), the largest window (nu_max = 32), a nonzero
initial guess, and argument errors that must leave the context usable."""
import numpy as np
import pytest

import workloads as W
from oracle import krylov as K
from oracle import operators as O
from oracle import preconditioners as PC
from tests._parity import check_solve, oracle_with_envelope

pytestmark = pytest.mark.gpu

ALL = ["fcg", "pipefcg", "gcr", "pipegcr", "pipegcr_w", "fgmres", "pipefgmres"]


@pytest.fixture(scope="module")
def ctx(lib):
    from paper_1511_07226_gb300 import pfk
    return pfk.Context(0)


@pytest.mark.parametrize("method", ALL)
def test_zero_rhs_returns_initial_guess(ctx, method):
    """b = 0 and x0 = 0: the initial residual is zero, so every method stops in
    its fill with x = 0 and no iteration."""
    from paper_1511_07226_gb300 import pfk
    c = W.poisson3d_gaussian(dims=(9, 7, 5), ell=2.0, config_id=2, item_id=30)
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"])
    pc = pfk.Preconditioner(ctx, op, "jacobi")
    x, info, _ = pfk.solve(ctx, op, pc, np.zeros(op.n), method=method, mmax=8, rtol=1e-8)
    assert info["status_name"] == "ok" and info["iterations"] == 0
    assert np.all(x == 0.0)


@pytest.mark.parametrize("dims", [(1, 1, 1), (1, 1), (37, 1, 1), (1, 29, 1), (1, 1, 41), (33, 1)])
@pytest.mark.parametrize("method", ["pipefcg", "pipegcr", "pipefgmres"])
def test_degenerate_grids(ctx, dims, method):
    """One cell, one row / column, one pillar: the stencil walk's edge lanes and
    the passes' ragged tails against the oracle."""
    from paper_1511_07226_gb300 import pfk
    n = int(np.prod(dims))
    g = W.rng(31, n)
    eta = np.power(10.0, g.uniform(-1.0, 1.0, size=n))
    b = g.uniform(-1.0, 1.0, size=n)
    aop = O.StencilOperator(dims, eta)
    prm = K.Params(mmax=8, rtol=1e-10, maxit=200)
    ref, alts = oracle_with_envelope(method, aop, lambda: PC.JacobiPC(aop), b, prm)
    op = pfk.Operator.stencil(ctx, dims, eta)
    x, info, hist = pfk.solve(ctx, op, pfk.Preconditioner(ctx, op, "jacobi"), b, method=method, mmax=8,
                              rtol=1e-10, maxit=200, history=400)
    check_solve(hist, info, ref, alts, rtol=1e-10, min_prefix=1)
    np.testing.assert_allclose(aop.apply(x), b, rtol=0, atol=1e-8 * np.linalg.norm(b))


@pytest.mark.parametrize("method", ["fcg", "pipefcg", "pipegcr", "pipegcr_w"])
def test_exact_preconditioner_one_step(ctx, method):
    """A diagonal operator with Jacobi is B = A^-1: the fill gives alpha_0 = 1 and
    the first iterate is the solution."""
    from paper_1511_07226_gb300 import pfk
    n = 500
    g = W.rng(32, 0)
    diag = g.uniform(1.0, 100.0, size=n)
    b = g.uniform(-1.0, 1.0, size=n)
    op = pfk.Operator.csr(ctx, np.arange(n + 1), np.arange(n), diag)
    x, info, hist = pfk.solve(ctx, op, pfk.Preconditioner(ctx, op, "jacobi"), b, method=method, mmax=4, rtol=1e-12,
                              history=10)
    assert info["status_name"] == "ok" and info["iterations"] == 1
    assert abs(hist[0, 3] - 1.0) <= 1e-14           # alpha_0
    np.testing.assert_allclose(x, b / diag, rtol=1e-14, atol=0)


def test_nu_max_one_is_ipcg(ctx):
    """nu_max = 1 (Sec. 5 remark: IPCG of Golub and Ye) against the oracle."""
    from paper_1511_07226_gb300 import pfk
    c = W.poisson3d_gaussian(dims=(14, 12, 10), ell=3.0, log_contrast=1.0, config_id=2, item_id=33)
    aop = O.StencilOperator(c["dims"], c["eta"])
    prm = K.Params(mmax=1, rtol=1e-8, maxit=800)
    ref, alts = oracle_with_envelope("pipefcg", aop, lambda: PC.InnerPCG(aop, 3), c["b"], prm)
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"])
    x, info, hist = pfk.solve(ctx, op, pfk.Preconditioner(ctx, op, "inner_pcg", 3), c["b"], method="pipefcg",
                              mmax=1, rtol=1e-8, maxit=800, history=2000)
    check_solve(hist, info, ref, alts, rtol=1e-8)


@pytest.mark.parametrize("method", ["pipefcg", "pipegcr", "fcg", "pipefgmres", "fgmres"])
def test_largest_window(ctx, method):
    """nu_max / restart length at its maximum (PFK_MAX_MMAX = 32): a full window
    occupies every lane of the transposed window dots and the widest
    reductions; against the oracle."""
    from paper_1511_07226_gb300 import pfk
    c = W.poisson3d_gaussian(dims=(18, 16, 13), ell=3.0, log_contrast=2.0, config_id=2, item_id=34)
    aop = O.StencilOperator(c["dims"], c["eta"])
    sigma = {"sigma": 1.5} if "gmres" in method else {}
    prm = K.Params(mmax=32, rtol=1e-9, maxit=600, **sigma)
    ref, alts = oracle_with_envelope(method, aop, lambda: PC.JacobiPC(aop), c["b"], prm)
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"])
    x, info, hist = pfk.solve(ctx, op, pfk.Preconditioner(ctx, op, "jacobi"), c["b"], method=method, mmax=32,
                              rtol=1e-9, maxit=600, history=4000, **sigma)
    assert ref.iterations > 40                  # the window fills and slides
    check_solve(hist, info, ref, alts, rtol=1e-9)


@pytest.mark.parametrize("method", ALL)
def test_nonzero_initial_guess(ctx, method):
    """x_0 != 0 for every method (r_0 = b - A x_0; FGMRES types update x_0 +
    U y at the cycle end), against the oracle from the same x_0."""
    from paper_1511_07226_gb300 import pfk
    c = W.poisson3d_gaussian(dims=(15, 13, 11), ell=3.0, log_contrast=1.5, config_id=2, item_id=35)
    aop = O.StencilOperator(c["dims"], c["eta"])
    x0 = W.random_vector(aop.n, 36)
    sigma = {"sigma": 1.5} if "gmres" in method else {}
    prm = K.Params(mmax=20, rtol=1e-8, maxit=600, **sigma)
    ref, alts = oracle_with_envelope(method, aop, lambda: PC.JacobiPC(aop), c["b"], prm, x0=x0)
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"])
    x, info, hist = pfk.solve(ctx, op, pfk.Preconditioner(ctx, op, "jacobi"), c["b"], x0=x0, method=method,
                              mmax=20, rtol=1e-8, maxit=600, history=4000, **sigma)
    check_solve(hist, info, ref, alts, rtol=1e-8)


def test_errors_leave_context_usable(ctx):
    from paper_1511_07226_gb300 import pfk
    c = W.poisson3d_gaussian(dims=(8, 8, 8), ell=2.0, config_id=2, item_id=34)
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"])
    with pytest.raises(pfk.PfkError):
        pfk.Operator.stencil(ctx, (0, 4, 4), np.ones(0))
    with pytest.raises(pfk.PfkError):
        pfk.solve(ctx, op, None, c["b"], method="pipefcg", mmax=0)
    with pytest.raises(pfk.PfkError):
        pfk.Preconditioner(ctx, op, "chebyshev", inner_iters=4, cheb_lo=2.0, cheb_hi=1.0)
    x, info, _ = pfk.solve(ctx, op, pfk.Preconditioner(ctx, op, "jacobi"), c["b"], method="pipefcg", mmax=8)
    assert info["status_name"] == "ok"
