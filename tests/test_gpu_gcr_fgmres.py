"""PIPEGCR (Alg. 11), PIPEGCR_w (Alg. 12) and PIPEFGMRES (Alg. 15) on the GPU
against the oracle, with the envelope protocol of tests/_parity.py."""
import numpy as np
import pytest

import workloads as W
from oracle import krylov as K
from oracle import operators as O
from oracle import preconditioners as PC
from tests._parity import check_solve, oracle_with_envelope

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    from paper_1511_07226_gb300 import pfk
    return pfk.Context(0)


def _problem(dims=(20, 18, 14), contrast=2.0, item=5, vel=(0.0, 0.0, 0.0)):
    c = W.poisson3d_gaussian(dims=dims, ell=4.0, log_contrast=contrast, config_id=2, item_id=item)
    return c, O.StencilOperator(c["dims"], c["eta"], vel)


@pytest.mark.parametrize("method", ["pipegcr", "pipegcr_w"])
@pytest.mark.parametrize("pc_kind", ["jacobi", "inner_pcg"])
@pytest.mark.parametrize("mmax,trunc,norm", [(30, "standard", "natural"), (5, "standard", "unpreconditioned"),
                                             (4, "restart", "natural")])
def test_pipegcr_stencil(ctx, method, pc_kind, mmax, trunc, norm):
    from paper_1511_07226_gb300 import pfk
    c, aop = _problem()
    mk = (lambda: PC.JacobiPC(aop)) if pc_kind == "jacobi" else (lambda: PC.InnerPCG(aop, 4))
    prm = K.Params(mmax=mmax, rtol=1e-8, truncation=trunc, norm=norm, maxit=600)
    ref, alts = oracle_with_envelope(method, aop, mk, c["b"], prm)
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"])
    pc = pfk.Preconditioner(ctx, op, pc_kind, inner_iters=4)
    x, info, hist = pfk.solve(ctx, op, pc, c["b"], method=method, mmax=mmax, truncation=trunc, norm=norm,
                              rtol=1e-8, maxit=600, history=4000)
    check_solve(hist, info, ref, alts, rtol=1e-8)


@pytest.mark.parametrize("method", ["pipegcr", "pipegcr_w"])
def test_pipegcr_csr_nonsymmetric(ctx, method):
    """CSR storage of an advective (nonsymmetric) stencil: the CR family needs no symmetry."""
    from paper_1511_07226_gb300 import pfk
    c, aop = _problem(dims=(24, 20, 10), contrast=1.0, item=6, vel=(20.0, -10.0, 5.0))
    csr = aop.to_csr()
    prm = K.Params(mmax=20, rtol=1e-8, norm="unpreconditioned", maxit=600)
    ref, alts = oracle_with_envelope(method, csr, lambda: PC.JacobiPC(csr), c["b"], prm)
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"], (20.0, -10.0, 5.0), storage="csr")
    x, info, hist = pfk.solve(ctx, op, pfk.Preconditioner(ctx, op, "jacobi"), c["b"], method=method, mmax=20,
                              norm="unpreconditioned", rtol=1e-8, maxit=600, history=4000)
    check_solve(hist, info, ref, alts, rtol=1e-8)


def test_pipegcr_w_first_iterations_match_pipegcr(ctx):
    """Alg. 11 and Alg. 12 differ only in how w_i is obtained (A tilde-u_i versus
    the recurrence w_{i-1} - alpha z_{i-1}): their first iterations agree up to
    rounding, on the GPU as in exact arithmetic."""
    from paper_1511_07226_gb300 import pfk
    c, aop = _problem(dims=(16, 14, 12), item=7)
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"])
    pc = pfk.Preconditioner(ctx, op, "jacobi")
    _, _, h11 = pfk.solve(ctx, op, pc, c["b"], method="pipegcr", mmax=10, rtol=1e-8, maxit=12, history=20)
    _, _, h12 = pfk.solve(ctx, op, pc, c["b"], method="pipegcr_w", mmax=10, rtol=1e-8, maxit=12, history=20)
    assert np.allclose(h12[:8, 0], h11[:8, 0], rtol=1e-9, atol=0.0)


@pytest.mark.parametrize("pc_kind,m,sigma", [("jacobi", 30, 1.5), ("inner_pcg", 10, 1.2), ("jacobi", 5, 1.0),
                                             ("inner_pcg", 30, float("nan"))])
def test_pipefgmres_stencil(ctx, pc_kind, m, sigma):
    from paper_1511_07226_gb300 import pfk
    c, aop = _problem(item=7)
    mk = (lambda: PC.JacobiPC(aop)) if pc_kind == "jacobi" else (lambda: PC.InnerPCG(aop, 4))
    prm = K.Params(mmax=m, rtol=1e-8, sigma=sigma, maxit=600)
    ref, alts = oracle_with_envelope("pipefgmres", aop, mk, c["b"], prm)
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"])
    pc = pfk.Preconditioner(ctx, op, pc_kind, inner_iters=4)
    x, info, hist = pfk.solve(ctx, op, pc, c["b"], method="pipefgmres", mmax=m, sigma=sigma, rtol=1e-8, maxit=600,
                              history=4000)
    check_solve(hist, info, ref, alts, rtol=1e-8)


def test_pipefgmres_advection_chebyshev(ctx):
    """Nonsymmetric upwind operator with a Chebyshev preconditioner (config 3 shape, small)."""
    from paper_1511_07226_gb300 import pfk
    c, aop = _problem(dims=(18, 16, 12), contrast=2.0, item=8, vel=(10.0, 10.0, 10.0))
    prm = K.Params(mmax=30, rtol=1e-8, sigma=1.0, maxit=600)
    ref, alts = oracle_with_envelope("pipefgmres", aop, lambda: PC.Chebyshev(aop, 8), c["b"], prm)
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"], (10.0, 10.0, 10.0))
    pc = pfk.Preconditioner(ctx, op, "chebyshev", inner_iters=8)
    x, info, hist = pfk.solve(ctx, op, pc, c["b"], method="pipefgmres", mmax=30, sigma=1.0, rtol=1e-8, maxit=600,
                              history=4000)
    check_solve(hist, info, ref, alts, rtol=1e-8)


def test_pipefgmres_maxit_mid_cycle_iterate(ctx):
    """maxit inside a cycle: x = x_0 + U y over the columns formed so far, as the oracle."""
    from paper_1511_07226_gb300 import pfk
    c, aop = _problem(item=9)
    prm = K.Params(mmax=30, rtol=1e-14, sigma=1.5, maxit=12)
    ref = K.solve("pipefgmres", aop, PC.JacobiPC(aop), c["b"], prm=prm)
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"])
    x, info, hist = pfk.solve(ctx, op, pfk.Preconditioner(ctx, op, "jacobi"), c["b"], method="pipefgmres",
                              mmax=30, sigma=1.5, rtol=1e-14, maxit=12, history=100)
    assert ref.status == "maxit" and info["status_name"] == "not_converged" and info["iterations"] == 12
    assert np.allclose(hist[:, 0], ref.rho(), rtol=1e-10, atol=0)
    assert np.linalg.norm(x - ref.x) <= 1e-10 * np.linalg.norm(ref.x)


def test_pipefgmres_breakdown_restarts(ctx):
    """A negative shift makes t = ||zbar||^2 - sum hbar^2 < 0 at some column: both sides
    detect it, solve the least-squares problem over the valid columns and restart.
    Near the breakdown t suffers cancellation, so values after it follow the
    rounding envelope rather than agreeing to 1e-10."""
    from paper_1511_07226_gb300 import pfk
    c, aop = _problem(dims=(10, 9, 8), item=10)
    prm = K.Params(mmax=30, rtol=1e-8, sigma=-50.0, maxit=300, max_restarts=5)
    ref, alts = oracle_with_envelope("pipefgmres", aop, lambda: PC.JacobiPC(aop), c["b"], prm)
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"])
    x, info, hist = pfk.solve(ctx, op, pfk.Preconditioner(ctx, op, "jacobi"), c["b"], method="pipefgmres",
                              mmax=30, sigma=-50.0, rtol=1e-8, maxit=300, max_restarts=5, history=1000)
    assert ref.breakdowns >= 1 and info["breakdowns"] >= 1
    # after a breakdown restart under this shift, whether the remaining
    # restarts end in convergence or in another breakdown depends on rounding
    # alone: the trajectory is checked against the envelope, the outcome for
    # validity
    check_solve(hist, info, ref, alts, min_prefix=1, check_status=False)
    assert info["status_name"] in ("ok", "breakdown")
    if info["status_name"] == "ok":
        assert info["rnorm_true"] <= 1e-8 * info["bnorm"] * (1 + 1e-12)


@pytest.mark.parametrize("method", ["fcg", "pipefcg", "gcr", "pipegcr", "pipegcr_w"])
def test_true_residual_stagnation_reported(ctx, method):
    """A goal below attainable accuracy ends, as in the oracle, with
    not-converged after max_restarts residual replacements, not with ok."""
    from paper_1511_07226_gb300 import pfk
    c = W.poisson2d_inclusions(16, 16)
    aop = O.StencilOperator(c["dims"], c["eta"])
    ref = K.solve(method, aop, PC.JacobiPC(aop), c["b"], prm=K.Params(mmax=10, rtol=1e-18, max_restarts=2,
                                                                      maxit=2000))
    assert ref.status == "stagnated"
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"])
    pc = pfk.Preconditioner(ctx, op, "jacobi")
    x, info, _ = pfk.solve(ctx, op, pc, c["b"], method=method, mmax=10, rtol=1e-18, max_restarts=2, maxit=2000)
    assert info["status_name"] == "not_converged"
    assert info["restarts"] == 2
    assert info["rnorm_true"] / info["bnorm"] < 1e-13
    assert "true residual" in info["message"]
