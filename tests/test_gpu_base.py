"""The non-pipelined comparison baselines on the GPU against the oracle:
FCG (Alg. 2), GCR (Alg. 9) and FGMRES (Alg. 13), envelope protocol."""
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


def _run(ctx, method, c, aop_for_oracle, mk, pc_kind, storage="matrix_free", vel=(0.0, 0.0, 0.0), **kw):
    from paper_1511_07226_gb300 import pfk
    prm = K.Params(**kw)
    ref, alts = oracle_with_envelope(method, aop_for_oracle, mk, c["b"], prm)
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"], vel, storage=storage)
    pc = pfk.Preconditioner(ctx, op, pc_kind, inner_iters=4)
    x, info, hist = pfk.solve(ctx, op, pc, c["b"], method=method, history=5000,
                              **{k: v for k, v in kw.items() if k in ("mmax", "rtol", "truncation", "norm",
                                                                      "maxit", "sigma")})
    return check_solve(hist, info, ref, alts, rtol=kw.get("rtol"))


def test_fcg_config1_csr_jacobi(ctx):
    c = W.poisson2d_inclusions()
    aop = O.StencilOperator(c["dims"], c["eta"]).to_csr()
    _run(ctx, "fcg", c, aop, lambda: PC.JacobiPC(aop), "jacobi", storage="csr", mmax=30, rtol=1e-8)


@pytest.mark.parametrize("mmax,trunc", [(30, "standard"), (5, "restart")])
def test_fcg_3d_inner_pcg(ctx, mmax, trunc):
    c = W.poisson3d_gaussian(dims=(20, 18, 14), ell=4.0, log_contrast=2.0, config_id=2, item_id=5)
    aop = O.StencilOperator(c["dims"], c["eta"])
    _run(ctx, "fcg", c, aop, lambda: PC.InnerPCG(aop, 4), "inner_pcg", mmax=mmax, truncation=trunc, rtol=1e-8,
         maxit=500)


@pytest.mark.parametrize("norm", ["natural", "unpreconditioned"])
def test_gcr_3d(ctx, norm):
    c = W.poisson3d_gaussian(dims=(20, 18, 14), ell=4.0, log_contrast=2.0, config_id=2, item_id=6)
    aop = O.StencilOperator(c["dims"], c["eta"])
    _run(ctx, "gcr", c, aop, lambda: PC.InnerPCG(aop, 4), "inner_pcg", mmax=30, norm=norm, rtol=1e-8, maxit=500)


def test_gcr_nonsymmetric_csr(ctx):
    vel = (20.0, -10.0, 5.0)
    c = W.poisson3d_gaussian(dims=(24, 20, 10), ell=4.0, log_contrast=1.0, config_id=2, item_id=7)
    aop = O.StencilOperator(c["dims"], c["eta"], vel).to_csr()
    _run(ctx, "gcr", c, aop, lambda: PC.JacobiPC(aop), "jacobi", storage="csr", vel=vel, mmax=20,
         norm="unpreconditioned", rtol=1e-8, maxit=500)


@pytest.mark.parametrize("m,pc_kind", [(30, "jacobi"), (10, "inner_pcg"), (4, "jacobi")])
def test_fgmres(ctx, m, pc_kind):
    c = W.poisson3d_gaussian(dims=(20, 18, 14), ell=4.0, log_contrast=2.0, config_id=2, item_id=8)
    aop = O.StencilOperator(c["dims"], c["eta"], (5.0, 0.0, 0.0))
    mk = (lambda: PC.JacobiPC(aop)) if pc_kind == "jacobi" else (lambda: PC.InnerPCG(aop, 4))
    _run(ctx, "fgmres", c, aop, mk, pc_kind, vel=(5.0, 0.0, 0.0), mmax=m, rtol=1e-8, maxit=800)


def test_fgmres_nonsymmetric_csr(ctx):
    """FGMRES on an assembled (CSR) advection operator: the row-per-thread
    operator path of the base methods."""
    vel = (10.0, -5.0, 2.0)
    c = W.poisson3d_gaussian(dims=(18, 16, 12), ell=4.0, log_contrast=1.5, config_id=2, item_id=9)
    aop = O.StencilOperator(c["dims"], c["eta"], vel).to_csr()
    _run(ctx, "fgmres", c, aop, lambda: PC.JacobiPC(aop), "jacobi", storage="csr", vel=vel, mmax=20,
         rtol=1e-8, maxit=800)
