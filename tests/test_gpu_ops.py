"""GPU parity of the operator and preconditioner kernels against the oracle.

Sizes span several thread blocks and end in ragged tails (no dimension is a
multiple of a warp or block)."""
import numpy as np
import pytest

import workloads as W
from oracle import operators as O
from oracle import preconditioners as PC

pytestmark = pytest.mark.gpu

CASES = [((37, 29, 1), (0.0, 0.0, 0.0)), ((19, 13, 11), (0.0, 0.0, 0.0)), ((23, 17, 9), (3.0, -2.0, 1.5)),
         ((1, 1, 1), (0.0, 0.0, 0.0)), ((5, 1, 1), (0.0, 0.0, 0.0)), ((64, 48, 40), (0.0, 0.0, 0.0))]


@pytest.fixture(scope="module")
def ctx(lib):
    from paper_1511_07226_gb300 import pfk
    return pfk.Context(0)


def _problem(dims, item):
    n = int(np.prod(dims))
    g = W.rng(950, item)
    eta = 10.0 ** g.uniform(-3, 3, size=n)
    return eta, g.standard_normal(n)


@pytest.mark.parametrize("dims,vel", CASES)
def test_stencil_apply(ctx, dims, vel):
    from paper_1511_07226_gb300 import pfk
    eta, x = _problem(dims, 1)
    ref = O.StencilOperator(dims, eta, vel).apply(x)
    op = pfk.Operator.stencil(ctx, dims, eta, vel)
    got = op.apply(x).cpu().numpy()
    scale = np.abs(ref).max()
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-14 * scale)


@pytest.mark.parametrize("dims,vel", CASES[:4])
def test_stencil_as_csr_apply(ctx, dims, vel):
    from paper_1511_07226_gb300 import pfk
    eta, x = _problem(dims, 2)
    ref = O.StencilOperator(dims, eta, vel).apply(x)
    op = pfk.Operator.stencil(ctx, dims, eta, vel, storage="csr")
    got = op.apply(x).cpu().numpy()
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-14 * np.abs(ref).max())


def test_general_csr_apply(ctx):
    from paper_1511_07226_gb300 import pfk
    rp, ci, va = W.random_csr(3001, per_row=9, item_id=3)
    x = W.random_vector(3001, 4)
    ref = O.CsrOperator(rp, ci, va).apply(x)
    got = pfk.Operator.csr(ctx, rp, ci, va).apply(x).cpu().numpy()
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-14 * np.abs(ref).max())


@pytest.mark.parametrize("dims,vel", [CASES[1], CASES[2], CASES[0]])
def test_jacobi(ctx, dims, vel):
    from paper_1511_07226_gb300 import pfk
    eta, v = _problem(dims, 5)
    aop = O.StencilOperator(dims, eta, vel)
    op = pfk.Operator.stencil(ctx, dims, eta, vel)
    got = pfk.Preconditioner(ctx, op, "jacobi").apply(v).cpu().numpy()
    assert np.allclose(got, PC.JacobiPC(aop)(v), rtol=1e-15, atol=0)


@pytest.mark.parametrize("k", [1, 2, 4, 5])
@pytest.mark.parametrize("dims", [(37, 29, 1), (19, 13, 11)])
def test_inner_pcg_fp64(ctx, dims, k):
    from paper_1511_07226_gb300 import pfk
    eta, v = _problem(dims, 6)
    aop = O.StencilOperator(dims, eta)
    op = pfk.Operator.stencil(ctx, dims, eta)
    pc = pfk.Preconditioner(ctx, op, "inner_pcg", inner_iters=k)
    ref = PC.InnerPCG(aop, k)(v)
    got = pc.apply(v).cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    # a second application reuses the control block: same result bit for bit
    assert np.array_equal(pc.apply(v).cpu().numpy(), got)


def test_inner_pcg_zero_input(ctx):
    from paper_1511_07226_gb300 import pfk
    dims = (19, 13, 11)
    eta, _ = _problem(dims, 7)
    op = pfk.Operator.stencil(ctx, dims, eta)
    pc = pfk.Preconditioner(ctx, op, "inner_pcg", inner_iters=4)
    assert np.array_equal(pc.apply(np.zeros(op.n)).cpu().numpy(), np.zeros(op.n))


@pytest.mark.parametrize("dims", [(23, 17, 9), (40, 17, 9), (32, 8, 2), (64, 24, 37)])
@pytest.mark.parametrize("precision,tol", [("fp32", 2e-5), ("bf16", 2e-5)])
def test_reduced_precision_pc_vs_emulation(ctx, precision, tol, dims):
    """The GPU's FP32 / BF16-coefficient kernels against the oracle's emulation
    of the same storage rules (the paper defines no reduced-precision
    arithmetic; the emulation is pinned in tests/test_oracle_operators.py;
    the FP32 rounding order differs, hence the tolerance).  x extents that are multiples of 8
    take the TMA-pipelined walk, the others the register walk."""
    from paper_1511_07226_gb300 import pfk
    eta, v = _problem(dims, 8)
    vel = (2.0, 1.0, -1.0)
    aop = O.StencilOperator(dims, eta, vel)
    op = pfk.Operator.stencil(ctx, dims, eta, vel)
    ref = PC.Chebyshev(aop, 6, precision=precision)(v)
    got = pfk.Preconditioner(ctx, op, "chebyshev", inner_iters=6, precision=precision).apply(v).cpu().numpy()
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)
    if precision == "fp32":
        aop2 = O.StencilOperator(dims, eta)
        op2 = pfk.Operator.stencil(ctx, dims, eta)
        ref = PC.InnerPCG(aop2, 4, precision="fp32")(v)
        got = pfk.Preconditioner(ctx, op2, "inner_pcg", inner_iters=4, precision="fp32").apply(v).cpu().numpy()
        assert np.linalg.norm(got - ref) <= 50 * tol * np.linalg.norm(ref)


@pytest.mark.parametrize("k", [1, 3, 8])
def test_chebyshev_fp64(ctx, k):
    from paper_1511_07226_gb300 import pfk
    dims = (23, 17, 9)
    eta, v = _problem(dims, 9)
    vel = (2.0, 1.0, -1.0)
    aop = O.StencilOperator(dims, eta, vel)
    op = pfk.Operator.stencil(ctx, dims, eta, vel)
    ref = PC.Chebyshev(aop, k)(v)
    got = pfk.Preconditioner(ctx, op, "chebyshev", inner_iters=k).apply(v).cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
