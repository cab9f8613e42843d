"""The persistent single-launch path (many PIPEFCG / FCG iterations per
cooperative launch, blocks meeting at bounded grid barriers) against the
oracle, with the protocol of tests/_parity.py: the 64 x 64 inclusion problem
assembled as CSR with Jacobi (the latency-bound workload), window and
truncation variants, ragged and edge sizes (1 unknown, sizes that are not a
multiple of the 32-row chunk, the largest eligible size with several chunks
per block), the identity preconditioner, the unpreconditioned norm with maxit,
and the breakdown restarts of an indefinite system.  The graph path (one
kernel per step) is checked on the same problem for comparison."""
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


def _csr_problem(dims, item=0):
    if dims == (64, 64):
        c = W.poisson2d_inclusions()
    else:
        c = W.poisson2d_inclusions(nx=dims[0], ny=dims[1], n_incl=3, item_id=item)
    return c, O.StencilOperator(c["dims"], c["eta"]).to_csr()


@pytest.mark.parametrize("method", ["pipefcg", "fcg"])
@pytest.mark.parametrize("mode", ["on", "off"])
def test_config1_persistent_and_graph(ctx, method, mode):
    """64 x 64 with 8 inclusions of 1e3, FP64 CSR, Jacobi, nu_max = 30, rtol 1e-8."""
    from paper_1511_07226_gb300 import pfk
    c, aop = _csr_problem((64, 64))
    prm = K.Params(mmax=30, rtol=1e-8)
    ref, alts = oracle_with_envelope(method, aop, lambda: PC.JacobiPC(aop), c["b"], prm)
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"], storage="csr")
    pc = pfk.Preconditioner(ctx, op, "jacobi")
    x, info, hist = pfk.solve(ctx, op, pc, c["b"], method=method, mmax=30, rtol=1e-8, history=4000,
                              persistent=mode)
    s = check_solve(hist, info, ref, alts, rtol=1e-8, check_restarts=True)
    assert s["prefix"] >= 30, s
    if mode == "on":
        # one cooperative launch runs up to 16 iterations
        assert info["kernel_launches"] < info["iterations"], info


@pytest.mark.parametrize("method", ["pipefcg", "fcg"])
@pytest.mark.parametrize("mmax,trunc", [(1, "standard"), (4, "standard"), (5, "restart"), (16, "standard")])
def test_windows_and_truncation(ctx, method, mmax, trunc):
    from paper_1511_07226_gb300 import pfk
    c, aop = _csr_problem((40, 33), item=3)
    prm = K.Params(mmax=mmax, rtol=1e-8, truncation=trunc, maxit=3000)
    ref, alts = oracle_with_envelope(method, aop, lambda: PC.JacobiPC(aop), c["b"], prm)
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"], storage="csr")
    x, info, hist = pfk.solve(ctx, op, pfk.Preconditioner(ctx, op, "jacobi"), c["b"], method=method, mmax=mmax,
                              truncation=trunc, rtol=1e-8, maxit=3000, history=4000, persistent="on")
    check_solve(hist, info, ref, alts, rtol=1e-8)


@pytest.mark.parametrize("dims", [(1, 1), (7, 5), (37, 29), (128, 128)])
@pytest.mark.parametrize("method", ["pipefcg", "fcg"])
def test_ragged_and_largest_sizes(ctx, dims, method):
    """1 unknown; 35 and 1073 unknowns (ragged last chunk); 16384 unknowns (the
    largest eligible size: several 32-row chunks per block)."""
    from paper_1511_07226_gb300 import pfk
    c, aop = _csr_problem(dims, item=4)
    maxit = 300 if dims == (128, 128) else 3000
    prm = K.Params(mmax=30, rtol=1e-8, maxit=maxit)
    ref, alts = oracle_with_envelope(method, aop, lambda: PC.JacobiPC(aop), c["b"], prm)
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"], storage="csr")
    x, info, hist = pfk.solve(ctx, op, pfk.Preconditioner(ctx, op, "jacobi"), c["b"], method=method, mmax=30,
                              rtol=1e-8, maxit=maxit, history=4000, persistent="on")
    # one unknown: the second rho is exactly 0 (relative differences undefined)
    check_solve(hist, info, ref, alts, rtol=1e-8, min_prefix=1 if dims == (1, 1) else 3)
    if dims == (1, 1):
        assert info["iterations"] <= 1 and np.allclose(x, c["b"] / aop.diagonal())


def test_too_large_rejected_when_required(ctx):
    from paper_1511_07226_gb300 import pfk
    c, _ = _csr_problem((129, 128), item=5)
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"], storage="csr")
    with pytest.raises(pfk.PfkError, match="persistent"):
        pfk.solve(ctx, op, pfk.Preconditioner(ctx, op, "jacobi"), c["b"], persistent="on")
    # a matrix-free stencil is not eligible either; auto falls back to the graph path
    op2 = pfk.Operator.stencil(ctx, (16, 16, 1), np.ones(256))
    with pytest.raises(pfk.PfkError, match="persistent"):
        pfk.solve(ctx, op2, None, np.ones(256), persistent="on")
    x, info, _ = pfk.solve(ctx, op2, None, np.ones(256), persistent="auto")
    assert info["status_name"] == "ok"


def test_identity_pc_unpreconditioned_norm_maxit(ctx):
    from paper_1511_07226_gb300 import pfk
    c, aop = _csr_problem((64, 64))
    prm = K.Params(mmax=30, rtol=1e-12, norm="unpreconditioned", maxit=40)
    ref, alts = oracle_with_envelope("pipefcg", aop, lambda: PC.IdentityPC(), c["b"], prm)
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"], storage="csr")
    x, info, hist = pfk.solve(ctx, op, None, c["b"], mmax=30, rtol=1e-12, norm="unpreconditioned", maxit=40,
                              history=100, persistent="on")
    assert ref.status == "maxit" and info["status_name"] == "not_converged" and info["iterations"] == 40
    s = check_solve(hist, info, ref, alts)
    assert s["prefix"] >= 20


@pytest.mark.parametrize("method", ["pipefcg", "fcg"])
def test_breakdown_restarts(ctx, method):
    """Indefinite system: eta_i <= 0 restarts from x_i, then PFK_ERR_BREAKDOWN (Sec. 5)."""
    from paper_1511_07226_gb300 import pfk
    a = W.random_spd(30, cond=10.0, item_id=17)
    b = W.random_vector(30, 17)
    d = np.linalg.eigvalsh(a)
    sh = a - (d[0] + 0.5 * (d[1] - d[0])) * np.eye(30)
    rp = np.arange(0, 31 * 30, 30, dtype=np.int32)
    ci = np.tile(np.arange(30, dtype=np.int32), 30)
    ref = K.solve(method, O.DenseOperator(sh), PC.IdentityPC(), b, prm=K.Params(rtol=1e-8, mmax=30, max_restarts=3))
    op = pfk.Operator.csr(ctx, rp, ci, sh.reshape(-1))
    x, info, hist = pfk.solve(ctx, op, None, b, method=method, mmax=30, rtol=1e-8, max_restarts=3, history=200,
                              persistent="on")
    assert ref.status == "breakdown" and info["status_name"] == "breakdown"
    assert info["breakdowns"] == ref.breakdowns and info["restarts"] == ref.restarts


@pytest.mark.parametrize("method", ["pipefcg", "fcg"])
def test_bitwise_reproducible(ctx, method):
    from paper_1511_07226_gb300 import pfk
    c, _ = _csr_problem((64, 64))
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"], storage="csr")
    pc = pfk.Preconditioner(ctx, op, "jacobi")
    kw = dict(method=method, history=2000, persistent="on")
    x1, i1, h1 = pfk.solve(ctx, op, pc, c["b"], **kw)
    x2, i2, h2 = pfk.solve(ctx, op, pc, c["b"], **kw)
    x3, i3, h3 = pfk.solve(ctx, op, pc, c["b"], graph_iters=1, **kw)
    assert np.array_equal(x1, x2) and np.array_equal(h1, h2, equal_nan=True)
    assert np.array_equal(x1, x3) and i3["iterations"] == i1["iterations"]
    assert i1["status_name"] == "ok"


@pytest.mark.parametrize("method", ["pipefcg", "fcg"])
def test_general_csr_jacobi_nonzero_initial_guess(ctx, method):
    """A general CSR operator (random, diagonally dominant, symmetrised) with
    Jacobi and a nonzero x_0: r_0 = b - A x_0 in the fill, D^-1 from the CSR
    diagonal."""
    from paper_1511_07226_gb300 import pfk
    rp, ci, va = W.random_csr(3000, per_row=6, item_id=31)
    a = np.zeros((3000, 3000))
    rows = np.repeat(np.arange(3000), np.diff(rp))
    a[rows, ci] = va
    a = 0.5 * (a + a.T)
    nz = np.nonzero(a)
    order = np.lexsort((nz[1], nz[0]))
    r_, c_ = nz[0][order], nz[1][order]
    rp2 = np.concatenate([[0], np.cumsum(np.bincount(r_, minlength=3000))]).astype(np.int32)
    ci2 = c_.astype(np.int32)
    va2 = a[r_, c_]
    aop = O.CsrOperator(rp2, ci2, va2)
    b = W.random_vector(3000, 32)
    x0 = 0.1 * W.random_vector(3000, 33)
    prm = K.Params(mmax=30, rtol=1e-9, maxit=2000)
    ref, alts = oracle_with_envelope(method, aop, lambda: PC.JacobiPC(aop), b, prm, x0=x0)
    op = pfk.Operator.csr(ctx, rp2, ci2, va2)
    x, info, hist = pfk.solve(ctx, op, pfk.Preconditioner(ctx, op, "jacobi"), b, x0=x0, method=method, mmax=30,
                              rtol=1e-9, maxit=2000, history=2100, persistent="on")
    check_solve(hist, info, ref, alts, rtol=1e-9)


@pytest.mark.parametrize("method", ["pipefcg", "fcg"])
def test_barrier_timeout_reported_and_context_usable(ctx, method):
    """Failure detection without a GPU fault: with no barrier wait allowed
    (barrier_timeout_us < 0), the first barrier that has to wait gives up, every
    block leaves, and the solve returns PFK_ERR_TIMEOUT; the context then solves
    the same problem normally, bitwise as before."""
    from paper_1511_07226_gb300 import pfk
    c, _ = _csr_problem((64, 64))
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"], storage="csr")
    pc = pfk.Preconditioner(ctx, op, "jacobi")
    kw = dict(method=method, mmax=30, rtol=1e-8, persistent="on")
    x0, i0, _ = pfk.solve(ctx, op, pc, c["b"], **kw)
    with pytest.raises(pfk.PfkError, match="timed out") as err:
        pfk.solve(ctx, op, pc, c["b"], barrier_timeout_us=-1, **kw)
    assert err.value.status == -6   # PFK_ERR_TIMEOUT
    x1, i1, _ = pfk.solve(ctx, op, pc, c["b"], **kw)
    assert i1["status_name"] == "ok" and i1["iterations"] == i0["iterations"]
    assert np.array_equal(x1, x0)
