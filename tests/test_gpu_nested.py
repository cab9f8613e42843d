"""Nested solve on the GPU (Sec. 6, ex43 structure): outer FGMRES / PIPEFGMRES on
the Stokes-like saddle-point system with the block upper-triangular
preconditioner whose velocity block is an inner (pipelined) flexible Krylov
solve, all recorded in the outer solve's CUDA graphs.  Against the oracle's
BlockUpperPC (single application, element by element) and whole solves
(envelope protocol, and the dense solution)."""
import numpy as np
import pytest

from oracle import krylov as K
from oracle import operators as O
from oracle import preconditioners as PC
from tests._parity import check_solve, oracle_with_envelope
from workloads import stokes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    from paper_1511_07226_gb300 import pfk
    return pfk.Context(0)


def _gpu_ops(ctx, d):
    from paper_1511_07226_gb300 import pfk
    A = pfk.Operator.csr(ctx, *d["A"])
    Kop = pfk.Operator.csr(ctx, *d["K"])
    Bt = pfk.Operator.csr(ctx, *d["Bt"])
    return A, Kop, Bt


@pytest.mark.parametrize("inner", ["fcg", "pipefcg", "gcr", "pipegcr", "pipegcr_w"])
def test_block_pc_application_matches_oracle(ctx, inner):
    from paper_1511_07226_gb300 import pfk
    d = S.stokes2d(n=20, item_id=3)
    A, Kop, Bt = _gpu_ops(ctx, d)
    pc = pfk.Preconditioner.block_upper(ctx, Kop, Bt, d["schur_diag"], inner, 20, 1e-5, 200)
    ref = PC.BlockUpperPC(O.CsrOperator(*d["K"]), O.CsrOperator(*d["Bt"]), d["schur_diag"], d["nu"],
                          inner_method=inner, inner_mmax=20, inner_rtol=1e-5, inner_maxit=200)
    for item in range(3):
        v = np.random.default_rng(40 + item).standard_normal(d["N"])
        got = pc.apply(v).cpu().numpy()
        want = ref(v)
        # the inner solve amplifies rounding: agreement to 1e-8 of the result's size
        assert np.linalg.norm(got - want) <= 1e-8 * np.linalg.norm(want), inner


@pytest.mark.parametrize("outer", ["fgmres", "pipefgmres"])
@pytest.mark.parametrize("inner", ["pipefcg", "fcg", "pipegcr"])
def test_nested_solve_matches_oracle(ctx, outer, inner):
    from paper_1511_07226_gb300 import pfk
    d = S.stokes2d(n=16, item_id=4)
    nu = d["nu"]
    A, Kop, Bt = _gpu_ops(ctx, d)
    mk = lambda: PC.BlockUpperPC(O.CsrOperator(*d["K"]), O.CsrOperator(*d["Bt"]), d["schur_diag"], nu,
                                 inner_method=inner, inner_mmax=30, inner_rtol=1e-4, inner_maxit=100)
    prm = K.Params(mmax=30, rtol=1e-8, norm="unpreconditioned", sigma=1.0, maxit=300)
    ref, alts = oracle_with_envelope(outer, O.CsrOperator(*d["A"]), mk, d["b"], prm)
    pc = pfk.Preconditioner.block_upper(ctx, Kop, Bt, d["schur_diag"], inner, 30, 1e-4, 100)
    x, info, hist = pfk.solve(ctx, A, pc, d["b"], method=outer, mmax=30, rtol=1e-8, norm="unpreconditioned",
                              sigma=1.0, maxit=300, history=1000)
    check_solve(hist, info, ref, alts, rtol=1e-8, min_prefix=1)
    xd = np.linalg.lstsq(_dense(d["A"]), d["b"], rcond=None)[0]
    assert np.linalg.norm(x[:nu] - xd[:nu]) <= 1e-6 * np.linalg.norm(xd[:nu])


def _dense(csr):
    rp, ci, va = csr
    n = len(rp) - 1
    a = np.zeros((n, n))
    for r in range(n):
        a[r, ci[rp[r]:rp[r + 1]]] += va[rp[r]:rp[r + 1]]
    return a


def test_block_pc_argument_errors(ctx):
    from paper_1511_07226_gb300 import pfk
    d = S.stokes2d(n=6, item_id=5)
    A, Kop, Bt = _gpu_ops(ctx, d)
    with pytest.raises(pfk.PfkError, match="inner method"):
        pfk.Preconditioner.block_upper(ctx, Kop, Bt, d["schur_diag"], "fgmres")
    bad = d["schur_diag"].copy()
    bad[3] = 0.0
    with pytest.raises(pfk.PfkError, match="Schur"):
        pfk.Preconditioner.block_upper(ctx, Kop, Bt, bad)
    with pytest.raises(pfk.PfkError):
        pfk.Preconditioner.block_upper(ctx, Kop, Kop, d["schur_diag"])     # Bt must be larger than K
