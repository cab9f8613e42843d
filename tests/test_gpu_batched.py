"""Batched PIPEFCG in one persistent launch (pfk_solve_batched): each system
against the oracle (envelope protocol), bitwise independence of the batch
composition, and the FP32 inner-CG preconditioner."""
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


def _systems(sides):
    return [W.batched2d_system(j, s, config_id=4) for j, s in enumerate(sides)]


@pytest.mark.parametrize("block_threads", [0, 128, 512])
def test_batched_systems_match_oracle(ctx, block_threads):
    from paper_1511_07226_gb300 import pfk
    sides = [33, 48, 20, 64, 40]
    sys = _systems(sides)
    ops = [pfk.Operator.stencil(ctx, c["dims"], c["eta"]) for c in sys]
    xs, infos, hists = pfk.solve_batched(ctx, ops, [c["b"] for c in sys], pc_kind="inner_pcg", inner_iters=4,
                                         precision="fp64", history=2000, block_threads=block_threads, mmax=20,
                                         rtol=1e-8, maxit=1000)
    for c, info, h in zip(sys, infos, hists):
        aop = O.StencilOperator(c["dims"], c["eta"])
        ref, alts = oracle_with_envelope("pipefcg", aop, lambda: PC.InnerPCG(aop, 4), c["b"],
                                         K.Params(mmax=20, rtol=1e-8, maxit=1000))
        # with this nonlinear preconditioner at contrast 1e4 the solves stagnate
        # and reach rtol only through replacement restarts whose timing is set
        # by rounding (the 1000-iteration cap can stop all oracle orders while
        # another valid order converges), so the outcome is not compared
        check_solve(h, info, ref, alts, rtol=1e-8, check_status=False)


def test_batch_composition_does_not_change_results(ctx):
    from paper_1511_07226_gb300 import pfk
    sides = [40, 25, 57, 32]
    sys = _systems(sides)
    ops = [pfk.Operator.stencil(ctx, c["dims"], c["eta"]) for c in sys]
    xs, infos, hists = pfk.solve_batched(ctx, ops, [c["b"] for c in sys], history=2000, block_threads=256,
                                         mmax=20, rtol=1e-8)
    for j in (0, 2):
        x1, i1, h1 = pfk.solve_batched(ctx, [ops[j]], [sys[j]["b"]], history=2000, block_threads=256, mmax=20,
                                       rtol=1e-8)
        assert np.array_equal(x1[0], xs[j])
        assert np.array_equal(h1[0], hists[j], equal_nan=True)
        assert i1[0]["iterations"] == infos[j]["iterations"]


def test_batched_3d_and_jacobi(ctx):
    from paper_1511_07226_gb300 import pfk
    cs = [W.poisson3d_gaussian(dims=(14, 12, 10), ell=3.0, log_contrast=2.0, config_id=4, item_id=70 + j)
          for j in range(3)]
    ops = [pfk.Operator.stencil(ctx, c["dims"], c["eta"]) for c in cs]
    xs, infos, hists = pfk.solve_batched(ctx, ops, [c["b"] for c in cs], pc_kind="jacobi", history=2000,
                                         mmax=30, rtol=1e-9, maxit=2000)
    for c, info, h in zip(cs, infos, hists):
        aop = O.StencilOperator(c["dims"], c["eta"])
        ref, alts = oracle_with_envelope("pipefcg", aop, lambda: PC.JacobiPC(aop), c["b"],
                                         K.Params(mmax=30, rtol=1e-9, maxit=2000))
        check_solve(h, info, ref, alts, rtol=1e-9)


def test_batched_fp32_preconditioner(ctx):
    """Mixed precision: FP32 inner CG under FP64 recurrences must still meet the
    FP64 true-residual tolerance."""
    from paper_1511_07226_gb300 import pfk
    sys = _systems([48, 96, 32])
    ops = [pfk.Operator.stencil(ctx, c["dims"], c["eta"]) for c in sys]
    xs, infos, _ = pfk.solve_batched(ctx, ops, [c["b"] for c in sys], precision="fp32", mmax=20, rtol=1e-8)
    for c, info, x in zip(sys, infos, xs):
        assert info["status"] == 0
        assert info["rnorm_true"] <= 1e-8 * info["bnorm"]
        aop = O.StencilOperator(c["dims"], c["eta"])
        assert np.linalg.norm(c["b"] - aop.apply(x)) <= 1e-8 * np.linalg.norm(c["b"]) * (1 + 1e-6)


def test_batched_advection_first_iterations(ctx):
    """Operators with an upwind advection part (2D and 3D) in one batch: the
    first iterations of each system against the oracle (strict)."""
    from paper_1511_07226_gb300 import pfk
    # mild contrast and advection: no norm breakdown within the compared iterations
    cases = [(W.batched2d_system(j, s, log_contrast=0.25, config_id=4), vel) for j, (s, vel) in
             enumerate([(37, (3.0, -2.0, 0.0)), (52, (-4.0, 1.0, 0.0))])]
    c3 = W.poisson3d_gaussian(dims=(12, 10, 9), ell=3.0, log_contrast=1.0, config_id=4, item_id=90)
    cases.append((c3, (0.2, 0.1, -0.3)))
    ops = [pfk.Operator.stencil(ctx, c["dims"], c["eta"], vel) for c, vel in cases]
    xs, infos, hists = pfk.solve_batched(ctx, ops, [c["b"] for c, _ in cases], pc_kind="jacobi", history=32,
                                         block_threads=256, mmax=20, rtol=1e-8, maxit=12)
    for (c, vel), h in zip(cases, hists):
        aop = O.StencilOperator(c["dims"], c["eta"], vel)
        ref = K.solve("pipefcg", aop, PC.JacobiPC(aop), c["b"], prm=K.Params(mmax=20, rtol=1e-8, maxit=12))
        rho = ref.rho()
        assert ref.breakdowns == 0
        assert len(h) == len(rho)
        assert np.allclose(h[:, 0], rho, rtol=1e-10, atol=0.0), c["dims"]


def test_batched_nonzero_initial_guess(ctx):
    """x_0 != 0 per system (r_0 = b - A x_0 in the fill), against the oracle."""
    from paper_1511_07226_gb300 import pfk
    sys_ = _systems([30, 45])
    ops = [pfk.Operator.stencil(ctx, c["dims"], c["eta"]) for c in sys_]
    # x_0 of the size of the solution (b ~ h^2): a unit-size x_0 makes the
    # initial residual so much larger than b that the first convergence of the
    # natural norm is far from the true-residual goal and the outcome hinges on
    # the replacement restart
    x0s = [1e-4 * W.random_vector(int(np.prod(c["dims"])), 40 + j) for j, c in enumerate(sys_)]
    xs, infos, hists = pfk.solve_batched(ctx, ops, [c["b"] for c in sys_], x0s=x0s, pc_kind="jacobi", history=2000,
                                         block_threads=256, mmax=20, rtol=1e-8, maxit=1000)
    for c, x0, info, h in zip(sys_, x0s, infos, hists):
        aop = O.StencilOperator(c["dims"], c["eta"])
        ref, alts = oracle_with_envelope("pipefcg", aop, lambda: PC.JacobiPC(aop), c["b"],
                                         K.Params(mmax=20, rtol=1e-8, maxit=1000), x0=x0)
        check_solve(h, info, ref, alts, rtol=1e-8)


def test_batched_restart_truncation(ctx):
    """Restart-style truncation (Sec. 5 remark, nu_i = ((i - 1) mod nu_max) + 1)
    in the batched kernel against the oracle, inner FP64 PCG."""
    from paper_1511_07226_gb300 import pfk
    sys_ = _systems([36, 28, 50])
    ops = [pfk.Operator.stencil(ctx, c["dims"], c["eta"]) for c in sys_]
    xs, infos, hists = pfk.solve_batched(ctx, ops, [c["b"] for c in sys_], pc_kind="inner_pcg", inner_iters=4,
                                         precision="fp64", history=2000, block_threads=256, mmax=20,
                                         truncation="restart", rtol=1e-8, maxit=1000, max_restarts=50)
    for c, info, h in zip(sys_, infos, hists):
        aop = O.StencilOperator(c["dims"], c["eta"])
        ref, alts = oracle_with_envelope("pipefcg", aop, lambda: PC.InnerPCG(aop, 4), c["b"],
                                         K.Params(mmax=20, rtol=1e-8, maxit=1000, truncation="restart",
                                                  max_restarts=50))
        check_solve(h, info, ref, alts, rtol=1e-8)
