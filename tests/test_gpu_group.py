"""Grouped persistent PIPEFCG, PIPEGCR and PIPEFGMRES (pfk_solve_grouped, and
the server's grouped path): each system against the oracle (envelope protocol of tests/_parity.py),
bitwise independence of the batch composition and of the serving order, CTA
counts from 1 to several per system, the headline regime at 32^3 against the
stored oracle envelope, the bounded group barrier's time-out, and edge cases
(b = 0, one-cell and one-row grids with more CTAs requested than rows, the
smallest and largest window)."""
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


def _cube(dims, item, log_contrast=2.0):
    return W.poisson3d_gaussian(dims=dims, ell=3.0, log_contrast=log_contrast, config_id=5, item_id=item)


@pytest.mark.parametrize("ctas", [0, 1, 3, 8])
def test_grouped_systems_match_oracle(ctx, ctas):
    """Several 3D systems in one grouped batch, 4 inner FP64 Jacobi-PCG
    iterations, nu_max = 30, rtol 1e-8: every system against the oracle."""
    from paper_1511_07226_gb300 import pfk
    cs = [_cube(d, 10 + j) for j, d in enumerate([(20, 18, 16), (24, 24, 24), (16, 14, 12)])]
    ops = [pfk.Operator.stencil(ctx, c["dims"], c["eta"]) for c in cs]
    xs, infos, hists = pfk.solve_grouped(ctx, ops, [c["b"] for c in cs], pc_kind="inner_pcg", inner_iters=4,
                                         history=3000, ctas_per_system=ctas, mmax=30, rtol=1e-8, maxit=2000,
                                         max_restarts=50)
    for c, info, h, x in zip(cs, infos, hists, xs):
        aop = O.StencilOperator(c["dims"], c["eta"])
        ref, alts = oracle_with_envelope("pipefcg", aop, lambda: PC.InnerPCG(aop, 4), c["b"],
                                         K.Params(mmax=30, rtol=1e-8, maxit=2000, max_restarts=50))
        s = check_solve(h, info, ref, alts, rtol=1e-8, check_restarts=True)
        assert s["prefix"] >= 5, s
        if info["status"] == 0:
            assert np.linalg.norm(c["b"] - aop.apply(x)) <= 1e-8 * np.linalg.norm(c["b"]) * (1 + 1e-6)
        assert info["pass_launches"] == (ctas or -(-c["b"].size // 4096))


@pytest.mark.parametrize("ctas", [0, 3])
def test_grouped_pipegcr_matches_oracle(ctx, ctas):
    """PIPEGCR (Alg. 11) on the grouped kernel, 4 inner FP64 Jacobi-PCG
    iterations, against the oracle."""
    from paper_1511_07226_gb300 import pfk
    cs = [_cube(d, 20 + j) for j, d in enumerate([(20, 18, 16), (16, 16, 24)])]
    ops = [pfk.Operator.stencil(ctx, c["dims"], c["eta"]) for c in cs]
    xs, infos, hists = pfk.solve_grouped(ctx, ops, [c["b"] for c in cs], pc_kind="inner_pcg", inner_iters=4,
                                         history=3000, ctas_per_system=ctas, method="pipegcr", mmax=30, rtol=1e-8,
                                         maxit=2000, max_restarts=50)
    for c, info, h in zip(cs, infos, hists):
        aop = O.StencilOperator(c["dims"], c["eta"])
        ref, alts = oracle_with_envelope("pipegcr", aop, lambda: PC.InnerPCG(aop, 4), c["b"],
                                         K.Params(mmax=30, rtol=1e-8, maxit=2000, max_restarts=50))
        s = check_solve(h, info, ref, alts, rtol=1e-8, check_restarts=True)
        assert s["prefix"] >= 5, s


def test_grouped_pipegcr_first_iterations_strict(ctx):
    """PIPEGCR's fill and first 12 iterations with 5 CTAs, Jacobi, against the
    oracle to 1e-10."""
    from paper_1511_07226_gb300 import pfk
    c = _cube((20, 22, 18), 45)
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"])
    xs, infos, hists = pfk.solve_grouped(ctx, [op], [c["b"]], pc_kind="jacobi", history=64, ctas_per_system=5,
                                         method="pipegcr", mmax=30, rtol=1e-8, maxit=12)
    aop = O.StencilOperator(c["dims"], c["eta"])
    ref = K.solve("pipegcr", aop, PC.JacobiPC(aop), c["b"], prm=K.Params(mmax=30, rtol=1e-8, maxit=12))
    rho = ref.rho()
    assert ref.breakdowns == 0
    assert len(hists[0]) == len(rho) == 13
    assert np.allclose(hists[0][:, 0], rho, rtol=1e-10, atol=0.0)


@pytest.mark.parametrize("sigma,ctas", [(1.0, 0), (float("nan"), 3)])
def test_grouped_pipefgmres_matches_oracle(ctx, sigma, ctas):
    """PIPEFGMRES (Alg. 15) with constant shift sigma (given, or estimated by
    the power iteration on both sides) on the grouped kernel, 4 inner FP64
    Jacobi-PCG iterations, restart length 30, against the oracle."""
    from paper_1511_07226_gb300 import pfk
    cs = [_cube(d, 25 + j) for j, d in enumerate([(20, 18, 16), (16, 16, 24)])]
    ops = [pfk.Operator.stencil(ctx, c["dims"], c["eta"]) for c in cs]
    xs, infos, hists = pfk.solve_grouped(ctx, ops, [c["b"] for c in cs], pc_kind="inner_pcg", inner_iters=4,
                                         history=3000, ctas_per_system=ctas, method="pipefgmres", sigma=sigma,
                                         mmax=30, rtol=1e-8, maxit=2000, max_restarts=50)
    for c, info, h in zip(cs, infos, hists):
        aop = O.StencilOperator(c["dims"], c["eta"])
        ref, alts = oracle_with_envelope("pipefgmres", aop, lambda: PC.InnerPCG(aop, 4), c["b"],
                                         K.Params(mmax=30, rtol=1e-8, maxit=2000, max_restarts=50, sigma=sigma))
        s = check_solve(h, info, ref, alts, rtol=1e-8)
        assert s["prefix"] >= 5, s


def test_grouped_pipefgmres_restart_cycles_strict(ctx):
    """Restart length 6 with Jacobi (several cycles: least squares, x update,
    new cycle), 4 CTAs: the history's leading entries against the oracle to
    1e-10, the whole solve within the envelope."""
    from paper_1511_07226_gb300 import pfk
    c = _cube((18, 20, 16), 47)
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"])
    xs, infos, hists = pfk.solve_grouped(ctx, [op], [c["b"]], pc_kind="jacobi", history=4000, ctas_per_system=4,
                                         method="pipefgmres", sigma=1.0, mmax=6, rtol=1e-8, maxit=3000)
    aop = O.StencilOperator(c["dims"], c["eta"])
    prm = K.Params(mmax=6, rtol=1e-8, maxit=3000, sigma=1.0)
    ref, alts = oracle_with_envelope("pipefgmres", aop, lambda: PC.JacobiPC(aop), c["b"], prm)
    s = check_solve(hists[0], infos[0], ref, alts, rtol=1e-8)
    assert s["prefix"] >= 8, s


@pytest.mark.parametrize("method", ["pipegcr", "pipefgmres"])
def test_grouped_advection_matches_oracle(ctx, method):
    """Operators with an upwind advection part (3D and 2D, non-symmetric) on the
    grouped kernel with the nonsymmetric methods, Jacobi, 3 CTAs each: the
    fill and first iterations to 1e-10, the whole solve within the envelope."""
    from paper_1511_07226_gb300 import pfk
    cases = [(_cube((18, 16, 14), 110, log_contrast=1.0), (0.6, -0.4, 0.3)),
             (W.batched2d_system(5, 40, log_contrast=0.5, config_id=4), (3.0, -2.0, 0.0))]
    ops = [pfk.Operator.stencil(ctx, c["dims"], c["eta"], vel) for c, vel in cases]
    xs, infos, hists = pfk.solve_grouped(ctx, ops, [c["b"] for c, _ in cases], pc_kind="jacobi", history=4000,
                                         ctas_per_system=3, method=method, sigma=1.0, mmax=30, rtol=1e-8,
                                         maxit=3000)
    for (c, vel), info, h in zip(cases, infos, hists):
        aop = O.StencilOperator(c["dims"], c["eta"], vel)
        prm = K.Params(mmax=30, rtol=1e-8, maxit=3000, sigma=1.0)
        ref, alts = oracle_with_envelope(method, aop, lambda: PC.JacobiPC(aop), c["b"], prm)
        s = check_solve(h, info, ref, alts, rtol=1e-8)
        assert s["prefix"] >= 8, s
        assert np.allclose(h[:6, 0], ref.rho()[:6], rtol=1e-10, atol=0.0)


def test_grouped_jacobi_2d_and_3d(ctx):
    """Jacobi preconditioner; 2D and 3D systems in the same batch."""
    from paper_1511_07226_gb300 import pfk
    cs = [W.batched2d_system(3, 80, config_id=4), _cube((18, 16, 14), 30), W.batched2d_system(4, 45, config_id=4)]
    ops = [pfk.Operator.stencil(ctx, c["dims"], c["eta"]) for c in cs]
    xs, infos, hists = pfk.solve_grouped(ctx, ops, [c["b"] for c in cs], pc_kind="jacobi", history=3000,
                                         ctas_per_system=4, mmax=30, rtol=1e-9, maxit=2500)
    for c, info, h in zip(cs, infos, hists):
        aop = O.StencilOperator(c["dims"], c["eta"])
        ref, alts = oracle_with_envelope("pipefcg", aop, lambda: PC.JacobiPC(aop), c["b"],
                                         K.Params(mmax=30, rtol=1e-9, maxit=2500))
        check_solve(h, info, ref, alts, rtol=1e-9)


def test_grouped_first_iterations_strict(ctx):
    """The fill and the first 12 iterations with 6 CTAs per system against the
    oracle to 1e-10 (before rounding differences grow)."""
    from paper_1511_07226_gb300 import pfk
    c = _cube((22, 20, 18), 40)
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"])
    xs, infos, hists = pfk.solve_grouped(ctx, [op], [c["b"]], pc_kind="inner_pcg", inner_iters=4, history=64,
                                         ctas_per_system=6, mmax=30, rtol=1e-8, maxit=12)
    aop = O.StencilOperator(c["dims"], c["eta"])
    ref = K.solve("pipefcg", aop, PC.InnerPCG(aop, 4), c["b"], prm=K.Params(mmax=30, rtol=1e-8, maxit=12))
    rho = ref.rho()
    assert len(hists[0]) == len(rho) == 13
    assert np.allclose(hists[0][:, 0], rho, rtol=1e-10, atol=0.0)
    assert infos[0]["iterations"] == 12 and infos[0]["status_name"] == "not_converged"


def test_grouped_composition_and_cta_count(ctx):
    """A system's result does not depend on the rest of the batch (bitwise);
    another CTA count changes only the reductions' rounding."""
    from paper_1511_07226_gb300 import pfk
    cs = [_cube(d, 50 + j) for j, d in enumerate([(16, 16, 16), (30, 20, 10), (12, 12, 40), (20, 20, 20)])]
    ops = [pfk.Operator.stencil(ctx, c["dims"], c["eta"]) for c in cs]
    kw = dict(pc_kind="inner_pcg", inner_iters=4, history=3000, mmax=30, rtol=1e-8, maxit=2000)
    xs, infos, hists = pfk.solve_grouped(ctx, ops, [c["b"] for c in cs], ctas_per_system=5, **kw)
    for j in (1, 3):
        x1, i1, h1 = pfk.solve_grouped(ctx, [ops[j]], [cs[j]["b"]], ctas_per_system=5, **kw)
        assert np.array_equal(x1[0], xs[j])
        assert np.array_equal(h1[0], hists[j], equal_nan=True)
        assert i1[0]["iterations"] == infos[j]["iterations"]
    x2, i2, h2 = pfk.solve_grouped(ctx, [ops[0]], [cs[0]["b"]], ctas_per_system=2, **kw)
    k = 8
    assert np.allclose(h2[0][:k, 0], hists[0][:k, 0], rtol=1e-11, atol=0.0)


def test_grouped_fp32_inner_pcg(ctx):
    """FP32 inner Jacobi-PCG (FP32 vectors and coefficient copies) under the
    FP64 recurrences on the grouped kernel: the leading history against the
    oracle's FP32 emulation (FP32 rounding order differs), the whole solve to
    the FP64 true-residual tolerance, and a system's result independent of
    the batch (bitwise)."""
    from paper_1511_07226_gb300 import pfk
    cs = [_cube(d, 120 + j) for j, d in enumerate([(20, 18, 16), (24, 16, 12), (16, 16, 16)])]
    ops = [pfk.Operator.stencil(ctx, c["dims"], c["eta"]) for c in cs]
    kw = dict(pc_kind="inner_pcg", inner_iters=4, precision="fp32", history=3000, ctas_per_system=3, mmax=30,
              rtol=1e-8, maxit=2000, max_restarts=50)
    xs, infos, hists = pfk.solve_grouped(ctx, ops, [c["b"] for c in cs], **kw)
    for c, info, h, x in zip(cs, infos, hists, xs):
        aop = O.StencilOperator(c["dims"], c["eta"])
        ref = K.solve("pipefcg", aop, PC.InnerPCG(aop, 4, precision="fp32"), c["b"],
                      prm=K.Params(mmax=30, rtol=1e-8, maxit=3))
        rho = ref.rho()
        assert np.allclose(h[:len(rho), 0], rho, rtol=1e-5, atol=0.0)
        assert info["status_name"] == "ok"
        assert np.linalg.norm(c["b"] - aop.apply(x)) <= 1e-8 * np.linalg.norm(c["b"]) * (1 + 1e-6)
    x1, i1, h1 = pfk.solve_grouped(ctx, [ops[1]], [cs[1]["b"]], **kw)
    assert np.array_equal(x1[0], xs[1]) and np.array_equal(h1[0], hists[1], equal_nan=True)


def test_grouped_tuned_group_size(ctx):
    """ctas_per_system = -1: the group size is chosen by timing trials (x
    restored afterwards) and cached; the solve then equals, bit for bit, the
    same batch with that CTA count given explicitly, and a second tuned call
    reuses the cached choice."""
    from paper_1511_07226_gb300 import pfk
    cs = [_cube((28, 28, 28), 100 + j) for j in range(6)]
    ops = [pfk.Operator.stencil(ctx, c["dims"], c["eta"]) for c in cs]
    bs = [c["b"] for c in cs]
    kw = dict(pc_kind="inner_pcg", inner_iters=4, history=3000, mmax=30, rtol=1e-8, maxit=2000)
    xs, infos, hists = pfk.solve_grouped(ctx, ops, bs, ctas_per_system=-1, **kw)
    ctas = infos[0]["pass_launches"]
    assert all(i["pass_launches"] == ctas for i in infos)
    assert ctas in {-(-28 ** 3 // c) for c in (2048, 4096, 8192, 16384)}
    x2, i2, h2 = pfk.solve_grouped(ctx, ops, bs, ctas_per_system=ctas, **kw)
    x3, i3, h3 = pfk.solve_grouped(ctx, ops, bs, ctas_per_system=-1, **kw)
    for j in range(len(cs)):
        assert np.array_equal(xs[j], x2[j]) and np.array_equal(xs[j], x3[j])
        assert np.array_equal(hists[j], h2[j], equal_nan=True)
        assert infos[j]["status_name"] == "ok"


def test_grouped_nonzero_initial_guess_and_restart_truncation(ctx):
    from paper_1511_07226_gb300 import pfk
    cs = [_cube(d, 60 + j) for j, d in enumerate([(18, 18, 18), (26, 14, 12)])]
    ops = [pfk.Operator.stencil(ctx, c["dims"], c["eta"]) for c in cs]
    x0s = [1e-4 * W.random_vector(c["b"].size, 70 + j) for j, c in enumerate(cs)]
    xs, infos, hists = pfk.solve_grouped(ctx, ops, [c["b"] for c in cs], x0s=x0s, pc_kind="inner_pcg",
                                         inner_iters=4, history=3000, ctas_per_system=3, mmax=20,
                                         truncation="restart", rtol=1e-8, maxit=2000, max_restarts=50)
    for c, x0, info, h in zip(cs, x0s, infos, hists):
        aop = O.StencilOperator(c["dims"], c["eta"])
        ref, alts = oracle_with_envelope("pipefcg", aop, lambda: PC.InnerPCG(aop, 4), c["b"],
                                         K.Params(mmax=20, rtol=1e-8, maxit=2000, max_restarts=50,
                                                  truncation="restart"), x0=x0)
        check_solve(h, info, ref, alts, rtol=1e-8)


@pytest.mark.parametrize("n", [32, 48])
@pytest.mark.parametrize("method", ["pipefcg", "pipegcr"])
def test_grouped_headline_regime(ctx, method, n):
    """The 32^3 and 48^3 headline cases (contrast 1e6, 4 inner FP64
    Jacobi-PCG, nu_max = 30, rtol 1e-8, residual-replacement restarts) on the
    grouped kernel with the automatic CTA count (8 and 27), against the stored
    oracle envelopes; status, band and restarts only where all its roundings
    agree on the outcome."""
    from paper_1511_07226_gb300 import pfk
    from tests import _oracle_pool as P
    from tests._headline_cases import CASES
    name = f"{method}_{n}"
    if P.load_stored(name) is None:
        pytest.skip("no stored envelope for these inputs")
    cs = CASES[name]
    c = P.problem(cs["problem"])
    prm = cs["prm"]
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"])
    xs, infos, hists = pfk.solve_grouped(ctx, [op], [c["b"]], pc_kind="inner_pcg", inner_iters=4,
                                         history=prm["maxit"] + 400, method=method, mmax=30, rtol=1e-8,
                                         maxit=prm["maxit"], max_restarts=prm["max_restarts"])
    ref, alts = P.envelope_runs(cs["problem"], cs["method"], cs["pc"], prm, orders=cs["orders"], big=cs["big"],
                                stored=name)()
    agree = all(a.status == ref.status for a in alts)
    s = check_solve(hists[0], infos[0], ref, alts, rtol=1e-8, check_status=agree, check_restarts=True)
    assert s["prefix"] >= 10, s
    if agree and ref.status == "converged":
        assert infos[0]["status_name"] == "ok"


def test_grouped_barrier_timeout_is_reported(ctx):
    """A group barrier that may not wait (barrier_timeout_us < 0) gives up at
    once: the system ends with PFK_ERR_TIMEOUT, the context stays usable."""
    from paper_1511_07226_gb300 import pfk
    c = _cube((16, 16, 16), 80)
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"])
    xs, infos, _ = pfk.solve_grouped(ctx, [op], [c["b"]], pc_kind="jacobi", ctas_per_system=4, mmax=10,
                                     rtol=1e-8, barrier_timeout_us=-1)
    assert infos[0]["status"] == -6
    xs, infos, _ = pfk.solve_grouped(ctx, [op], [c["b"]], pc_kind="jacobi", ctas_per_system=4, mmax=10,
                                     rtol=1e-8)
    assert infos[0]["status"] == 0


def test_server_grouped_request_barrier_timeout(ctx):
    """A served grouped request whose system barrier may not wait
    (barrier_timeout_us < 0, 4 CTAs) ends with PFK_ERR_TIMEOUT through the
    server; requests before and after it are served normally."""
    from paper_1511_07226_gb300 import pfk
    c = _cube((24, 24, 24), 130)
    kw = dict(mmax=30, rtol=1e-8, maxit=2000)
    srv = pfk.Server(ctx, workers=1)
    try:
        t0 = srv.submit(c["dims"], c["eta"], c["b"], **kw)
        t1 = srv.submit(c["dims"], c["eta"], c["b"], barrier_timeout_us=-1, **kw)
        assert srv.poll(t0)[1]["status_name"] == "ok"
        with pytest.raises(pfk.PfkError, match="timed out"):
            srv.poll(t1)
        t2 = srv.submit(c["dims"], c["eta"], c["b"], **kw)
        x2, i2, _ = srv.poll(t2)
        assert i2["status_name"] == "ok" and i2["pass_launches"] == 4
    finally:
        srv.close()


def test_server_grouped_requests_bitwise_and_oracle(ctx):
    """Requests served together through the grouped path (PIPEFCG, PIPEGCR,
    PIPEFGMRES up to group_max_n unknowns) equal, bit for bit, the same
    requests solved alone by pfk_solve_grouped; a larger request in the same
    stream goes to a whole-GPU worker and equals pfk_solve alone; one served
    grouped request is also checked against the oracle's envelope."""
    from paper_1511_07226_gb300 import pfk
    cs = [_cube(d, 90 + j) for j, d in enumerate([(24, 24, 24), (16, 16, 16), (20, 18, 22), (12, 30, 14)])]
    meths = ["pipefcg", "pipegcr", "pipefgmres", "pipegcr"]
    big = _cube((26, 26, 26), 95)
    kw = dict(mmax=30, rtol=1e-8, maxit=2000, max_restarts=50, sigma=1.0)
    srv = pfk.Server(ctx, workers=2, group_max_n=16000)
    try:
        tickets = [srv.submit(c["dims"], c["eta"], c["b"], method=m, **kw) for c, m in zip(cs, meths)]
        tg = srv.submit(big["dims"], big["eta"], big["b"], method="pipefgmres", **kw)
        served = [srv.poll(t) for t in tickets]
        xg, ig, _ = srv.poll(tg)
    finally:
        srv.close()
    for c, m, (x, info, lat) in zip(cs, meths, served):
        op = pfk.Operator.stencil(ctx, c["dims"], c["eta"])
        x1, i1, _ = pfk.solve_grouped(ctx, [op], [c["b"]], pc_kind="inner_pcg", inner_iters=4, method=m, **kw)
        assert np.array_equal(x, x1[0]), m
        assert info["iterations"] == i1[0]["iterations"] and info["restarts"] == i1[0]["restarts"]
        assert info["pass_launches"] == i1[0]["pass_launches"] >= 1
    op = pfk.Operator.stencil(ctx, big["dims"], big["eta"])
    pc = pfk.Preconditioner(ctx, op, "inner_pcg", inner_iters=4)
    x1, i1, _ = pfk.solve(ctx, op, pc, big["b"], method="pipefgmres", **kw)
    assert np.array_equal(xg, x1) and ig["iterations"] == i1["iterations"]
    # the served solution of the first request against the oracle's
    c = cs[0]
    aop = O.StencilOperator(c["dims"], c["eta"])
    ref, alts = oracle_with_envelope("pipefcg", aop, lambda: PC.InnerPCG(aop, 4), c["b"],
                                     K.Params(mmax=30, rtol=1e-8, maxit=2000, max_restarts=50))
    x, info, _ = served[0]
    if ref.status == "converged" and all(a.status == "converged" for a in alts):
        assert info["status_name"] == "ok"
        band = 2 * max(abs(a.iterations - ref.iterations) for a in alts) + 0.05 * ref.iterations + 2
        assert abs(info["iterations"] - ref.iterations) <= band
        err = np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x)
        assert err <= 1e-5, err


@pytest.mark.parametrize("method", ["pipefcg", "pipegcr", "pipefgmres"])
def test_grouped_zero_rhs(ctx, method):
    """b = 0, x0 = 0: every system stops in its fill with x = 0 and no
    iteration, whatever its CTA count."""
    from paper_1511_07226_gb300 import pfk
    cs = [_cube(d, 140 + j) for j, d in enumerate([(9, 7, 5), (12, 12, 12)])]
    ops = [pfk.Operator.stencil(ctx, c["dims"], c["eta"]) for c in cs]
    xs, infos, _ = pfk.solve_grouped(ctx, ops, [np.zeros(op.n) for op in ops], pc_kind="jacobi",
                                     ctas_per_system=3, method=method, sigma=1.0, mmax=8, rtol=1e-8)
    for x, info in zip(xs, infos):
        assert info["status_name"] == "ok" and info["iterations"] == 0
        assert np.all(x == 0.0)


@pytest.mark.parametrize("dims", [(1, 1, 1), (1, 1), (37, 1, 1), (1, 29, 1), (1, 1, 41), (33, 1), (70, 3)])
@pytest.mark.parametrize("method", ["pipefcg", "pipegcr", "pipefgmres"])
def test_grouped_degenerate_grids(ctx, dims, method):
    """One cell, one row or column, one pillar, a 70 x 3 strip, all in one
    batch with 8 CTAs requested (capped at one per x-row): the group's row
    split, its ragged tails and a one-CTA group against the oracle."""
    from paper_1511_07226_gb300 import pfk
    n = int(np.prod(dims))
    g = W.rng(31, n)
    eta = np.power(10.0, g.uniform(-1.0, 1.0, size=n))
    b = g.uniform(-1.0, 1.0, size=n)
    aop = O.StencilOperator(dims, eta)
    prm = K.Params(mmax=8, rtol=1e-10, maxit=200, sigma=1.0)
    ref, alts = oracle_with_envelope(method, aop, lambda: PC.JacobiPC(aop), b, prm)
    op = pfk.Operator.stencil(ctx, dims, eta)
    xs, infos, hists = pfk.solve_grouped(ctx, [op], [b], pc_kind="jacobi", history=400, ctas_per_system=8,
                                         method=method, sigma=1.0, mmax=8, rtol=1e-10, maxit=200)
    rows = dims[1] * (dims[2] if len(dims) > 2 else 1)
    assert infos[0]["pass_launches"] == min(8, rows)
    check_solve(hists[0], infos[0], ref, alts, rtol=1e-10, min_prefix=1)
    np.testing.assert_allclose(aop.apply(xs[0]), b, rtol=0, atol=1e-8 * np.linalg.norm(b))


def test_grouped_window_and_inner_extremes(ctx):
    """nu_max = 1 (IPCG) with one inner PCG iteration, and the largest window
    (nu_max = 32) with eight, on the grouped kernel against the oracle."""
    from paper_1511_07226_gb300 import pfk
    c = _cube((16, 14, 12), 150)
    aop = O.StencilOperator(c["dims"], c["eta"])
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"])
    for mmax, inner in ((1, 1), (32, 8)):
        xs, infos, hists = pfk.solve_grouped(ctx, [op], [c["b"]], pc_kind="inner_pcg", inner_iters=inner,
                                             history=3000, ctas_per_system=4, mmax=mmax, rtol=1e-8, maxit=2000)
        ref, alts = oracle_with_envelope("pipefcg", aop, lambda: PC.InnerPCG(aop, inner), c["b"],
                                         K.Params(mmax=mmax, rtol=1e-8, maxit=2000))
        check_solve(hists[0], infos[0], ref, alts, rtol=1e-8)
