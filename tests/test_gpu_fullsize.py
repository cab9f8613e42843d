"""Parity at the workloads' full sizes, in the launch configurations the bench
times, on what the oracle can compute at that size in seconds:

* the 256^3 two-phase advection operator (every entry);
* its 8-sweep Chebyshev-Jacobi preconditioner, BF16 coefficients / FP32
  vectors and FP64, on sampled cells: a cell's output after k sweeps depends
  only on inputs within k cells, so the oracle runs the sweeps on a box of
  radius k around the cell (cut from the full-size operator's arrays; the
  cut's error travels one cell per operator application and stops k - 1
  cells inside the box);
* the first PIPEFGMRES(30) iterations at 256^3 against the oracle (Jacobi);
* the 512-system batch: sampled systems (the largest, the smallest, random
  ones) against the oracle, inner PCG in FP64 (strict) and FP32 (emulated);
* full-size serving requests (the largest of the stream's first 48): each
  served result equals the same request solved alone, bit for bit.
"""
import types

import numpy as np
import pytest

import workloads as W
from oracle import krylov as K
from oracle import operators as O
from oracle import preconditioners as PC

pytestmark = pytest.mark.gpu

SWEEPS = 8


@pytest.fixture(scope="module")
def ctx(lib):
    from paper_1511_07226_gb300 import pfk
    return pfk.Context(0)


@pytest.fixture(scope="module")
def two_phase():
    c = W.poisson3d_two_phase()
    return c, O.StencilOperator(c["dims"], c["eta"], c["vel"])


def test_two_phase_operator_full_size(ctx, two_phase):
    from paper_1511_07226_gb300 import pfk
    c, aop = two_phase
    x = W.random_vector(aop.n, 11)
    ref = aop.apply(x)
    got = pfk.Operator.stencil(ctx, c["dims"], c["eta"], c["vel"]).apply(x).cpu().numpy()
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-14 * np.abs(ref).max())


def _sample_cells(shape, count, seed):
    g = W.rng(970, seed)
    nz, ny, nx = shape
    cells = [(0, 0, 0), (nz - 1, ny - 1, nx - 1), (0, ny // 2, nx - 1), (nz // 2, 0, nx // 2)]
    cells += [tuple(int(g.integers(0, s)) for s in shape) for _ in range(count)]
    return cells


def _patch_chebyshev(full, v, cell, lo, hi, precision):
    """The oracle's Chebyshev sweeps on the box of radius SWEEPS around `cell`
    (clipped to the domain), using the full operator's arrays; returns the
    output at the cell."""
    shape = full.shape if precision != "fp64" else full.op_shape
    sl = tuple(slice(max(0, c - SWEEPS), min(s, c + SWEEPS + 1)) for c, s in zip(cell, shape))
    centre = tuple(c - s.start for c, s in zip(cell, sl))
    vp = v.reshape(shape)[sl].reshape(-1)
    pshape = tuple(s.stop - s.start for s in sl)
    if precision == "fp64":
        aop = full.op
        diag = full.diag.reshape(shape)[sl]
        patch_op = types.SimpleNamespace(shape=pshape, axes=aop.axes, vel=aop.vel, adv=aop.adv,
                                         K={key: k[sl] for key, k in aop.K.items()})
        apply_a = lambda u: O.StencilOperator.apply(patch_op, u)   # noqa: E731
        dinv = (1.0 / diag).reshape(-1)
        dt = np.float64
    else:
        rs = types.SimpleNamespace(shape=pshape, op=full.op, adv=full.adv, d=full.d[sl], dinv=full.dinv[sl],
                                   K={key: k[sl] for key, k in full.K.items()})
        apply_a = lambda u: PC.RoundedStencil.apply(rs, u)          # noqa: E731
        dinv = rs.dinv.reshape(-1)
        dt = np.float32
    ch = types.SimpleNamespace(lo=lo, hi=hi, k=SWEEPS, precision=precision, apply_A=apply_a, dinv=dinv, dt=dt)
    out = PC.Chebyshev.__call__(ch, vp).reshape(pshape)
    return float(out[centre])


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-12), ("bf16", 1e-4)])
def test_two_phase_chebyshev_sampled_cells(ctx, two_phase, precision, rtol):
    from paper_1511_07226_gb300 import pfk
    c, aop = two_phase
    lo, hi = PC.chebyshev_bounds(aop)
    if precision == "fp64":
        full = types.SimpleNamespace(op=aop, op_shape=aop.shape, diag=aop.diagonal())
    else:
        full = PC.RoundedStencil(aop, precision)
    v = W.random_vector(aop.n, 12)
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"], c["vel"])
    got = pfk.Preconditioner(ctx, op, "chebyshev", inner_iters=SWEEPS, precision=precision).apply(v).cpu().numpy()
    shape = aop.shape
    scale = np.abs(got).max()
    for cell in _sample_cells(shape, 12, 1):
        ref = _patch_chebyshev(full, v, cell, lo, hi, precision)
        idx = np.ravel_multi_index(cell, shape)
        assert abs(got[idx] - ref) <= rtol * abs(ref) + 1e-3 * rtol * scale, (cell, got[idx], ref)


def test_two_phase_pipefgmres_first_iterations(ctx, two_phase):
    """PIPEFGMRES(30) at 256^3 with the advection term: the fill and the first
    three iterations agree with the oracle to 1e-10.  Jacobi here (the
    Chebyshev preconditioner is checked on its own above: the oracle's eight
    FP64 sweeps take ~10 s per application at this size)."""
    from paper_1511_07226_gb300 import pfk
    c, aop = two_phase
    prm = K.Params(mmax=30, rtol=1e-8, sigma=1.0, maxit=3)
    ref = K.solve("pipefgmres", aop, PC.JacobiPC(aop), c["b"], prm=prm)
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"], c["vel"])
    pc = pfk.Preconditioner(ctx, op, "jacobi")
    x, info, hist = pfk.solve(ctx, op, pc, c["b"], method="pipefgmres", mmax=30, sigma=1.0, rtol=1e-8, maxit=3,
                              history=16)
    rho = ref.rho()
    assert len(hist) == len(rho)
    assert np.allclose(hist[:, 0], rho, rtol=1e-10, atol=0.0)


@pytest.fixture(scope="module")
def batch():
    sides = W.batched2d_sides()
    return sides, [W.batched2d_system(j, int(s)) for j, s in enumerate(sides)]


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-10), ("fp32", 1e-4)])
def test_full_batch_sampled_systems(ctx, batch, precision, rtol):
    """All 512 systems in one launch (block size autotuned, as the bench runs
    it), 6 iterations each; sampled systems' residual histories against the
    oracle (FP32: the oracle emulates the FP32 inner CG, rounding order
    differs)."""
    from paper_1511_07226_gb300 import pfk
    sides, sys_ = batch
    ops = [pfk.Operator.stencil(ctx, c["dims"], c["eta"]) for c in sys_]
    xs, infos, hists = pfk.solve_batched(ctx, ops, [c["b"] for c in sys_], pc_kind="inner_pcg", inner_iters=4,
                                         precision=precision, mmax=20, rtol=1e-8, maxit=6, history=16)
    g = W.rng(971, 0)
    picks = {int(np.argmax(sides)), int(np.argmin(sides))} | {int(j) for j in g.integers(0, len(sides), size=3)}
    for j in sorted(picks):
        c = sys_[j]
        aop = O.StencilOperator(c["dims"], c["eta"])
        ref = K.solve("pipefcg", aop, PC.InnerPCG(aop, 4, precision=precision), c["b"],
                      prm=K.Params(mmax=20, rtol=1e-8, maxit=6))
        rho = ref.rho()
        h = hists[j]
        assert len(h) == len(rho), (j, len(h), len(rho))
        assert np.allclose(h[:, 0], rho, rtol=rtol, atol=0.0), (j, sides[j])


def test_full_size_requests_served_equal_alone(ctx):
    """The largest request of each method among the stream's first 48 (sides
    up to 160) and the largest overall, served concurrently by 8 workers,
    equal the same solves alone."""
    from paper_1511_07226_gb300 import pfk
    meth = {0: "pipefcg", 1: "pipegcr", 2: "pipefgmres"}
    stream = sorted(W.request_stream(count=48), key=lambda r: -r["side"])
    reqs = [stream[0]] + [next(r for r in stream if r["method"] == m and r is not stream[0]) for m in meth]
    probs = [W.request_problem(r) for r in reqs]
    kw = dict(mmax=30, rtol=1e-8, maxit=400, max_restarts=20)
    srv = pfk.Server(ctx, workers=8)
    tickets = [srv.submit(p["dims"], p["eta"], p["b"], method=meth[r["method"]], **kw) for r, p in zip(reqs, probs)]
    served = [srv.poll(t) for t in tickets]
    srv.close()
    for r, p, (x, info, _) in zip(reqs, probs, served):
        op = pfk.Operator.stencil(ctx, p["dims"], p["eta"])
        pc = pfk.Preconditioner(ctx, op, "inner_pcg", 4, "fp64")
        xa, ia, _ = pfk.solve(ctx, op, pc, p["b"], method=meth[r["method"]], **kw)
        assert info["status_name"] == ia["status_name"], (r, info, ia)
        assert info["iterations"] == ia["iterations"]
        assert np.array_equal(x, xa), r
