"""The continuous-batching server (pfk_server_*): every served result is bit for
bit the result of the same request solved alone -- through pfk_solve_grouped
for the small requests the server advances on the grouped kernel, through
pfk_solve for the rest -- whatever else runs concurrently;
admission, queue limit and ticket handling."""
import time

import numpy as np
import pytest

import workloads as W
from oracle import operators as O

pytestmark = pytest.mark.gpu

METHOD_OF = {0: "pipefcg", 1: "pipegcr", 2: "pipefgmres"}
KW = dict(mmax=30, rtol=1e-8, maxit=3000)


@pytest.fixture(scope="module")
def ctx(lib):
    from paper_1511_07226_gb300 import pfk
    return pfk.Context(0)


def _requests(count, lo=12, hi=36):
    out = []
    for r in W.request_stream(count=count, side_lo=lo, side_hi=hi):
        c = W.request_problem(r, ell=4.0)
        out.append((r, c))
    return out


GROUP_MAX_N = 110592   # the server's default bound of grouped requests


def _grouped(c, method, group_max_n=0):
    """Whether a default server runs this request on the grouped kernel."""
    bound = GROUP_MAX_N if group_max_n == 0 else group_max_n
    return method in ("pipefcg", "pipegcr", "pipefgmres") and c["b"].size <= bound


def _alone(ctx, c, method, group_max_n=0):
    from paper_1511_07226_gb300 import pfk
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"])
    if _grouped(c, method, group_max_n):
        xs, infos, _ = pfk.solve_grouped(ctx, [op], [c["b"]], pc_kind="inner_pcg", inner_iters=4, method=method,
                                         **KW)
        return xs[0], infos[0]
    pc = pfk.Preconditioner(ctx, op, "inner_pcg", 4, "fp64")
    x, info, _ = pfk.solve(ctx, op, pc, c["b"], method=method, **KW)
    return x, info


@pytest.mark.parametrize("workers", [1, 4])
def test_served_results_equal_solves_alone(ctx, workers):
    from paper_1511_07226_gb300 import pfk
    reqs = _requests(10)
    srv = pfk.Server(ctx, workers=workers)
    tickets = [srv.submit(c["dims"], c["eta"], c["b"], method=METHOD_OF[r["method"]], **KW) for r, c in reqs]
    got = [srv.poll(t) for t in tickets]
    srv.close()
    for (r, c), (x, info, lat) in zip(reqs, got):
        method = METHOD_OF[r["method"]]
        xa, ia = _alone(ctx, c, method)
        assert info["status_name"] == ia["status_name"] == "ok", (method, info, ia)
        assert info["iterations"] == ia["iterations"]
        assert np.array_equal(x, xa), method
        assert lat > 0.0
        aop = O.StencilOperator(c["dims"], c["eta"])
        res = np.linalg.norm(c["b"] - aop.apply(x)) / np.linalg.norm(c["b"])
        assert res < 1e-6, (method, res)


def test_tiny_budget_admits_one_at_a_time_in_order(ctx):
    """With a budget below any request's estimate, a request is admitted only
    when nothing else is active: requests finish in arrival order (all on the
    workers: the arrival order holds within each admission path)."""
    from paper_1511_07226_gb300 import pfk
    reqs = _requests(6, 16, 28)
    srv = pfk.Server(ctx, workers=4, memory_budget=1, group_max_n=-1)
    t0 = []
    tickets = []
    for r, c in reqs:
        t0.append(time.perf_counter())
        tickets.append(srv.submit(c["dims"], c["eta"], c["b"], method=METHOD_OF[r["method"]], **KW))
    done = []
    for t, ts in zip(tickets, t0):
        x, info, lat = srv.poll(t)
        assert info["status_name"] == "ok"
        done.append(ts + lat / 1e3)
    srv.close()
    # completion instants (submission + latency) do not decrease, up to clock jitter
    assert all(b >= a - 2e-3 for a, b in zip(done, done[1:])), np.diff(done)


def test_queue_capacity_and_tickets(ctx):
    from paper_1511_07226_gb300 import pfk
    (r, c), = _requests(1, 12, 12)
    srv = pfk.Server(ctx, workers=1, queue_capacity=2)
    a = srv.submit(c["dims"], c["eta"], c["b"], **KW)
    b = srv.submit(c["dims"], c["eta"], c["b"], **KW)
    with pytest.raises(pfk.PfkError, match="busy"):
        srv.submit(c["dims"], c["eta"], c["b"], **KW)
    xa, _, _ = srv.poll(a)
    xb, _, _ = srv.poll(b)
    assert np.array_equal(xa, xb)
    with pytest.raises(KeyError):
        srv.poll(a)
    # a slot frees once a result is collected
    t = srv.submit(c["dims"], c["eta"], c["b"], **KW)
    assert srv.poll(t) is not None
    srv.close()


def test_pending_poll_and_destroy_with_queued_requests(ctx):
    from paper_1511_07226_gb300 import pfk
    reqs = _requests(4, 40, 48)
    srv = pfk.Server(ctx, workers=1)
    tickets = [srv.submit(c["dims"], c["eta"], c["b"], method="pipefcg", **KW) for r, c in reqs]
    # the last of four sequential solves cannot be done right after submission
    assert srv.poll(tickets[-1], wait_ms=0) is None
    srv.close()   # finishes the active solve, drops the queued ones


def test_csr_requests_and_validation(ctx):
    """General sparse requests (the 64x64 inclusion problem assembled as CSR, with
    Jacobi) served alongside stencil requests equal their solves alone; a CSR
    request with inconsistent row pointers is rejected at submission."""
    from paper_1511_07226_gb300 import pfk
    c = W.poisson2d_inclusions()
    rp, ci, va = _csr_arrays(c)
    srv = pfk.Server(ctx, workers=3)
    (r1, c1), = _requests(1, 20, 20)
    tickets = [srv.submit_csr(rp, ci, va, c["b"], method=m, mmax=30, rtol=1e-8) for m in ("pipefcg", "pipegcr")]
    ts = srv.submit(c1["dims"], c1["eta"], c1["b"], method="pipefcg", **KW)
    got = [srv.poll(t) for t in tickets]
    assert srv.poll(ts)[1]["status_name"] == "ok"
    op = pfk.Operator.csr(ctx, rp, ci, va)
    for (x, info, _), m in zip(got, ("pipefcg", "pipegcr")):
        xa, ia, _ = pfk.solve(ctx, op, pfk.Preconditioner(ctx, op, "jacobi"), c["b"], method=m, mmax=30, rtol=1e-8)
        assert info["status_name"] == ia["status_name"]
        assert info["iterations"] == ia["iterations"]
        assert np.array_equal(x, xa)
    bad = rp.copy()
    bad[-1] += 1
    with pytest.raises(pfk.PfkError, match="row pointers"):
        srv.submit_csr(bad, ci, va, c["b"])
    srv.close()


def _csr_arrays(c):
    csr = O.StencilOperator(c["dims"], c["eta"]).to_csr()
    return csr.rowptr, csr.colidx, csr.vals


def test_smallest_first_order(ctx):
    """PFK_SERVE_SMALLEST_FIRST with one worker and a budget below any
    request's estimate: one solve at a time, so completion order is admission
    order.  The largest request is submitted first (it is admitted at once and
    its solve outlasts the submission of the others); the rest must then run by
    increasing size (equal sizes by arrival).  Every result equals the request
    solved alone."""
    from paper_1511_07226_gb300 import pfk
    reqs = _requests(6, 14, 30)
    big = W.request_problem(dict(side=40, log_contrast=4.0, method=0, item_id=777), ell=4.0)
    reqs = [(dict(side=40, method=0), big)] + reqs
    srv = pfk.Server(ctx, workers=1, memory_budget=1, order="smallest_first", group_max_n=-1)
    t0, tickets = [], []
    for r, c in reqs:
        t0.append(time.perf_counter())
        tickets.append(srv.submit(c["dims"], c["eta"], c["b"], method=METHOD_OF[r["method"]], **KW))
    results = [srv.poll(t) for t in tickets]
    srv.close()
    done = [ts + lat / 1e3 for ts, (_, _, lat) in zip(t0, results)]
    completion = sorted(range(len(reqs)), key=lambda j: done[j])
    expected = [0] + sorted(range(1, len(reqs)), key=lambda j: (reqs[j][0]["side"], j))
    assert completion == expected, (completion, expected)
    for (r, c), (x, info, _) in zip(reqs, results):
        xa, ia = _alone(ctx, c, METHOD_OF[r["method"]], group_max_n=-1)
        assert info["status_name"] == ia["status_name"] == "ok"
        assert np.array_equal(x, xa)


def test_tiny_budget_grouped_requests_one_at_a_time(ctx):
    """The grouped path under the same tiny budget: grouped requests are
    admitted one at a time in arrival order and each equals its grouped solve
    alone."""
    from paper_1511_07226_gb300 import pfk
    reqs = _requests(5, 14, 26)
    srv = pfk.Server(ctx, workers=1, memory_budget=1)
    t0, tickets = [], []
    for r, c in reqs:
        t0.append(time.perf_counter())
        tickets.append(srv.submit(c["dims"], c["eta"], c["b"], method=METHOD_OF[r["method"]], **KW))
    results = [srv.poll(t) for t in tickets]
    srv.close()
    done = [ts + lat / 1e3 for ts, (_, _, lat) in zip(t0, results)]
    assert all(b >= a - 2e-3 for a, b in zip(done, done[1:])), np.diff(done)
    for (r, c), (x, info, _) in zip(reqs, results):
        xa, ia = _alone(ctx, c, METHOD_OF[r["method"]])
        assert info["status_name"] == ia["status_name"] == "ok"
        assert np.array_equal(x, xa)


def test_unknown_order_rejected(ctx):
    """An admission order the library does not know: PFK_ERR_INVALID from
    pfk_server_create itself (raw call), and the binding's name lookup."""
    import ctypes as C
    from paper_1511_07226_gb300 import pfk
    lib = pfk.load()
    p = pfk.ServerParams()
    p.workers, p.order = 1, 2
    h = C.c_void_p()
    assert lib.pfk_server_create(ctx.h, C.byref(p), C.byref(h)) == -1   # PFK_ERR_INVALID
    assert not h.value
    with pytest.raises(KeyError):
        pfk.Server(ctx, order="largest_first")


@pytest.mark.parametrize("method", ["pipefcg", "pipegcr", "pipefgmres"])
def test_served_results_match_oracle(ctx, method):
    """Served solves (4 workers, several requests in flight) against the oracle
    with the protocol of tests/_parity.py: a request of each method on the
    stream's field, contrast 1e2 (small sides), histories from a served run of
    the same request on a fresh server."""
    from oracle import krylov as K
    from oracle import preconditioners as PC
    from paper_1511_07226_gb300 import pfk
    from tests._parity import check_solve, oracle_with_envelope
    reqs = _requests(4, 14, 20)
    c = W.request_problem(dict(side=16, log_contrast=2.0, method=0, item_id=4242), ell=4.0)
    srv = pfk.Server(ctx, workers=4)
    others = [srv.submit(cc["dims"], cc["eta"], cc["b"], method=METHOD_OF[r["method"]], **KW) for r, cc in reqs]
    t = srv.submit(c["dims"], c["eta"], c["b"], method=method, sigma=1.0, **KW)
    x, info, _ = srv.poll(t)
    for o in others:
        srv.poll(o)
    srv.close()
    # the served history is that of the same solve alone (bitwise, tested
    # above); the alone run provides it
    op = pfk.Operator.stencil(ctx, c["dims"], c["eta"])
    if _grouped(c, method):
        xs, ias, hs = pfk.solve_grouped(ctx, [op], [c["b"]], pc_kind="inner_pcg", inner_iters=4, method=method,
                                        sigma=1.0, history=4000, **KW)
        xa, ia, hist = xs[0], ias[0], hs[0]
    else:
        pc = pfk.Preconditioner(ctx, op, "inner_pcg", 4, "fp64")
        xa, ia, hist = pfk.solve(ctx, op, pc, c["b"], method=method, sigma=1.0, history=4000, **KW)
    assert np.array_equal(x, xa) and info["iterations"] == ia["iterations"]
    aop = O.StencilOperator(c["dims"], c["eta"])
    prm = K.Params(mmax=30, rtol=1e-8, maxit=3000, sigma=1.0)
    ref, alts = oracle_with_envelope(method, aop, lambda: PC.InnerPCG(aop, 4), c["b"], prm)
    check_solve(hist, ia, ref, alts, rtol=1e-8)
