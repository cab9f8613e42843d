"""Pins for the oracle's Krylov methods (CPU only).

What fixes each method without another implementation of it:

* dense LU (numpy.linalg.solve) on small systems;
* minimisation over the Krylov subspace, computed by brute force with a dense
  basis: CG-type iterates minimise the A-norm error (Sec. 3.1, eq. cdorth),
  CR-type iterates minimise ||r||_2 (Sec. 4), right-preconditioned GMRES
  iterates minimise ||r||_2 over x0 + M^-1 K_k(A M^-1, r0) (Sec. 5);
* exact-arithmetic invariants that hold for any (nonlinear) preconditioner:
  A-orthogonal directions, r_i orthogonal to the explored space, s = A p,
  w = A u, z = A q, n = A m, A U = P H with orthonormal P;
* equivalences the paper states: PIPEFCG = CG = FCG for a linear preconditioner
  (Sec. 3.2.3), CGFCG = FCG for any B (Sec. 3.2), PIPEFGMRES = FGMRES for a
  linear B (Sec. 5.3);
* finite termination, the B = A^-1 special case, norm-breakdown handling, and
  the toy experiment of Fig. FCGtoy (naive pipelining stagnates near the noise
  level, PIPEFCG does not).
"""
import numpy as np
import pytest

import workloads as W
from oracle import krylov as K
from oracle import operators as O
from oracle import preconditioners as PC

CG_TYPE = ["pcg", "fcg", "cgfcg", "pipefcg", "pipefcg_naive"]
CR_TYPE = ["gcr", "pipegcr", "pipegcr_w"]
GMRES_TYPE = ["fgmres", "cgfgmres", "pipefgmres"]


def _spd_system(n=40, cond=50.0, item=1):
    a = W.random_spd(n, cond=cond, item_id=item)
    return a, O.DenseOperator(a), W.random_vector(n, item)


def _nonsym_system(n=40, item=2):
    a = W.random_nonsym(n, item_id=item)
    return a, O.DenseOperator(a), W.random_vector(n, item)


@pytest.mark.parametrize("method", CG_TYPE + CR_TYPE + GMRES_TYPE)
def test_dense_lu(method):
    if method in CG_TYPE:
        a, A, b = _spd_system()
    else:
        a, A, b = _nonsym_system()
    xs = np.linalg.solve(a, b)
    B = PC.JacobiPC(A)
    r = K.solve(method, A, B, b, prm=K.Params(rtol=1e-13, mmax=40, maxit=400))
    assert r.status == "converged"
    assert np.linalg.norm(r.x - xs) <= 1e-10 * np.linalg.norm(xs) * np.linalg.cond(a)


def _basis(mat, v, k):
    vs, w = [], v.copy()
    for _ in range(k):
        for _ in range(2):
            for q in vs:
                w = w - (q @ w) * q
        vs.append(w / np.linalg.norm(w))
        w = mat @ vs[-1]
    return np.column_stack(vs)


@pytest.mark.parametrize("method", CG_TYPE)
@pytest.mark.parametrize("k", [1, 2, 4, 7])
def test_cg_type_minimises_a_norm_error(method, k):
    a, A, b = _spd_system(n=30, cond=30.0, item=3)
    dinv = 1.0 / np.diag(a)
    xs = np.linalg.solve(a, b)
    V = _basis(dinv[:, None] * a, dinv * b, k)
    xk = V @ np.linalg.solve(V.T @ a @ V, V.T @ b)
    r = K.solve(method, A, PC.JacobiPC(A), b, prm=K.Params(rtol=0.0, mmax=30, maxit=k))
    assert r.iterations == k
    assert np.linalg.norm(r.x - xk) <= 1e-9 * np.linalg.norm(xs)


@pytest.mark.parametrize("method", CR_TYPE)
@pytest.mark.parametrize("k", [1, 2, 4, 7])
def test_cr_type_minimises_residual(method, k):
    a, A, b = _nonsym_system(n=30, item=4)
    dinv = 1.0 / np.diag(a)
    V = _basis(dinv[:, None] * a, dinv * b, k)
    y = np.linalg.lstsq(a @ V, b, rcond=None)[0]
    r = K.solve(method, A, PC.JacobiPC(A), b, prm=K.Params(rtol=0.0, mmax=30, maxit=k, norm="unpreconditioned"))
    assert r.iterations == k
    assert np.linalg.norm(r.x - V @ y) <= 1e-9 * np.linalg.norm(np.linalg.solve(a, b))


@pytest.mark.parametrize("method", GMRES_TYPE)
@pytest.mark.parametrize("k", [1, 2, 4, 7])
def test_gmres_type_minimises_residual(method, k):
    a, A, b = _nonsym_system(n=30, item=5)
    dinv = 1.0 / np.diag(a)
    V = _basis(a * dinv[None, :], b, k)            # K_k(A M^-1, r0)
    y = np.linalg.lstsq(a @ (dinv[:, None] * V), b, rcond=None)[0]
    xk = dinv * (V @ y)
    r = K.solve(method, A, PC.JacobiPC(A), b, prm=K.Params(rtol=0.0, mmax=30, maxit=k, sigma=2.0))
    assert r.iterations == k
    assert np.linalg.norm(r.x - xk) <= 1e-9 * np.linalg.norm(np.linalg.solve(a, b))
    # the history's last entry is the least-squares residual of x_k
    assert np.isclose(r.history[-1]["rho"], np.linalg.norm(b - a @ xk), rtol=1e-8)


def _stencil_problem(dims=(6, 5, 4), item=6, contrast=2.0):
    c = W.poisson3d_gaussian(dims=dims, ell=2.0, log_contrast=contrast, config_id=901, item_id=item)
    op = O.StencilOperator(c["dims"], c["eta"])
    return op, c["b"]


def test_fcg_invariants_with_nonlinear_preconditioner():
    """Full orthogonalisation: A-orthogonal p's, r_i orthogonal to them, CD minimisation."""
    op, b = _stencil_problem()
    a = op.to_dense()
    xs = np.linalg.solve(a, b)
    B = PC.InnerPCG(op, 2)
    r = K.solve("fcg", op, B, b, prm=K.Params(rtol=0.0, mmax=200, maxit=12, trace=True))
    for t in r.trace[3:]:
        ps = [t["window"][k] for k in sorted(t["window"])]
        for k, pk in enumerate(ps[:-1]):
            c = (ps[-1] @ a @ pk) / np.sqrt((ps[-1] @ a @ ps[-1]) * (pk @ a @ pk))
            assert abs(c) < 1e-8
            assert abs(t["r"] @ pk) <= 1e-9 * max(np.linalg.norm(t["r"]), 1e-6 * np.linalg.norm(b)) * \
                np.linalg.norm(pk)
        P = np.column_stack(ps[:-1])
        xk = P @ np.linalg.solve(P.T @ a @ P, P.T @ b)
        assert np.linalg.norm(t["x"] - xk) <= 1e-8 * np.linalg.norm(xs)


def test_cgfcg_equals_fcg_for_nonlinear_preconditioner():
    op, b = _stencil_problem(item=7)
    prm = K.Params(rtol=1e-10, mmax=10)
    h1 = K.solve("fcg", op, PC.InnerPCG(op, 2), b, prm=prm).rho()
    h2 = K.solve("cgfcg", op, PC.InnerPCG(op, 2), b, prm=prm).rho()
    k = min(len(h1), len(h2), 20)
    assert np.allclose(h1[:k], h2[:k], rtol=1e-8, atol=1e-14 * h1[0])


@pytest.mark.parametrize("naive", [False, True])
def test_pipefcg_recurrence_invariants_nonlinear(naive):
    """s = A p, w = A u, z = A q, n = A m, eta = <p, A p>, r = b - A x and A-orthogonality.

    Drift is measured against the largest norm each quantity takes in the run, since
    the recurred vectors shrink by orders of magnitude as the solve converges.
    """
    op, b = _stencil_problem(item=8)
    a = op.to_dense()
    B = PC.InnerPCG(op, 3)
    r = K.pipefcg(op, B, b, np.zeros_like(b), K.Params(rtol=0.0, mmax=200, maxit=15, trace=True), naive=naive)
    scale = {k: max(np.linalg.norm(t[k]) for t in r.trace) for k in ("s", "w", "z", "n")}
    for t in r.trace:
        assert np.linalg.norm(t["s"] - a @ t["p"]) <= 1e-10 * scale["s"]
        assert np.linalg.norm(t["w"] - a @ t["u"]) <= 1e-10 * scale["w"]
        assert np.linalg.norm(t["z"] - a @ t["q"]) <= 1e-10 * scale["z"]
        assert np.linalg.norm(t["n"] - a @ t["m"]) <= 1e-12 * scale["n"]
        assert np.linalg.norm(t["r"] - (b - a @ t["x"])) <= 1e-10 * np.linalg.norm(b)
        if t["i"] <= 8:
            assert np.isclose(t["eta"], t["p"] @ a @ t["p"], rtol=1e-6)
            for k, pk in t["window"].items():
                if k < t["i"]:
                    c = (t["p"] @ a @ pk) / np.sqrt((t["p"] @ a @ t["p"]) * (pk @ a @ pk))
                    assert abs(c) < 1e-6


@pytest.mark.parametrize("method", ["pipegcr", "pipegcr_w"])
def test_pipegcr_recurrence_invariants_nonlinear(method):
    op, b = _stencil_problem(item=9)
    a = op.to_dense()
    B = PC.InnerPCG(op, 3)
    r = K.solve(method, op, B, b, prm=K.Params(rtol=0.0, mmax=200, maxit=15, trace=True,
                                               norm="unpreconditioned"))
    scale = {k: max(np.linalg.norm(t[k]) for t in r.trace) for k in ("s", "w")}
    for t in r.trace:
        assert np.linalg.norm(t["s"] - a @ t["p"]) <= 1e-10 * scale["s"]
        assert np.linalg.norm(t["w"] - a @ t["u"]) <= 1e-10 * scale["w"]
        if t["z"] is not None:
            zs = max(np.linalg.norm(tt["z"]) for tt in r.trace)
            assert np.linalg.norm(t["z"] - a @ t["q"]) <= 1e-10 * zs
        assert np.linalg.norm(t["r"] - (b - a @ t["x"])) <= 1e-10 * np.linalg.norm(b)
        if t["i"] <= 8:
            assert np.isclose(t["eta"], t["s"] @ t["s"], rtol=1e-6)
            for k, sk in t["window_s"].items():
                if k < t["i"]:
                    assert abs(t["s"] @ sk) <= 1e-6 * np.linalg.norm(t["s"]) * np.linalg.norm(sk)


def test_gcr_minimal_residual_nonlinear():
    op, b = _stencil_problem(item=10)
    a = op.to_dense()
    r = K.solve("gcr", op, PC.InnerPCG(op, 2), b,
                prm=K.Params(rtol=0.0, mmax=200, maxit=20, trace=True, norm="unpreconditioned"))
    rn = r.rho()
    assert np.all(np.diff(rn) <= 1e-12 * rn[0])
    for t in r.trace[2:]:
        P = np.column_stack([t["window"][k] for k in sorted(t["window"]) if k < t["i"]])
        y = np.linalg.lstsq(a @ P, b, rcond=None)[0]
        assert np.linalg.norm(t["x"] - P @ y) <= 1e-8 * np.linalg.norm(np.linalg.solve(a, b))


@pytest.mark.parametrize("method", ["cgfgmres", "pipefgmres"])
def test_fgmres_arnoldi_relation_nonlinear(method):
    """A U = P H with orthonormal P for any B; x minimises ||b - A x|| over x0 + span(U)."""
    op, b = _stencil_problem(item=11)
    a = op.to_dense()
    r = K.solve(method, op, PC.InnerPCG(op, 3), b,
                prm=K.Params(rtol=0.0, mmax=12, maxit=12, sigma=1.5, trace=True))
    t = r.trace[0]
    k = t["ncols"]
    # the cycle stops at column m-1 without forming p_m: check the first m-1 columns
    U = np.column_stack(t["U"][:k - 1])
    Pm = np.column_stack(t["P"][:k])
    H = t["H"][:k, :k - 1]
    assert np.linalg.norm(a @ U - Pm @ H) <= 1e-9 * np.linalg.norm(a @ U)
    # classical Gram-Schmidt loses orthogonality once the residual is tiny: check the
    # columns built while the residual estimate is still above 1e-6 of its start
    k_ok = sum(1 for h in r.history[1:] if h["rho"] > 1e-6 * r.history[0]["rho"])
    k_ok = max(2, min(k_ok, k))
    assert np.linalg.norm(Pm[:, :k_ok].T @ Pm[:, :k_ok] - np.eye(k_ok)) <= 1e-8
    U = np.column_stack(t["U"][:k])
    y = np.linalg.lstsq(a @ U, b, rcond=None)[0]
    assert np.linalg.norm(r.x - U @ y) <= 1e-8 * np.linalg.norm(np.linalg.solve(a, b))


@pytest.mark.parametrize("method", ["fcg", "cgfcg", "pipefcg", "pipefcg_naive"])
def test_linear_pc_equals_pcg_history(method):
    op, b = _stencil_problem(item=12, contrast=1.0)
    prm = K.Params(rtol=1e-9, mmax=30)
    ref = K.solve("pcg", op, PC.JacobiPC(op), b, prm=prm).rho()
    got = K.solve(method, op, PC.JacobiPC(op), b, prm=prm).rho()
    k = min(len(ref), len(got), 25)
    assert np.allclose(got[:k], ref[:k], rtol=1e-9, atol=1e-14 * ref[0])


@pytest.mark.parametrize("method", ["cgfgmres", "pipefgmres"])
def test_linear_pc_equals_fgmres_history(method):
    op, b = _stencil_problem(item=13, contrast=1.0)
    prm = K.Params(rtol=1e-9, mmax=30, sigma=1.0)
    ref = K.solve("fgmres", op, PC.JacobiPC(op), b, prm=prm).rho()
    got = K.solve(method, op, PC.JacobiPC(op), b, prm=prm).rho()
    k = min(len(ref), len(got), 20)
    assert np.allclose(got[:k], ref[:k], rtol=1e-8, atol=1e-14 * ref[0])


def test_pipegcr_linear_pc_equals_gcr_and_is_monotone():
    op, b = _stencil_problem(item=14, contrast=1.0)
    prm = K.Params(rtol=1e-9, mmax=30, norm="unpreconditioned")
    ref = K.solve("gcr", op, PC.JacobiPC(op), b, prm=prm).rho()
    for method in ("pipegcr", "pipegcr_w"):
        got = K.solve(method, op, PC.JacobiPC(op), b, prm=prm).rho()
        k = min(len(ref), len(got), 20)
        assert np.allclose(got[:k], ref[:k], rtol=1e-8, atol=1e-14 * ref[0])
        assert np.all(np.diff(got[:k]) <= 1e-12 * got[0])


@pytest.mark.parametrize("method", ["fcg", "pipefcg", "fgmres", "pipefgmres"])
def test_finite_termination(method):
    n = 24
    a, A, b = _spd_system(n=n, cond=20.0, item=15)
    r = K.solve(method, A, PC.JacobiPC(A), b, prm=K.Params(rtol=1e-8, mmax=n + 2, maxit=200, sigma=1.0))
    assert r.status == "converged"
    assert r.iterations <= n + 2


def test_exact_preconditioner_one_step():
    a, A, b = _spd_system(n=20, item=16)
    B = PC.DensePC(np.linalg.inv(a))
    r = K.solve("pipefcg", A, B, b, prm=K.Params(rtol=1e-10, mmax=5))
    assert np.isclose(r.history[0]["alpha"], 1.0, rtol=1e-12)
    assert r.status == "converged" and r.iterations == 1


def test_breakdown_detected_and_reported():
    d = np.concatenate([np.linspace(1.0, 2.0, 10), -np.linspace(1.0, 2.0, 10)])
    A = O.DiagonalOperator(d)
    b = np.ones(20)
    r = K.solve("pipefcg", A, PC.IdentityPC(), b, prm=K.Params(rtol=1e-10, mmax=5, max_restarts=3))
    assert r.status == "breakdown"
    assert r.breakdowns >= 1 or r.history[0]["eta"] <= 0


def test_breakdown_restart_counting():
    """Indefinite A: eta_i <= 0 is detected mid-solve, each breakdown restarts from x_i,
    and the solve ends with status "breakdown" once max_restarts is exhausted."""
    a, A, b = _spd_system(n=30, cond=10.0, item=17)
    d = np.linalg.eigvalsh(a)
    shifted = O.DenseOperator(a - (d[0] + 0.5 * (d[1] - d[0])) * np.eye(30))   # one negative eigenvalue
    for method in ("fcg", "pipefcg"):
        r = K.solve(method, shifted, PC.IdentityPC(), b, prm=K.Params(rtol=1e-8, mmax=40, max_restarts=3))
        assert r.status == "breakdown"
        assert r.breakdowns == 4 and r.restarts == 3
        assert r.history[0]["eta"] > 0                  # the first fill itself was fine


@pytest.mark.parametrize("eta_noise", [1e-2, 1e-4])
@pytest.mark.parametrize("seed", range(5))
def test_toy_noise_experiment(eta_noise, seed):
    """Fig. FCGtoy: n = 100, kappa = 5, b = 1/sqrt(n), nu_max = n, B(r) = r + eta ||r|| xi
    (parameters read from tests/golden/toy_experiment.txt)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "toy_experiment.txt")
    g = dict(ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#"))
    t = W.toy_diagonal(n=int(g["n"]), kappa=float(g["condition_number"]))
    assert np.allclose(t["b"], float(g["b_entry"]))
    assert np.isclose(t["diag"].max() / t["diag"].min(), float(g["condition_number"]))
    A = O.DiagonalOperator(t["diag"])
    b = t["b"]
    xs = b / t["diag"]
    best = {}
    for m in ("fcg", "pipefcg", "pipefcg_naive"):
        B = PC.NoisyPC(eta_noise, W.noise_bank(100, 500, seed_item=seed))
        r = K.solve(m, A, B, b, prm=K.Params(mmax=int(g["nu_max"]), rtol=0.0, maxit=60,
                                            true_residual_check=False, trace=True))
        errs = [np.linalg.norm(tr["x"] - xs) / np.linalg.norm(xs) for tr in r.trace]
        best[m] = (min(errs), errs[-1])
    assert best["fcg"][0] <= 1e-2 * eta_noise
    assert best["pipefcg"][0] <= 1e-2 * eta_noise
    assert 0.1 * eta_noise <= best["pipefcg_naive"][0] <= 10 * eta_noise


def test_truncation_rules():
    prm = K.Params(mmax=3)
    assert [K.nu_window(i, prm) for i in range(1, 8)] == [1, 2, 3, 3, 3, 3, 3]
    prm = K.Params(mmax=3, truncation="restart")
    assert [K.nu_window(i, prm) for i in range(1, 8)] == [1, 2, 3, 1, 2, 3, 1]


def test_sigma_estimate_approaches_largest_eigenvalue():
    """Power iteration on A B: for a symmetric A with B = D^-1 the estimate tends to
    the largest eigenvalue of A D^-1 (checked against numpy.linalg.eigvals)."""
    op, b = _stencil_problem(item=18, contrast=1.0)
    a = op.to_dense()
    lam = np.abs(np.linalg.eigvals(a / np.diag(a)[None, :])).max()
    est = K.estimate_sigma(op, PC.JacobiPC(op), b, iters=200)
    assert abs(est - lam) <= 1e-3 * lam
    assert K.estimate_sigma(op, PC.JacobiPC(op), b) <= lam * (1 + 1e-12)


@pytest.mark.parametrize("method", ["fcg", "pipefcg", "gcr", "pipegcr", "pipegcr_w"])
def test_true_residual_stagnation_is_not_convergence(method):
    """A goal below the attainable accuracy: the recurred residual keeps falling
    but ||b - A x|| stalls at rounding level, so after max_restarts residual
    replacements the solve reports "stagnated" (x is the last iterate)."""
    c = W.poisson2d_inclusions(16, 16)
    A = O.StencilOperator(c["dims"], c["eta"])
    r = K.solve(method, A, PC.JacobiPC(A), c["b"], prm=K.Params(mmax=10, rtol=1e-18, max_restarts=2, maxit=2000))
    assert r.status == "stagnated"
    assert r.restarts == 2 and r.replacements >= 1
    rel = r.rnorm_true / r.bnorm
    assert 1e-18 < rel < 1e-13
    # with an attainable goal the same solve converges
    r2 = K.solve(method, A, PC.JacobiPC(A), c["b"], prm=K.Params(mmax=10, rtol=1e-10, max_restarts=2))
    assert r2.status == "converged" and r2.rnorm_true <= 1e-10 * r2.bnorm


def test_theta_projection_reduces_to_alg8_and_alg7():
    """eq. (proj): m_i = theta tilde-u_i + B(w_i - theta r_i).  With a linear B
    every theta gives B(w_i) + theta (tilde-u_i - B(r_i)) = B(w_i) (tilde-u_i =
    B(r_i) in exact arithmetic), so the theta variant equals Alg. 8 and CG; and
    the computed theta_i is <r_i, w_i> / <r_i, r_i> of the run's own vectors."""
    a, A, b = _spd_system(n=30, cond=30.0, item=11)
    prm = K.Params(rtol=0.0, mmax=30, maxit=12, trace=True)
    r8 = K.pipefcg(A, PC.JacobiPC(A), b, np.zeros_like(b), prm)
    rt = K.pipefcg(A, PC.JacobiPC(A), b, np.zeros_like(b), prm, theta=True)
    xs = np.linalg.solve(a, b)
    for t8, tt in zip(r8.trace, rt.trace):
        assert np.linalg.norm(tt["x"] - t8["x"]) <= 1e-10 * np.linalg.norm(xs)


def test_theta_projection_with_nonlinear_b():
    """With the noisy B of Fig. FCGtoy (B ~ I) the theta variant converges like
    Alg. 8, unlike Alg. 7; theta_i = <r_i, A tilde-u_i> / <r_i, r_i> is then a
    Rayleigh quotient of A (eigenvalues 1..5), not 1 (theta tends to 1 only as
    B tends to A^-1)."""
    t = W.toy_diagonal()
    A = O.DiagonalOperator(t["diag"])
    xs = t["b"] / t["diag"]
    bank = W.noise_bank(100, 500, seed_item=7)
    r = K.solve("pipefcg_theta", A, PC.NoisyPC(1e-3, bank), t["b"],
                prm=K.Params(mmax=32, rtol=0.0, maxit=60, true_residual_check=False, trace=True))
    err = min(np.linalg.norm(tr["x"] - xs) / np.linalg.norm(xs) for tr in r.trace)
    assert err <= 1e-6
    for tr in r.trace[:10]:
        th = (tr["r"] @ tr["w"]) / (tr["r"] @ tr["r"])
        assert 0.9 < th < 5.1


def test_theta_projection_step_replay():
    """Each m_i of the theta variant with a deterministic nonlinear B (inner PCG)
    equals theta_i tilde-u_i + B(w_i - theta_i r_i), theta_i = <r_i, w_i> / <r_i, r_i>
    recomputed from the trace; a wrong theta (e.g. 1, or <r, w> / <w, w>) fails."""
    op, b = _stencil_problem(item=12)
    B = PC.InnerPCG(op, 2)
    r = K.solve("pipefcg_theta", op, B, b, prm=K.Params(rtol=0.0, mmax=10, maxit=8, trace=True))
    for tr in r.trace[1:]:
        th = float(np.dot(tr["r"], tr["w"]) / np.dot(tr["r"], tr["r"]))
        m = th * tr["u"] + PC.InnerPCG(op, 2)(tr["w"] - th * tr["r"])
        assert np.linalg.norm(m - tr["m"]) <= 1e-12 * np.linalg.norm(m)
        m1 = tr["u"] + PC.InnerPCG(op, 2)(tr["w"] - tr["r"])
        assert np.linalg.norm(m1 - tr["m"]) > 1e-6 * np.linalg.norm(m)
