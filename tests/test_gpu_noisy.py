"""The noisy preconditioner of the paper's toy experiment (Sec. 3.2, Fig. FCGtoy)
on the GPU: B(r) = r + eta ||r|| xi_j / ||xi_j|| with the noise bank as an
input, so the oracle draws the same rows.  Checks the application sequence
element by element and the experiment itself: naive pipelining (Alg. 7)
stagnates near the noise level, PIPEFCG (Alg. 8) and FCG do not."""
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


def _diag_operator(ctx, diag):
    from paper_1511_07226_gb300 import pfk
    n = len(diag)
    return pfk.Operator.csr(ctx, np.arange(n + 1), np.arange(n), diag)


def test_noisy_sequence_matches_oracle(ctx):
    from paper_1511_07226_gb300 import pfk
    n, count = 1000, 7
    bank = W.noise_bank(n, count, seed_item=3)
    op = _diag_operator(ctx, np.linspace(1.0, 2.0, n))
    pc = pfk.Preconditioner.noisy(ctx, op, 1e-2, bank)
    ref = PC.NoisyPC(1e-2, bank)
    for j in range(10):     # wraps around the bank
        v = W.random_vector(n, item_id=j)
        got = pc.apply(v).cpu().numpy()
        want = ref(v)
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-15 * np.abs(want).max())


def test_noisy_bank_validation(ctx):
    from paper_1511_07226_gb300 import pfk
    op = _diag_operator(ctx, np.ones(10))
    bank = np.ones((3, 10))
    bank[1] = 0.0
    with pytest.raises(pfk.PfkError, match="zero norm"):
        pfk.Preconditioner.noisy(ctx, op, 1e-2, bank)
    with pytest.raises(pfk.PfkError, match="eta"):
        pfk.Preconditioner.noisy(ctx, op, -1.0, np.ones((2, 10)))


@pytest.mark.parametrize("eta_noise", [1e-2, 1e-4])
@pytest.mark.parametrize("seed", [0, 1])
def test_toy_experiment(ctx, eta_noise, seed):
    """n = 100, kappa = 5, b = 1/sqrt(n), nu_max = 32 (the library's maximum;
    the paper uses n), 60 iterations."""
    from paper_1511_07226_gb300 import pfk
    t = W.toy_diagonal()
    xs = t["b"] / t["diag"]
    op = _diag_operator(ctx, t["diag"])
    bank = W.noise_bank(100, 500, seed_item=seed)
    err = {}
    for m in ("fcg", "pipefcg", "pipefcg_naive"):
        pc = pfk.Preconditioner.noisy(ctx, op, eta_noise, bank)
        x, info, hist = pfk.solve(ctx, op, pc, t["b"], method=m, mmax=32, rtol=0.0, maxit=60,
                                  true_residual_check=False, history=200)
        pc.close()
        # rtol = 0: the run ends at maxit, or earlier with a norm breakdown or a
        # natural norm of exactly zero once the recurrences are at rounding
        # level or, for Alg. 7, noise-driven -- there the trajectory depends on
        # rounding alone, on either side, so only the error level is compared
        assert info["status_name"] in ("not_converged", "breakdown", "ok")
        assert info["iterations"] == 60 or info["status_name"] != "not_converged"
        err[m] = np.linalg.norm(x - xs) / np.linalg.norm(xs)
        ref = K.solve(m, O.DiagonalOperator(t["diag"]), PC.NoisyPC(eta_noise, bank), t["b"],
                      prm=K.Params(mmax=32, rtol=0.0, maxit=60, true_residual_check=False))
        ref_err = np.linalg.norm(ref.x - xs) / np.linalg.norm(xs)
        # same outcome class as the oracle
        assert (err[m] <= 1e-2 * eta_noise) == (ref_err <= 1e-2 * eta_noise), (m, err[m], ref_err)
    assert err["fcg"] <= 1e-2 * eta_noise
    assert err["pipefcg"] <= 1e-2 * eta_noise
    assert 0.1 * eta_noise <= err["pipefcg_naive"] <= 10 * eta_noise


def test_noisy_pipefcg_trajectory_parity(ctx):
    """Rho history of PIPEFCG with the noisy B against the oracle's (envelope protocol)."""
    from paper_1511_07226_gb300 import pfk
    t = W.toy_diagonal()
    bank = W.noise_bank(100, 500, seed_item=4)
    op = _diag_operator(ctx, t["diag"])
    aop = O.DiagonalOperator(t["diag"])
    prm = K.Params(mmax=32, rtol=1e-10, maxit=200)
    ref, alts = oracle_with_envelope("pipefcg", aop, lambda: PC.NoisyPC(1e-3, bank), t["b"], prm)
    pc = pfk.Preconditioner.noisy(ctx, op, 1e-3, bank)
    x, info, hist = pfk.solve(ctx, op, pc, t["b"], method="pipefcg", mmax=32, rtol=1e-10, maxit=200, history=400)
    check_solve(hist, info, ref, alts, rtol=1e-10)


def test_theta_variant_toy_and_trajectory(ctx):
    """eq. (proj) variant with the noisy B: converges like Alg. 8 (error <= 1e-2 eta
    after 60 iterations) and follows the oracle's trajectory (envelope protocol)."""
    from paper_1511_07226_gb300 import pfk
    t = W.toy_diagonal()
    xs = t["b"] / t["diag"]
    bank = W.noise_bank(100, 500, seed_item=5)
    op = _diag_operator(ctx, t["diag"])
    pc = pfk.Preconditioner.noisy(ctx, op, 1e-3, bank)
    x, info, _ = pfk.solve(ctx, op, pc, t["b"], method="pipefcg_theta", mmax=32, rtol=0.0, maxit=60,
                           true_residual_check=False)
    pc.close()
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-5
    aop = O.DiagonalOperator(t["diag"])
    prm = K.Params(mmax=32, rtol=1e-10, maxit=200)
    ref, alts = oracle_with_envelope("pipefcg_theta", aop, lambda: PC.NoisyPC(1e-3, bank), t["b"], prm)
    pc = pfk.Preconditioner.noisy(ctx, op, 1e-3, bank)
    x, info, hist = pfk.solve(ctx, op, pc, t["b"], method="pipefcg_theta", mmax=32, rtol=1e-10, maxit=200,
                              history=400)
    check_solve(hist, info, ref, alts, rtol=1e-10)
