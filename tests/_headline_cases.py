"""The oracle envelopes of the headline-regime parity tests
(tests/test_gpu_headline.py), shared with the script that stores them
(tests/golden/make_oracle_envelopes.py).

Each case: the workload generator and its arguments, the method, the
preconditioner, the oracle parameters and the summation orders of its
envelope (the first is the reference run).
"""
ALL_ORDERS = ("numpy", "pairwise", "reversed", "fsum", "fma", "rowsum")
FAST_ORDERS = ("numpy", "pairwise", "reversed", "fma")
SIGMA_256 = 1.0


def field(n: int) -> dict:
    """The config-2 field at n^3 with the correlation length scaled to the grid."""
    return {"gen": "poisson3d_gaussian", "kw": {"n": n, "ell": 8.0 * n / 128.0, "log_contrast": 3.0}}


CASES = {}
for _m in ("pipefcg", "pipegcr"):
    for _n in (32, 48):
        # iteration cap 5000: a rounding that makes the solve stagnate ends
        # there ("maxit"), and the outcome is then not compared (the
        # alternative runs disagree on it)
        CASES[f"{_m}_{_n}"] = dict(problem=field(_n), method=_m, pc=("inner_pcg", {"k": 4}),
                                   prm=dict(mmax=30, rtol=1e-8, maxit=5000, max_restarts=200),
                                   orders=ALL_ORDERS, big=False)
    CASES[f"{_m}_128_first100"] = dict(problem={"gen": "poisson3d_gaussian", "kw": {"n": 128}}, method=_m,
                                       pc=("inner_pcg", {"k": 4}), prm=dict(mmax=30, rtol=1e-8, maxit=100),
                                       orders=FAST_ORDERS, big=True)
CASES["pipefgmres_256_cheb_first10"] = dict(problem={"gen": "poisson3d_two_phase", "kw": {}}, method="pipefgmres",
                                            pc=("chebyshev", {"k": 8}),
                                            prm=dict(mmax=30, rtol=1e-8, sigma=SIGMA_256, maxit=10),
                                            orders=FAST_ORDERS, big=True)
