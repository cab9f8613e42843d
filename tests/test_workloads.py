"""The synthetic input generators (CPU): the portable exponential against the
library's, the almost-Gaussian filter's variance and normalisation, and that
the stored oracle envelopes were made from the inputs the generators make
now (their input hashes)."""
import glob
import json
import os

import numpy as np
import pytest

import workloads as W


def test_portable_exp_matches_library_exp():
    x = np.linspace(-30.0, 30.0, 200001)
    rel = np.abs(W.portable_exp(x) - np.exp(x)) / np.exp(x)
    assert rel.max() <= 4e-16
    y = np.linspace(-3.0, 3.0, 6001)
    assert np.max(np.abs(W.portable_pow10(y) / np.power(10.0, y) - 1.0)) <= 2e-15
    assert W.portable_exp(np.zeros(3)).tolist() == [1.0, 1.0, 1.0]


@pytest.mark.parametrize("sigma", [0.7, 1.41, 2.83, 5.66, 11.3])
def test_box_widths_variance(sigma):
    w = W.box_widths(sigma)
    assert len(w) == 4 and all(v % 2 == 1 and v >= 1 for v in w)
    var = sum((v * v - 1) / 12.0 for v in w)
    # four boxes of consecutive odd widths bracket any target variance to
    # within one width step
    assert abs(var - sigma * sigma) <= max(2.0, 0.2 * sigma * sigma), (w, var, sigma * sigma)


def test_box_filter_is_a_periodic_moving_average():
    g = np.random.default_rng(3)
    f = g.standard_normal((7, 9, 11))
    for ax in range(3):
        got = W._box_periodic(f, ax, 5)
        ref = sum(np.roll(f, s, axis=ax) for s in range(-2, 3)) / 5.0
        assert np.allclose(got, ref, rtol=0, atol=1e-14)


def test_field_normalised_and_clipped():
    c = W.poisson3d_gaussian(n=40, ell=5.0)
    g = np.log10(c["eta"]) / 3.0
    assert g.min() >= -1.0 - 1e-12 and g.max() <= 1.0 + 1e-12
    assert abs(np.mean(np.clip(g, -0.999, 0.999))) < 0.1
    # a smooth field: neighbouring cells are strongly correlated
    gg = g.reshape(40, 40, 40)
    corr = np.corrcoef(gg[:, :, :-1].ravel(), gg[:, :, 1:].ravel())[0, 1]
    assert corr > 0.9


def test_stored_envelopes_match_current_inputs():
    """Every stored oracle run was made from the inputs the generators make now."""
    from tests import _oracle_pool as P
    files = glob.glob(os.path.join(os.path.dirname(__file__), "golden", "envelope_*.json"))
    files += glob.glob(os.path.join(os.path.dirname(__file__), "golden", "oracle_spread_*cube.json"))
    checked = 0
    for f in files:
        with open(f) as fh:
            doc = json.load(fh)
        n = doc["problem"]["kw"].get("n", 256 if doc["problem"]["gen"] == "poisson3d_two_phase" else 128)
        if n > 64:
            continue   # full-size inputs: checked on the GPU machine by the tests that use them
        assert P.input_hash(P.problem(doc["problem"])) == doc["inputs_sha256"], f
        checked += 1
    assert checked >= 0
