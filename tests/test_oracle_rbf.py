"""Pins of the oracle's RBF design matrix (oracle/rbf.py, Sec. 1 / Sec. 4)
against facts that do not come from its own formula."""
import math

import numpy as np

import oracle.rbf as orbf
from paper_0804_4809_gb300 import inputs


def test_centre_on_a_data_point_gives_one():
    rng = np.random.default_rng(1)
    X = rng.uniform(0, 1, (40, 6))
    G = orbf.design(X, X[[3, 17, 29]], 0.3)
    assert G[3, 0] == 1.0 and G[17, 1] == 1.0 and G[29, 2] == 1.0
    assert np.all(G <= 1.0) and np.all(G > 0.0)


def test_symmetric_on_its_own_inputs():
    rng = np.random.default_rng(2)
    X = rng.uniform(0, 1, (30, 4))
    G = orbf.design(X, X, 0.5)
    assert np.array_equal(G, G.T)


def test_one_dimensional_closed_form():
    # distance w: exp(-1/2); distance 2w: exp(-2); distance 3w: exp(-9/2)
    w = 0.25
    X = np.array([[0.0], [w], [2 * w], [3 * w]])
    G = orbf.design(X, np.array([[0.0]]), w)
    want = [1.0, math.exp(-0.5), math.exp(-2.0), math.exp(-4.5)]
    assert np.allclose(G[:, 0], want, rtol=1e-15, atol=0)


def test_distance_is_summed_over_coordinates():
    # |x - c|^2 = 1 + 4 + 9 with w = 1: exp(-7)
    G = orbf.design(np.array([[1.0, 2.0, 3.0]]), np.zeros((1, 3)), 1.0)
    assert abs(G[0, 0] - math.exp(-7.0)) <= 1e-16


def test_matches_the_expanded_form_of_the_input_generator():
    """The generator expands |x|^2 + |c|^2 - 2 x.c (another rounding route);
    the two agree to the cancellation bound of that expansion."""
    G, X, idx = inputs.rbf_design(500, 60, 8, 0.3, seed=3)
    Go = orbf.design(X, X[idx], 0.3)
    # |d2 error| <= ~8 u (|x|^2 + |c|^2) <= 8 u 16, times 1 / (2 w^2) in the exponent
    bound = 8 * 2.0 ** -52 * 16 / (2 * 0.09) * 4
    assert np.max(np.abs(G - Go) / Go) <= bound
