"""Pins of the FP64 fuzzy-graph oracle (oracle/fuzzy_graph.py) against facts
fixed by the mathematics: the k = 3 and k = 4 closed forms of the sigma
equation (the latter through a cubic solved by numpy.roots), scale
invariance, the unreachable-target limit, and a hand-worked fuzzy union."""
import math

import numpy as np

from oracle import fuzzy_graph as F


def test_k3_closed_form():
    # d = [r, r + D, r + D]: 1 + 2 exp(-D / sigma) = log2 3
    r, D = 0.7, 0.3
    rho, sigma, flag = F.rho_sigma(np.array([[r, r + D, r + D]]))
    expect = D / math.log(2.0 / (math.log2(3) - 1.0))
    assert flag[0] == 0 and rho[0] == r
    assert abs(sigma[0] - expect) < 1e-10 * expect


def test_k4_cubic():
    # d = [r, r + a, r + 2a, r + 3a]: 1 + q + q^2 + q^3 = 2 with q = exp(-a / sigma)
    r, a = 1.5, 0.2
    rho, sigma, flag = F.rho_sigma(np.array([[r, r + a, r + 2 * a, r + 3 * a]]))
    roots = np.roots([1.0, 1.0, 1.0, -1.0])
    q = float([z.real for z in roots if abs(z.imag) < 1e-12 and z.real > 0][0])
    assert abs(sigma[0] - (-a / math.log(q))) < 1e-9 * sigma[0]


def test_target_reached_scale_invariance_and_weights():
    rng = np.random.default_rng(1)
    d = np.sort(rng.uniform(0.1, 3.0, size=(50, 15)), axis=1)
    rho, sigma, flag = F.rho_sigma(d)
    assert not flag.any()
    w = F.weights(d, rho, sigma)
    np.testing.assert_allclose(w.sum(1), math.log2(15), atol=1e-10)
    np.testing.assert_allclose(w[:, 0], 1.0)  # the nearest neighbour sits at rho
    assert (np.diff(w, axis=1) <= 0).all()
    rho2, sigma2, _ = F.rho_sigma(3.0 * d)
    np.testing.assert_allclose(rho2, 3.0 * rho)
    np.testing.assert_allclose(sigma2, 3.0 * sigma, rtol=1e-9)
    np.testing.assert_allclose(F.weights(3.0 * d, rho2, sigma2), w, atol=1e-9)


def test_unreachable_rows_take_the_limit():
    d = np.array([[0.0, 0.0, 0.0, 1.0, 2.0], [0.0, 0.0, 0.0, 0.0, 0.0]])
    rho, sigma, flag = F.rho_sigma(d)
    assert list(flag) == [1, 1] and list(rho) == [1.0, 0.0]
    w = F.weights(d, rho, sigma)
    np.testing.assert_array_equal(w, [[1, 1, 1, 1, 0], [1, 1, 1, 1, 1]])


def test_fuzzy_union_hand_example():
    idx = np.array([[1], [0], [1]])
    w = np.array([[0.5], [0.25], [0.8]])
    rp, col, val = F.fuzzy_union(idx, w, 3)
    assert list(rp) == [0, 1, 3, 4]
    assert list(col) == [1, 0, 2, 1]
    np.testing.assert_allclose(val, [0.625, 0.625, 0.8, 0.8])


def test_graph_is_symmetric_in_unit_interval():
    rng = np.random.default_rng(2)
    X = rng.normal(size=(200, 5))
    (rp, col, val), idx, d, rho, sigma, flag = F.graph(X, 15)
    n = len(X)
    dense = np.zeros((n, n))
    for i in range(n):
        dense[i, col[rp[i]:rp[i + 1]]] = val[rp[i]:rp[i + 1]]
    np.testing.assert_array_equal(dense, dense.T)
    assert (val > 0).all() and (val <= 1).all()
    assert np.diag(dense).sum() == 0
    # every directed neighbour edge is present, with weight >= its own strength
    w = F.weights(d, rho, sigma)
    for i in range(n):
        for jj, j in enumerate(idx[i]):
            assert dense[i, j] >= w[i, jj] - 1e-15
