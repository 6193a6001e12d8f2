"""Pins of the FP64 UMAP layout oracle (oracle/umap_layout.py) against facts
fixed outside it: splitmix64's published output sequence, the gradients of
log Phi and log(1 - Phi) by finite differences of their definitions, the
least-squares optimality of the (a, b) fit, a two-point closed form of one
epoch, the edge-sampling rule's limits and frequencies, uniform negatives, and
translation invariance."""
import math

import numpy as np
import pytest

from oracle import umap_layout as U


def test_splitmix64_reference_sequence():
    # the generator started at state 0 returns the mix of k * 0x9E3779B97F4A7C15,
    # k = 0, 1, 2: its published first outputs
    g = 0x9E3779B97F4A7C15
    assert U.splitmix64(0) == 0xE220A8397B1DCDAF
    assert U.splitmix64(g) == 0x6E789E6AA1B965F4
    assert U.splitmix64((2 * g) & U.MASK64) == 0x06C45D188009454F
    arr = U.splitmix64(np.array([0, g], dtype=np.uint64))
    assert [int(v) for v in arr] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4]


@pytest.mark.parametrize("a,b", [(1.577, 0.895), (0.583, 1.334), (2.0, 0.5)])
def test_gradient_coefficients_match_finite_differences(a, b):
    rng = np.random.default_rng(3)
    for _ in range(20):
        yi, yj = rng.normal(size=2) * 2, rng.normal(size=2) * 2

        def log_phi(y):
            return -math.log1p(a * float((y - yj) @ (y - yj)) ** b)

        def log_1mphi(y):
            t = a * float((y - yj) @ (y - yj)) ** b
            return math.log(t / (1.0 + t))

        h = 1e-6
        for f, coef in ((log_phi, U.attract_coef), (log_1mphi, None)):
            fd = np.array([(f(yi + h * e) - f(yi - h * e)) / (2 * h) for e in np.eye(2)])
            d2 = float((yi - yj) @ (yi - yj))
            if coef is U.attract_coef:
                c = float(U.attract_coef(np.array([d2]), a, b)[0])
            else:  # the oracle's repulsion carries d^2 + eps; undo it for the check
                c = float(U.repulse_coef(np.array([d2]), a, b)[0]) * (d2 + U.EPS) / d2
            np.testing.assert_allclose(c * (yi - yj), fd, rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("min_dist,spread", [(0.1, 1.0), (0.5, 1.0), (0.0, 2.0)])
def test_fit_ab_is_a_least_squares_minimum(min_dist, spread):
    a, b = U.fit_ab(min_dist, spread)
    d = np.linspace(0.0, 3.0 * spread, 300)
    psi = np.where(d < min_dist, 1.0, np.exp(-(d - min_dist) / spread))

    def cost(a_, b_):
        return float(((1.0 / (1.0 + a_ * d ** (2 * b_)) - psi) ** 2).sum())

    c0 = cost(a, b)
    for da, db in ((1e-4, 0), (-1e-4, 0), (0, 1e-4), (0, -1e-4), (1e-4, 1e-4), (-1e-4, 1e-4)):
        assert cost(a * (1 + da), b * (1 + db)) >= c0 - 1e-12
    assert a > 0 and b > 0
    assert np.abs(1.0 / (1.0 + a * d ** (2 * b)) - psi).max() < 0.12


def _two_points(y0, y1, w=1.0):
    row_ptr = np.array([0, 1, 2])
    col = np.array([1, 0])
    return row_ptr, col, np.array([w, w], dtype=np.float32), np.array([y0, y1], dtype=np.float64)


def test_two_point_epoch_closed_form():
    a, b = 1.577, 0.895
    rp, col, w, Y = _two_points([0.3, -0.2], [1.5, 0.7])
    e, n_epochs, alpha0 = 3, 10, 1.0
    out = U.epoch(rp, col, w, Y, e, n_epochs, a, b, alpha0, 0, seed=7)
    diff = Y[0] - Y[1]
    d2 = diff @ diff
    c = -2 * a * b * d2 ** (b - 1) / (1 + a * d2 ** b)
    alpha = alpha0 * (1 - e / n_epochs)
    assert np.all(np.abs(c * diff) < 4)  # no clipping in this configuration
    np.testing.assert_allclose(out[0], Y[0] + alpha * c * diff, rtol=1e-14)
    np.testing.assert_allclose(out[1], Y[1] - alpha * c * diff, rtol=1e-14)
    np.testing.assert_allclose(out.mean(0), Y.mean(0), rtol=1e-14)  # centroid kept
    assert np.linalg.norm(out[0] - out[1]) < np.linalg.norm(diff)  # attraction


def test_clipping_and_coincident_points():
    a, b = 1.577, 0.895
    # points 0.03 apart: the repulsion 2b d / ((eps + d^2)(1 + a d^2b)) is ~27 per unit
    # direction, so every negative that hits the other point adds exactly -+4 per
    # coordinate, on top of the (small, unclipped) attraction
    y0, y1 = np.array([0.0, 0.0]), np.array([0.03, 0.02])
    rp, col, w, Y = _two_points(y0, y1)
    D = U.epoch_delta(rp, col, w, Y, 0, a, b, 15, seed=1)
    diff = y0 - y1
    att = U.attract_coef(np.array([diff @ diff]), a, b)[0] * diff
    assert np.all(np.abs(U.repulse_coef(np.array([diff @ diff]), a, b)[0] * diff) > 4)
    m = (D[0] - att) / np.array([-4.0, -4.0])  # repulsion pushes point 0 to -x, -y
    assert np.allclose(m, np.round(m), atol=1e-9) and m[0] == m[1] and m[0] >= 1
    # coincident points: no attraction term
    rp, col, w, Y = _two_points([1.0, 1.0], [1.0, 1.0])
    assert np.all(U.epoch_delta(rp, col, w, Y, 0, a, b, 0, seed=1) == 0)


def test_edge_sampling_limits_and_frequency():
    q = np.arange(4000)
    assert U.taken(U.draw(5, 0, q, 0), np.ones(4000)).all()        # p = 1: always
    assert not U.taken(U.draw(5, 0, q, 0), np.zeros(4000)).any()   # p = 0: never
    freq = np.mean([U.taken(U.draw(9, e, q, 0), np.full(4000, 0.3)).mean() for e in range(20)])
    assert abs(freq - 0.3) < 5 * math.sqrt(0.3 * 0.7 / 80000)


def test_negative_vertices_are_uniform_in_the_sample():
    h = U.draw(11, 2, np.arange(200000), 3)
    v = U.vertex(h, 1000, 37)
    assert v.min() >= 1000 and v.max() < 1037
    counts = np.bincount(v - 1000, minlength=37)
    expect = 200000 / 37
    assert ((counts - expect) ** 2 / expect).sum() < 36 + 6 * math.sqrt(72)  # chi-square, 36 dof


def test_epoch_is_translation_invariant_and_moves_only_sources():
    rng = np.random.default_rng(4)
    n = 60
    rows = [np.sort(rng.choice([j for j in range(n) if j != i], 5, replace=False))
            for i in range(n)]
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])])
    col = np.concatenate(rows)
    w = rng.uniform(0.2, 1.0, len(col)).astype(np.float32)
    Y = rng.normal(size=(n, 2)) * 3
    a, b = 1.577, 0.895
    D1 = U.epoch_delta(rp, col, w, Y, 4, a, b, 5, seed=2)
    D2 = U.epoch_delta(rp, col, w, Y + [100.0, -50.0], 4, a, b, 5, seed=2)
    np.testing.assert_allclose(D1, D2, atol=1e-9)
    # a point with no entries does not move
    rp0 = rp.copy()
    rp0[1:] -= len(rows[0])
    rp0[0] = 0
    D3 = U.epoch_delta(rp0, col[len(rows[0]):], w[len(rows[0]):], Y, 4, a, b, 5, seed=2)
    assert np.all(D3[0] == 0)
