"""Pins of the FP64 CPU oracle against facts fixed by the mathematics.

Each test checks the oracle against something other than itself: a brute-force
definition written differently (full sort, dense matrices), a closed form, an
invariant, or a hand-worked example under tests/golden/.  The readings of the
textbook t-SNE definitions are listed in the oracle's C header.
"""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _mix(n, d, seed, scale=3.0):
    rng = np.random.default_rng(seed)
    c = rng.normal(0, scale, size=(4, d))
    return c[rng.integers(0, 4, n)] + rng.normal(size=(n, d))


# ----------------------------------------------------------------------------- kNN
@pytest.mark.parametrize("n,d,k", [(60, 5, 7), (33, 3, 32), (2, 4, 1)])
def test_knn_equals_full_sort(n, d, k):
    X = _mix(n, d, n)
    idx, d2 = oracle.knn(X, k)
    D = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    for i in range(n):
        j = np.array([j for j in range(n) if j != i])
        order = np.lexsort((j, D[i, j]))[:k]
        assert np.array_equal(idx[i], j[order])
        np.testing.assert_allclose(d2[i], D[i, j[order]], rtol=1e-13, atol=0)


def test_knn_ties_and_duplicates_break_by_index():
    # integer grid with duplicated points: many exact distance ties
    g = np.array([[a, b] for a in range(3) for b in range(3)], dtype=np.float64)
    X = np.concatenate([g, g[:3]])
    idx, d2 = oracle.knn(X, 6)
    D = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    for i in range(len(X)):
        j = np.array([j for j in range(len(X)) if j != i])
        order = np.lexsort((j, D[i, j]))[:6]
        assert np.array_equal(idx[i], j[order])
    assert d2[9, 0] == 0.0 and idx[9, 0] == 0  # duplicate of point 0 found first


def test_knn_row_subset_matches_full():
    X = _mix(80, 6, 3)
    full_i, full_d = oracle.knn(X, 9)
    rows = np.array([0, 17, 79, 40])
    sub_i, sub_d = oracle.knn(X, 9, rows=rows)
    assert np.array_equal(sub_i, full_i[rows])
    assert np.array_equal(sub_d, full_d[rows])


# ------------------------------------------------------------------- calibration
def test_calibration_hits_perplexity_and_gibbs_form():
    X = _mix(300, 10, 1)
    idx, d2 = oracle.knn(X, 45)
    pc, beta, flag = oracle.calibrate(d2, 15.0)
    assert (flag == 0).all()
    np.testing.assert_allclose(pc.sum(1), 1.0, rtol=0, atol=1e-13)
    H = -(pc * np.log(pc)).sum(1)
    assert np.abs(np.exp(H) / 15.0 - 1).max() < 1e-10
    # p_j / p_0 = exp(-beta (d_j - d_0)) for every row
    lhs = np.log(pc) - np.log(pc[:, :1])
    rhs = -beta[:, None] * (d2 - d2[:, :1])
    np.testing.assert_allclose(lhs, rhs, rtol=1e-9, atol=1e-9)


def test_calibration_k2_closed_form():
    # two neighbours at distances 0 and delta: p1 = 1/(1+exp(-beta delta)) and the binary
    # entropy h(p1) = log(perp); solve h(p) = log perp on p in (1/2, 1) by bisection here.
    perp = 1.5
    target = np.log(perp)

    def h(p):
        return -p * np.log(p) - (1 - p) * np.log(1 - p)

    lo, hi = 0.5, 1 - 1e-15
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if h(mid) > target else (lo, mid)
    p_star = 0.5 * (lo + hi)
    for delta in (0.25, 1.0, 7.0):
        pc, beta, flag = oracle.calibrate(np.array([[3.0, 3.0 + delta]]), perp)
        assert flag[0] == 0
        assert abs(pc[0, 0] - p_star) < 1e-10
        assert abs(beta[0] - np.log(p_star / (1 - p_star)) / delta) < 1e-8 / delta


def test_cond_at_beta_reproduces_calibrated_rows():
    X = _mix(100, 6, 12)
    _, d2 = oracle.knn(X, 20)
    pc, beta, _ = oracle.calibrate(d2, 7.0)
    np.testing.assert_allclose(oracle.cond_at_beta(d2, beta), pc, rtol=1e-12, atol=0)
    # k = 2 closed form at an arbitrary beta: p1 = 1 / (1 + exp(-beta * delta))
    p = oracle.cond_at_beta(np.array([[1.0, 1.5]]), np.array([3.0]))
    assert abs(p[0, 0] - 1 / (1 + np.exp(-1.5))) < 1e-15
    u = oracle.cond_at_beta(np.array([[2.0, 2.0, 3.0]]), np.array([np.inf]))
    np.testing.assert_array_equal(u[0], [0.5, 0.5, 0.0])


def test_calibration_unreachable_rows_are_flagged_uniform():
    d2 = np.array([[2.0] * 8,                       # all equal: H = log 8 for every beta
                   [1.0, 1.0, 1.0, 1.0, 5.0, 6.0, 7.0, 8.0]])  # 4 ties >= perplexity 3
    pc, beta, flag = oracle.calibrate(d2, 3.0)
    assert flag.tolist() == [1, 1]
    np.testing.assert_array_equal(pc[0], np.full(8, 1 / 8))
    np.testing.assert_array_equal(pc[1], [0.25] * 4 + [0.0] * 4)


# ---------------------------------------------------------------- symmetrisation
def test_symmetrize_equals_dense_definition():
    n, k = 40, 6
    X = _mix(n, 4, 5)
    idx, d2 = oracle.knn(X, k)
    pc, _, _ = oracle.calibrate(d2, 3.0)
    P = oracle.symmetrize(idx, pc)
    C = np.zeros((n, n))
    for i in range(n):
        C[i, idx[i]] = pc[i]
    np.testing.assert_allclose(P.dense(), (C + C.T) / (2 * n), rtol=1e-15, atol=1e-18)
    assert abs(P.val.sum() - 1) < 1e-12
    assert n * k <= P.nnz <= 2 * n * k
    for i in range(n):
        c = P.col[P.row_ptr[i]:P.row_ptr[i + 1]]
        assert (np.diff(c) > 0).all() and i not in c


# ------------------------------------------------------------ Z, KL and gradient
def test_Z_closed_forms():
    Y = np.zeros((7, 2))
    assert oracle.Z(Y) == 7 * 6  # coincident points: every w = 1
    a, b, D = 3, 5, 2.5  # two coincident groups a distance D apart
    Y = np.concatenate([np.zeros((a, 2)), np.tile([[D, 0.0]], (b, 1))])
    expect = a * (a - 1) + b * (b - 1) + 2 * a * b / (1 + D * D)
    assert abs(oracle.Z(Y) - expect) < 1e-12 * expect


def _random_P(n, k, seed):
    X = _mix(n, 5, seed)
    P, *_ = oracle.affinities(X, k, k / 3)
    return P


def test_kl_equals_definition_p_log_p_over_q():
    P = _random_P(50, 9, 11)
    Y = np.random.default_rng(2).normal(size=(50, 2))
    D = ((Y[:, None] - Y[None]) ** 2).sum(-1)
    W = 1 / (1 + D)
    np.fill_diagonal(W, 0)
    Q = W / W.sum()
    Pd = P.dense()
    m = Pd > 0
    kl_def = (Pd[m] * np.log(Pd[m] / Q[m])).sum()
    assert abs(oracle.kl(P, Y, 1.0) - kl_def) < 1e-12
    assert kl_def > 0


@pytest.mark.parametrize("alpha", [1.0, 12.0])
def test_gradient_central_finite_differences(alpha):
    n = 40
    P = _random_P(n, 9, 3)
    Y = np.random.default_rng(4).normal(size=(n, 2))
    g, _ = oracle.grad(P, Y, alpha)
    h = 1e-6
    fd = np.zeros_like(Y)
    for i in range(n):
        for c in range(2):
            Yp = Y.copy(); Yp[i, c] += h
            Ym = Y.copy(); Ym[i, c] -= h
            fd[i, c] = (oracle.kl(P, Yp, alpha) - oracle.kl(P, Ym, alpha)) / (2 * h)
    assert np.linalg.norm(fd - g) / np.linalg.norm(g) < 1e-7


def test_gradient_two_points_closed_form():
    P = oracle.CSR(np.array([0, 1, 2]), np.array([1, 0]), np.array([0.5, 0.5]))
    Y = np.array([[0.3, -1.2], [2.0, 0.7]])
    r = Y[0] - Y[1]
    w = 1 / (1 + r @ r)
    for alpha in (1.0, 4.0, 12.0):
        g, Z = oracle.grad(P, Y, alpha)
        expect = 4 * (alpha * 0.5 - 0.5) * w * r
        np.testing.assert_allclose(g[0], expect, rtol=1e-14, atol=1e-15)
        np.testing.assert_allclose(g[1], -expect, rtol=1e-14, atol=1e-15)
        assert abs(Z - 2 * w) < 1e-15


def test_gradient_vanishes_when_P_equals_Q():
    n = 25
    Y = np.random.default_rng(7).normal(size=(n, 2))
    D = ((Y[:, None] - Y[None]) ** 2).sum(-1)
    W = 1 / (1 + D)
    np.fill_diagonal(W, 0)
    P = oracle.CSR.from_dense(W / W.sum())
    g, _ = oracle.grad(P, Y, 1.0)
    assert np.abs(g).max() < 1e-14
    assert abs(oracle.kl(P, Y, 1.0)) < 1e-13
    g12, _ = oracle.grad(P, Y, 12.0)
    assert np.abs(g12).max() > 1e-3


def test_gradient_rigid_motion_invariances():
    n = 60
    P = _random_P(n, 12, 8)
    Y = np.random.default_rng(9).normal(size=(n, 2)) * 3
    g, _ = oracle.grad(P, Y, 12.0)
    assert np.abs(g.sum(0)).max() < 1e-12 * np.abs(g).sum()
    g_t, _ = oracle.grad(P, Y + np.array([5.0, -2.0]), 12.0)
    np.testing.assert_allclose(g_t, g, rtol=1e-9, atol=1e-13)
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    g_r, _ = oracle.grad(P, Y @ R.T, 12.0)
    np.testing.assert_allclose(g_r, g @ R.T, rtol=1e-9, atol=1e-13)


def test_force_split_matches_gradient():
    n = 70
    P = _random_P(n, 12, 10)
    Y = np.random.default_rng(1).normal(size=(n, 2)) * 2
    g, Z = oracle.grad(P, Y, 5.0)
    Fa, Fr, Zi = oracle.forces_rows(P, Y)
    assert abs(Zi.sum() - Z) < 1e-12 * Z
    np.testing.assert_allclose(4 * (5.0 * Fa - Fr / Z), g, rtol=1e-10, atol=1e-14)


def test_force_magnitude_sums_closed_forms():
    """Aa_i = sum_j p_ij w_ij |y_i - y_j| and Ar_i = sum_j w_ij^2 |y_i - y_j|:
    points 1, 2, 3 on a line to one side of point 0 push it the same way, so
    |Fr_0| = Ar_0 = 1/4 + 2/25 + 3/100 = 0.36 (w = 1/2, 1/5, 1/10); a point
    midway between two others has Fr = 0 but Ar = 2 (1/4); the triangle
    inequality bounds every row."""
    Y = np.array([[0.0, 0.0], [1.0, 0.0], [2.0, 0.0], [3.0, 0.0]])
    P = oracle.CSR(np.array([0, 2, 3, 4, 4]), np.array([1, 2, 0, 0]),
                   np.array([0.1, 0.2, 0.1, 0.2]))
    Fa, Fr, Zi, Aa, Ar = oracle.forces_rows(P, Y, scales=True)
    assert abs(Ar[0] - 0.36) < 1e-15 and abs(abs(Fr[0, 0]) - Ar[0]) < 1e-15
    assert abs(Aa[0] - (0.1 * 0.5 * 1 + 0.2 * 0.2 * 2)) < 1e-15
    assert abs(abs(Fa[0, 0]) - Aa[0]) < 1e-15
    Y3 = np.array([[-1.0, 0.0], [0.0, 0.0], [1.0, 0.0]])
    P3 = oracle.CSR(np.zeros(4, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0))
    _, Fr3, _, Aa3, Ar3 = oracle.forces_rows(P3, Y3, rows=np.array([1]), scales=True)
    assert np.abs(Fr3).max() == 0.0 and abs(Ar3[0] - 0.5) < 1e-15 and Aa3[0] == 0.0
    n = 90
    Pr = _random_P(n, 10, 8)
    Yr = np.random.default_rng(4).normal(size=(n, 2)) * 3
    Fa, Fr, _, Aa, Ar = oracle.forces_rows(Pr, Yr, scales=True)
    assert np.all(np.hypot(Fa[:, 0], Fa[:, 1]) <= Aa * (1 + 1e-12))
    assert np.all(np.hypot(Fr[:, 0], Fr[:, 1]) <= Ar * (1 + 1e-12))
    Fa2, Fr2, Zi2 = oracle.forces_rows(Pr, Yr)
    np.testing.assert_array_equal(Fa, Fa2)
    np.testing.assert_array_equal(Fr, Fr2)


# ------------------------------------------------------------------------- optimiser
def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                key, v = line.split()
                vals[key] = float(v)
    return vals


def test_optimiser_two_point_hand_worked_trajectory():
    gold = _golden("two_point_trajectory.txt")
    P = oracle.CSR(np.array([0, 1, 2]), np.array([1, 0]), np.array([0.5, 0.5]))
    Y0 = np.array([[1.0, 0.0], [-1.0, 0.0]])
    for steps, key in ((1, "y1x_after_1"), (2, "y1x_after_2"), (3, "y1x_after_3")):
        Y, U, G, tr = oracle.run(P, Y0, n_iter=steps, ee_iters=2, ee=12.0, mom0=0.5, mom1=0.8,
                                 eta=1 / 6, kl_every=1)
        assert abs(Y[0, 0] - gold[key]) < 1e-14
        assert abs(Y[1, 0] + gold[key]) < 1e-14
        assert np.abs(Y[:, 1]).max() == 0.0
        assert np.abs(tr).max() < 1e-15  # p = q = 1/2 for N = 2
    assert abs(U[0, 0] - gold["u1x_after_3"]) < 1e-14
    np.testing.assert_allclose(G, gold["gain_after_3"], rtol=1e-15)
