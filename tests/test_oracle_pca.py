"""Pins of the FP64 PCA oracle against facts fixed by the mathematics, not by
re-running its own formulas: a matrix built from a known singular value
decomposition, the 2-D closed form, the variance-maximising direction found by
brute-force search, and invariants (orthogonal scores, trace, exact
reconstruction, translation / scaling / row-permutation behaviour)."""
import math

import numpy as np
import pytest

from oracle import pca as O


def _orthonormal(rng, m, r, centred=False):
    G = rng.normal(size=(m, r))
    if centred:
        G -= G.mean(axis=0)  # columns orthogonal to the ones vector
    Q, _ = np.linalg.qr(G)
    return Q


@pytest.mark.parametrize("n,g,r", [(400, 30, 6), (90, 120, 12), (1000, 64, 64)])
def test_known_svd_is_recovered(n, g, r):
    rng = np.random.default_rng(n + g)
    U = _orthonormal(rng, n, r, centred=True)
    V = _orthonormal(rng, g, r)
    S = np.sort(rng.uniform(1.0, 50.0, size=r))[::-1] + np.arange(r, 0, -1) * 0.5
    m = rng.normal(size=g) * 3.0
    A = U @ np.diag(S) @ V.T + m[None, :]
    k = min(r, 10)
    out = O.pca(A, k)
    np.testing.assert_allclose(out["mean"], m, atol=1e-12)
    np.testing.assert_allclose(out["sigma"], S[:k], rtol=1e-11)
    np.testing.assert_allclose(out["explained_variance"], S[:k] ** 2 / (n - 1), rtol=1e-11)
    np.testing.assert_allclose(out["total_var"], (S ** 2).sum() / (n - 1), rtol=1e-11)
    np.testing.assert_allclose(out["ratio"], S[:k] ** 2 / (S ** 2).sum(), rtol=1e-11)
    for c in range(k):
        s = np.sign(out["components"][c] @ V[:, c])
        np.testing.assert_allclose(out["components"][c], s * V[:, c], atol=1e-10)
        np.testing.assert_allclose(out["scores"][:, c], s * S[c] * U[:, c], atol=1e-9)


def test_two_dimensional_closed_form():
    rng = np.random.default_rng(3)
    n = 257
    A = rng.normal(size=(n, 2)) @ np.array([[2.0, 0.7], [0.0, 0.5]]) + np.array([5.0, -1.0])
    # scatter entries summed row by row, then the 2 x 2 symmetric eigen closed form
    mx = sum(A[i, 0] for i in range(n)) / n
    my = sum(A[i, 1] for i in range(n)) / n
    a = sum((A[i, 0] - mx) ** 2 for i in range(n))
    c = sum((A[i, 1] - my) ** 2 for i in range(n))
    b = sum((A[i, 0] - mx) * (A[i, 1] - my) for i in range(n))
    root = math.sqrt(((a - c) / 2) ** 2 + b * b)
    l1, l2 = (a + c) / 2 + root, (a + c) / 2 - root
    th = 0.5 * math.atan2(2 * b, a - c)
    v1 = np.array([math.cos(th), math.sin(th)])
    if v1[0 if abs(v1[0]) >= abs(v1[1]) else 1] < 0:  # largest entry positive
        v1 = -v1
    out = O.pca(A, 2)
    np.testing.assert_allclose(out["sigma"] ** 2, [l1, l2], rtol=1e-12)
    np.testing.assert_allclose(out["components"][0], v1, atol=1e-12)
    np.testing.assert_allclose(out["mean"], [mx, my], rtol=1e-13)


def test_first_axis_maximises_projected_variance_brute_force():
    rng = np.random.default_rng(11)
    A = rng.normal(size=(300, 2)) @ np.array([[1.0, 0.9], [0.2, 0.4]])
    Ac = A - A.mean(axis=0)
    th = np.linspace(0.0, math.pi, 200001)
    var = ((Ac[:, :1] * np.cos(th)[None, :] + Ac[:, 1:] * np.sin(th)[None, :]) ** 2).sum(axis=0)
    best = th[np.argmax(var)]
    v = O.pca(A, 1)["components"][0]
    ang = math.atan2(v[1], v[0]) % math.pi
    assert abs(ang - best) < 2e-5
    assert abs(var.max() - O.pca(A, 1)["sigma"][0] ** 2) < 1e-8 * var.max()


def test_invariants():
    rng = np.random.default_rng(5)
    n, g = 500, 40
    A = rng.normal(size=(n, g)) @ rng.normal(size=(g, g)) * 0.3 + rng.normal(size=g)
    full = O.pca(A, g)
    T, V = full["scores"], full["components"]
    # orthogonal scores with squared norms lambda, orthonormal axes
    np.testing.assert_allclose(T.T @ T, np.diag(full["sigma"] ** 2),
                               atol=1e-8 * full["sigma"][0] ** 2)
    np.testing.assert_allclose(V @ V.T, np.eye(g), atol=1e-12)
    # the eigenvalues sum to the total variance; reconstruction is exact at k = g
    np.testing.assert_allclose((full["sigma"] ** 2).sum() / (n - 1), full["total_var"], rtol=1e-12)
    np.testing.assert_allclose(full["mean"][None, :] + T @ V, A, atol=1e-10)
    # descending order and the sign convention
    assert np.all(np.diff(full["sigma"]) <= 0)
    for row in V:
        j = np.argmax(np.abs(row))
        assert row[j] > 0
    k = 7
    base = O.pca(A, k)
    # translation: same axes and scores; scaling: sigma scales, axes unchanged
    tr = O.pca(A + rng.normal(size=g)[None, :] * 10, k)
    np.testing.assert_allclose(tr["components"], base["components"], atol=1e-9)
    np.testing.assert_allclose(tr["scores"], base["scores"], atol=1e-8)
    sc = O.pca(-2.5 * A, k)
    np.testing.assert_allclose(sc["sigma"], 2.5 * base["sigma"], rtol=1e-11)
    np.testing.assert_allclose(sc["components"], base["components"], atol=1e-9)
    # row permutation permutes the scores only
    p = rng.permutation(n)
    pr = O.pca(A[p], k)
    np.testing.assert_allclose(pr["components"], base["components"], atol=1e-9)
    np.testing.assert_allclose(pr["scores"], base["scores"][p], atol=1e-8)
    # transform of the fitted rows reproduces the scores
    np.testing.assert_allclose(O.transform(A, base["mean"], base["components"]), base["scores"],
                               atol=1e-9)


def test_sign_fix_tie_takes_lowest_index():
    V = np.array([[0.5, -0.5, 0.1], [-0.3, 0.3, 0.0], [0.0, 0.0, 0.0]])
    W, s = O.sign_fix(V)
    assert list(s) == [1.0, -1.0, 1.0]
    np.testing.assert_array_equal(W[1], [0.3, -0.3, -0.0])
