"""GPU parity of the UMAP layout optimisation (tsne_umap_layout) against the
FP64 oracle (oracle/umap_layout.py), one epoch at a time from the same state.

Both sides take the same FP32 positions and FP32 graph weights and the same
counter-based draws, so every sampling decision and every negative vertex is
the same integer decision on both sides; what differs is arithmetic.  Bound per
point and coordinate: each term is a clipped product of a few FP32 operations
(d^2, the hardware power function __powf, ~1e-7, the coefficient) and the lane sums add up to
deg x (1 + n_neg) terms of magnitude <= 4, so the epoch's sum differs by at
most 1e-5 x 4 x deg x (1 + n_neg) (errors ~1e-6 of each term, generously
rounded up), scaled by alpha_e, plus the FP32 rounding of the updated position.
"""
import numpy as np
import pytest
import torch

from oracle import fuzzy_graph as F
from oracle import umap_layout as U
from paper_2605_13928_b300 import _lib as L
from paper_2605_13928_b300 import api, synth

pytestmark = pytest.mark.gpu

A, B = 1.577, 0.895


def _graph(X, k):
    (rp, col, val), *_ = F.graph(X.astype(np.float64), k)
    return rp.astype(np.int64), col.astype(np.int32), val.astype(np.float32)


def _dev(rp, col, val, gpu):
    return api.CSR.from_numpy(rp, col, val, gpu)


def _bound(rp, Y, alpha, n_neg):
    deg = np.diff(rp).astype(np.float64)
    return alpha * 1e-5 * 4 * deg * (1 + n_neg) + 2.0 ** -22 * np.abs(Y).max(1) + 1e-30


def _one_epoch(G, Y, e, n_epochs, n_neg, seed, gpu, batch=None):
    Yd = torch.tensor(Y, device=gpu)
    st = api.new_status(gpu)
    api.umap_layout(G, Yd, n_epochs=n_epochs, a=A, b=B, n_neg=n_neg, seed=seed, epoch0=e,
                    n_run=1, batch=batch, status=st)
    torch.cuda.synchronize()
    assert st.item() == 0
    return Yd.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("e", [0, 57, 199])
def test_epoch_matches_oracle(gpu, e):
    X = synth.mixture(1500, 6, d=20, seed=synth.SEED_BASE + 400)
    rp, col, val = _graph(X, 15)
    G = _dev(rp, col, val, gpu)
    Y = (np.random.default_rng(40 + e).uniform(-10, 10, size=(1500, 2))).astype(np.float32)
    n_epochs, n_neg, seed = 200, 5, 12345
    got = _one_epoch(G, Y, e, n_epochs, n_neg, seed, gpu)
    ref = U.epoch(rp, col, val, Y.astype(np.float64), e, n_epochs, A, B, 1.0, n_neg, seed)
    err = np.abs(got - ref).max(1)
    alpha = 1.0 - e / n_epochs
    assert np.all(err <= _bound(rp, Y, alpha, n_neg)), float(err.max())
    if e < n_epochs - 1:
        assert np.abs(got - Y).max() > 1e-3  # the epoch moved points


def test_batched_samples_sample_negatives_inside_each_sample(gpu):
    sizes = [400, 1100, 97]
    Xs = [synth.mixture(s, 4, d=10, seed=synth.SEED_BASE + 410 + i) for i, s in enumerate(sizes)]
    parts = [_graph(X, 10) for X in Xs]
    off = np.concatenate([[0], np.cumsum(sizes)])
    rp = np.concatenate([[0]] + [p[0][1:] + sum(len(q[1]) for q in parts[:i])
                                 for i, p in enumerate(parts)]).astype(np.int64)
    col = np.concatenate([p[1] + off[i] for i, p in enumerate(parts)]).astype(np.int32)
    val = np.concatenate([p[2] for p in parts]).astype(np.float32)
    G = _dev(rp, col, val, gpu)
    Y = np.random.default_rng(41).uniform(-5, 5, size=(off[-1], 2)).astype(np.float32)
    batch = api.Batch(sizes)
    got = _one_epoch(G, Y, 3, 50, 7, 99, gpu, batch=batch)
    ref = U.epoch(rp, col, val, Y.astype(np.float64), 3, 50, A, B, 1.0, 7, 99, pt_off=off)
    assert np.all(np.abs(got - ref).max(1) <= _bound(rp, Y, 1.0 - 3 / 50, 7))


def test_runs_are_reproducible_and_split_freely(gpu):
    X = synth.mixture(800, 5, d=8, seed=synth.SEED_BASE + 420)
    rp, col, val = _graph(X, 12)
    G = _dev(rp, col, val, gpu)
    Y0 = torch.tensor(np.random.default_rng(42).uniform(-10, 10, (800, 2)).astype(np.float32),
                      device=gpu)
    outs = []
    for _ in range(2):
        Y = Y0.clone()
        api.umap_layout(G, Y, n_epochs=30, a=A, b=B, seed=5, epoch0=0, n_run=7)
        outs.append(Y)
    Y = Y0.clone()
    for e in range(7):  # the same epochs one call at a time (odd and even buffer parity)
        api.umap_layout(G, Y, n_epochs=30, a=A, b=B, seed=5, epoch0=e, n_run=1)
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], Y)


def test_layout_separates_clusters(gpu):
    """A whole 200-epoch run on 6 well-separated clusters: most 2-D neighbours of a
    point are in its own cluster, and the layout stays finite and bounded."""
    rng = np.random.default_rng(43)
    centres = rng.normal(size=(6, 10)) * 20
    lab = rng.integers(0, 6, 2400)
    X = (centres[lab] + rng.normal(size=(2400, 10))).astype(np.float32)
    Xd = torch.tensor(X, device=gpu)
    idx, d2 = api.knn(Xd, 15)
    G, _, _, _ = api.knn_graph(idx, d2)
    Y = torch.tensor(rng.uniform(-10, 10, (2400, 2)).astype(np.float32), device=gpu)
    st = api.new_status(gpu)
    api.umap_layout(G, Y, n_epochs=200, seed=1, status=st)
    torch.cuda.synchronize()
    assert st.item() == 0
    Yh = Y.cpu().numpy().astype(np.float64)
    assert np.isfinite(Yh).all() and np.abs(Yh).max() < 1e3
    D = ((Yh[:, None, :] - Yh[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(D, np.inf)
    nn = np.argsort(D, axis=1)[:, :10]
    assert (lab[nn] == lab[:, None]).mean() > 0.95


def test_bad_column_sets_status(gpu):
    rp = np.array([0, 1, 2], dtype=np.int64)
    col = np.array([1, 7], dtype=np.int32)  # 7 is outside [0, 2)
    val = np.array([1.0, 1.0], dtype=np.float32)
    G = _dev(rp, col, val, gpu)
    Y = torch.tensor([[0.0, 0.0], [1.0, 1.0]], device=gpu)
    st = api.new_status(gpu)
    api.umap_layout(G, Y, n_epochs=10, a=A, b=B, n_neg=0, n_run=1, status=st)
    torch.cuda.synchronize()
    assert st.item() & L.TSNE_STATUS_BAD_INDEX


def test_degenerate_rows_and_samples(gpu):
    """Rows without entries, a one-point sample (every negative draw is the point
    itself and is skipped) and coincident points, against the oracle."""
    sizes = [1, 6, 3]
    off = np.concatenate([[0], np.cumsum(sizes)])
    # sample 0: the single point with an entry to itself (d = 0: no attraction, and
    # its negatives can only draw the point itself); sample 1: a chain with one empty
    # row; sample 2: two coincident points linked both ways, the third isolated
    rows = [[0], [2], [1, 3], [2], [], [6], [5], [8], [7], []]
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64)
    col = np.array([c for r in rows for c in r], dtype=np.int32)
    val = np.linspace(0.3, 1.0, len(col)).astype(np.float32)
    Y = np.array([[0, 0], [1, 0], [2, 1], [0, 3], [5, 5], [-1, -1], [4, -2], [7, 7], [7, 7],
                  [3, 3]], dtype=np.float32)
    G = _dev(rp, col, val, gpu)
    batch = api.Batch(sizes)
    got = _one_epoch(G, Y, 2, 10, 4, 17, gpu, batch=batch)
    ref = U.epoch(rp, col, val, Y.astype(np.float64), 2, 10, A, B, 1.0, 4, 17, pt_off=off)
    assert np.all(np.abs(got - ref).max(1) <= _bound(rp, Y, 1.0 - 2 / 10, 4))
    assert np.array_equal(got[0], Y[0]) and np.array_equal(got[4], Y[4])  # nothing moves them


@pytest.mark.parametrize("n,k", [(1, 2), (777, 2), (100003, 50)])
def test_umap_init_centres_and_scales_the_scores(gpu, n, k):
    """tsne_umap_init against its definition in FP64 on the host: the first two
    score columns minus their means, times 10 / max |.|; strided rows."""
    S = np.random.default_rng(n).normal(size=(n, k)).astype(np.float32) * 3 + 5
    Sd = torch.tensor(S, device=gpu)
    st = api.new_status(gpu)
    U = api.umap_init(Sd, status=st).cpu().numpy().astype(np.float64)
    torch.cuda.synchronize()
    assert st.item() == 0
    C = S[:, :2].astype(np.float64)
    C = C - C.mean(0)
    ref = C * (10.0 / max(np.abs(C).max(), 1e-30))
    np.testing.assert_allclose(U, ref, rtol=0, atol=1e-5 * 10)
    assert abs(np.abs(U).max() - 10.0) < 1e-5 or n == 1
