"""GPU parity of the fuzzy neighbour graph (tsne_knn_graph) against the FP64
oracle's own pipeline on the same X (oracle/fuzzy_graph.py: FP64 kNN, rho,
sigma to 1e-12, fuzzy union).

Tolerance, first order in what the GPU is allowed to differ by:
* its bisection stops at |f - log2 k| <= 1e-5, so sigma_i moves by at most
  1e-5 / f'(sigma_i), f'(sigma) = sum_j x_j / sigma^2 exp(-x_j / sigma);
* its distances are square roots of FP32 squared distances (<= 2e-5 relative
  on d^2, so <= 1e-5 relative on d, hence on rho and x_j up to 1e-5 (d_j + rho));
* w = exp(-x / sigma) then moves by w (x / sigma) (dsigma / sigma) + w dx / sigma,
  plus 1e-6 relative for FP32 exp; the union a + c - a c moves by at most
  da + dc.  Values must lie within three times that bound; the pattern is
  integer work and must be identical.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import fuzzy_graph as F
from paper_2605_13928_b300 import _lib as L
from paper_2605_13928_b300 import api, synth

pytestmark = pytest.mark.gpu


def _gpu_graph(X, k, gpu, batch=None, mode=L.TSNE_KNN_BF16_RERANK):
    idx, d2 = api.knn(torch.tensor(X, device=gpu), k, batch=batch, mode=mode)
    st = api.new_status(gpu)
    G, rho, sigma, n_bad = api.knn_graph(idx, d2, batch=batch, status=st)
    torch.cuda.synchronize()
    assert st.item() == 0
    return G, rho.cpu().numpy(), sigma.cpu().numpy(), int(n_bad.item())


def _check(X, k, G, rho, sigma, n_bad, sizes):
    row_ptr, col, val = G.to_numpy()
    off = np.concatenate([[0], np.cumsum(sizes)])
    bad_total = 0
    for s in range(len(sizes)):
        a, b = off[s], off[s + 1]
        (rp_r, col_r, val_r), idx_r, d_r, rho_r, sig_r, flag_r = F.graph(X[a:b], k)
        bad_total += int(flag_r.sum())
        np.testing.assert_allclose(rho[a:b], rho_r, rtol=1e-5, atol=1e-12)
        x = np.maximum(d_r - rho_r[:, None], 0.0)
        ok = sig_r > 0
        sg = np.where(ok, sig_r, 1.0)[:, None]
        e = np.exp(-x / sg)
        fprime = (x / sg ** 2 * e).sum(1)
        dsig = np.where(ok & (fprime > 0), 1e-5 / np.where(fprime > 0, fprime, 1.0), 0.0)
        dx = 1e-5 * (d_r + rho_r[:, None])
        np.testing.assert_array_equal(sigma[a:b] > 0, ok)
        # sigma: the stopping rule, plus the distances' relative error (which
        # rescales sigma with them)
        assert np.all(np.abs(sigma[a:b][ok] - sig_r[ok]) <= 3 * dsig[ok] + 1e-4 * sig_r[ok])
        w = F.weights(d_r, rho_r, sig_r)
        dw = np.where(ok[:, None], w * (x / sg * (dsig[:, None] / sg) + dx / sg + 1e-6), 1e-6)
        # symmetric bound: the union moves by at most dw_ij + dw_ji
        n_s = b - a
        dense = {}
        for i in range(n_s):
            for jj, j in enumerate(idx_r[i]):
                dense[(i, int(j))] = dense.get((i, int(j)), 0.0) + dw[i, jj]
                dense[(int(j), i)] = dense.get((int(j), i), 0.0) + dw[i, jj]
        rp = row_ptr[a:b + 1] - row_ptr[a]
        assert np.array_equal(rp, rp_r)
        seg = slice(row_ptr[a], row_ptr[b])
        assert np.array_equal(col[seg] - a, col_r)
        bound = np.array([dense[(i, int(j))] for i in range(n_s)
                          for j in col_r[rp_r[i]:rp_r[i + 1]]])
        assert np.all(np.abs(val[seg] - val_r) <= 3 * bound + 1e-7), \
            float(np.max(np.abs(val[seg] - val_r) / (3 * bound + 1e-7)))
        assert (val[seg] > 0).all() and (val[seg] <= 1.0 + 1e-6).all()
    assert n_bad == bad_total


@pytest.mark.parametrize("n,d,k", [(2000, 50, 15), (700, 10, 30), (129, 50, 15)])
def test_graph_matches_oracle(gpu, n, d, k):
    X = synth.mixture(n, 8, d=d, seed=synth.SEED_BASE + 300 + n)
    G, rho, sigma, n_bad = _gpu_graph(X, k, gpu)
    _check(X, k, G, rho, sigma, n_bad, [n])


def test_graph_batched_samples(gpu):
    sizes = [300, 1200, 91, 777]
    X = np.concatenate([synth.mixture(s, 5, d=20, seed=synth.SEED_BASE + 320 + i)
                        for i, s in enumerate(sizes)])
    batch = api.Batch(sizes)
    G, rho, sigma, n_bad = _gpu_graph(X, 15, gpu, batch=batch)
    _check(X, 15, G, rho, sigma, n_bad, sizes)


def test_graph_duplicates_take_the_limit(gpu):
    rng = np.random.default_rng(4)
    X = np.concatenate([np.zeros((20, 6)), rng.normal(size=(200, 6))]).astype(np.float32)
    G, rho, sigma, n_bad = _gpu_graph(X, 15, gpu, mode=L.TSNE_KNN_FP32)
    assert n_bad >= 20 and (sigma[:20] == 0).all() and (rho[:20] == 0).all()
    _check(X, 15, G, rho, sigma, n_bad, [len(X)])
    # duplicates are joined with weight 1
    rp, col, val = G.to_numpy()
    for i in range(20):
        row = dict(zip(col[rp[i]:rp[i + 1]].tolist(), val[rp[i]:rp[i + 1]].tolist()))
        assert all(row[j] == 1.0 for j in range(20) if j != i and j in row)


def test_graph_argument_errors(gpu):
    idx = torch.zeros((10, 1), dtype=torch.int32, device=gpu)
    d2 = torch.zeros((10, 1), dtype=torch.float32, device=gpu)
    with pytest.raises(L.TsneError):
        api.knn_graph(idx, d2)  # k < 2
