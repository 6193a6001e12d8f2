"""Parity at the full atlas size (N = 1,000,000, 50-D, k = 90, perplexity 30) in
the launch configuration bench.py times (BF16 tcgen05 kNN, AUTO repulsion =
symmetric split with 1024-point groups), on outputs the FP64 oracle can
compute row by row, plus properties that hold at any size:

* kNN of 200 sampled rows against the oracle's brute force over all 1M
  points (sets equal modulo ties within 1e-6 of the k-th distance);
* beta of those rows against the oracle's calibration of its own distances
  (within the GPU's stopping rule, as in the small affinity tests);
* P symmetric on the sampled rows, sum(P) = 1;
* with an empty P, -Z g / 4 = F_r: the GPU's repulsive forces of 200 sampled
  rows against the oracle's exact FP64 sums over all 1M points (1e-4
  relative L2, and 3e-4 of each row's term-magnitude sum), and Z >= the
  sampled rows' own sums, for the default split and its fixed-point form, on
  a Gaussian cloud and on host-generated clumped and spread layouts;
* one full optimiser step (AUTO variant) with the real P: no status bit,
  finite result, gradient sum ~ 0 (translation invariance);
* the whole gradient 4 (alpha F_a - F_r / Z) at 1M with a host-generated P of the
  benchmark's shape (90 entries per row, neighbours near in index): 200 sampled
  rows against the oracle's F_a and exact F_r, with the exact FP64 Z of all
  pairs, at alpha = 12 and 1;
* PCA at 1M x 2000 by properties of the exact answer (see the test);
* one UMAP layout epoch at 1M points (~24 entries per row, 5 negatives, the
  benchmarked launch): 200 sampled rows against the oracle's per-row update.
"""
import threading

import numpy as np
import pytest
import torch

import oracle
from paper_2605_13928_b300 import _lib as L
from paper_2605_13928_b300 import api, synth
from problems import ROW_TOL, record, row_err_scaled

pytestmark = pytest.mark.gpu

ROWS = 200


@pytest.fixture(scope="module")
def atlas(gpu):
    wl = synth.WORKLOADS["atlas_n1m"]
    X = wl.data()
    Xd = torch.tensor(X, device=gpu)
    st = api.new_status(gpu)
    idx, d2 = api.knn(Xd, wl.k, mode=L.TSNE_KNN_BF16_RERANK, status=st)
    P, beta, n_bad = api.affinities(idx, d2, wl.perplexity, status=st)
    torch.cuda.synchronize()
    assert st.item() == 0
    rows = np.sort(np.random.default_rng(11).choice(wl.n, ROWS, replace=False))
    return wl, X, idx, d2, P, beta, int(n_bad.item()), rows


def test_knn_rows_at_full_size(atlas):
    wl, X, idx, d2, P, beta, n_bad, rows = atlas
    X64 = X.astype(np.float64)
    idx_r, d2_r = oracle.knn(X64, wl.k, rows=rows)
    gi, gd = idx[rows].cpu().numpy(), d2[rows].cpu().numpy()
    record("knn_bf16/atlas_n1m/200_rows",
           neighbours_differing=sum(len(set(a.tolist()) - set(b.tolist())) for a, b in zip(gi, idx_r)))
    for r, i in enumerate(rows):
        assert i not in gi[r] and len(set(gi[r].tolist())) == wl.k
        np.testing.assert_allclose(gd[r], ((X64[gi[r]] - X64[i]) ** 2).sum(1), rtol=1e-5)
        sg, sr = set(gi[r].tolist()), set(idx_r[r].tolist())
        dk = d2_r[r, -1]
        for j in sg - sr:
            assert ((X64[j] - X64[i]) ** 2).sum() <= dk * (1 + 1e-6)
        for j in sr - sg:
            assert ((X64[j] - X64[i]) ** 2).sum() >= dk * (1 - 1e-6)


def test_calibration_rows_at_full_size(atlas):
    wl, X, idx, d2, P, beta, n_bad, rows = atlas
    assert n_bad == 0
    _, d2_r = oracle.knn(X.astype(np.float64), wl.k, rows=rows)
    pc_r, beta_r, flag_r = oracle.calibrate(d2_r, wl.perplexity)
    assert not flag_r.any()
    s = d2_r - d2_r.min(1, keepdims=True)
    E = (pc_r * s).sum(1)
    var = (pc_r * (s - E[:, None]) ** 2).sum(1)
    dbeta = 1e-5 / (beta_r * var)  # the GPU's stopping rule, 1e-5 nats
    bg = beta.cpu().numpy()[rows].astype(np.float64)
    record("affinities/atlas_n1m/200_rows", beta_max_rel=np.max(np.abs(bg - beta_r) / beta_r),
           beta_max_over_bound=np.max(np.abs(bg - beta_r) / (3 * dbeta + 3e-5 * beta_r)))
    assert np.all(np.abs(bg - beta_r) <= 3 * dbeta + 3e-5 * beta_r)


def test_P_symmetric_and_normalised_at_full_size(atlas):
    wl, X, idx, d2, P, beta, n_bad, rows = atlas
    rp, col, val = P.to_numpy()
    assert abs(val.astype(np.float64).sum() - 1.0) < 1e-5
    assert wl.n * wl.k <= len(col) <= 2 * wl.n * wl.k
    for i in rows:
        for e in range(rp[i], rp[i + 1]):
            j = col[e]
            seg = col[rp[j]:rp[j + 1]]
            f = np.searchsorted(seg, i)
            assert f < len(seg) and seg[f] == i and val[rp[j] + f] == val[e]


STATES = {
    # a plain Gaussian cloud, std 30
    "gauss30": lambda n: (np.random.default_rng(12).normal(size=(n, 2)) * 30).astype(np.float32),
    # clumped, like early exaggeration: 100 Zipf-sized clusters of std 0.05 whose
    # centres lie within a few units, so the forces of many near-coincident points
    # nearly cancel
    "clumped": lambda n: synth.embedding_state(n, 100, 2.0, 0.05, seed=16),
    # spread, like late iterations: centres std 40, clusters std 2, so w spans
    # about eight orders of magnitude
    "spread": lambda n: synth.embedding_state(n, 100, 40.0, 2.0, seed=17),
}


@pytest.mark.parametrize("state", list(STATES))
@pytest.mark.parametrize("variant", [L.TSNE_VARIANT_AUTO, L.TSNE_VARIANT_SYM4_FX])
def test_repulsion_rows_at_full_size(atlas, gpu, variant, state):
    """AUTO (the benchmarked split) and the fixed-point form, on host-generated
    states: F_r of the sampled rows to 1e-4 relative L2 and, row by row, to 3e-4
    of the row's term-magnitude sum Ar_i (problems.ROW_TOL)."""
    wl = atlas[0]
    n = wl.n
    Y = STATES[state](n)
    Pe = api.CSR(torch.zeros(n + 1, dtype=torch.int64, device=gpu),
                 torch.zeros(1, dtype=torch.int32, device=gpu),
                 torch.zeros(1, dtype=torch.float32, device=gpu))
    g, Z, _ = api.kl_grad(Pe, torch.tensor(Y, device=gpu), 1.0,
                          params=L.default_params(variant=variant))
    rows = atlas[7]
    Pempty = oracle.CSR(np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32),
                        np.zeros(0))
    _, Fr, Zi, _, Ar = oracle.forces_rows(Pempty, Y.astype(np.float64), rows, scales=True)
    Fr_gpu = -g.cpu().numpy()[rows].astype(np.float64) * Z.item() / 4.0
    l2, re = np.linalg.norm(Fr_gpu - Fr) / np.linalg.norm(Fr), row_err_scaled(Fr_gpu - Fr, Ar)
    record(f"repulsion/atlas_n1m/variant{variant}/{state}", Fr_rel_l2=l2, Fr_max_row=re)
    assert l2 < 1e-4
    assert re < ROW_TOL
    assert Z.item() > Zi.sum()


def test_full_step_at_full_size(atlas, gpu):
    wl, X, idx, d2, P, beta, n_bad, rows = atlas
    n = wl.n
    Y = torch.tensor(synth.initial_embedding(n, 13) * 100, device=gpu)
    U, G = torch.zeros_like(Y), torch.ones_like(Y)
    st = api.new_status(gpu)
    g, Z, _ = api.kl_grad(P, Y, 12.0, status=st)
    api.step(P, Y, U, G, 0, L.default_params(), status=st)
    torch.cuda.synchronize()
    assert st.item() == 0 and torch.isfinite(Y).all()
    g64 = g.cpu().numpy().astype(np.float64)
    assert np.abs(g64.sum(0)).max() < 1e-4 * np.abs(g64).sum(0).max()


def test_combined_gradient_rows_at_full_size(atlas, gpu):
    """The attraction and repulsion together at 1M, as AUTO runs them (the
    attraction on a side stream beside the tiled repulsion), with a P from a
    host generator (no GPU output enters the oracle): per sampled row 3e-4 of
    its scale 4 (alpha Aa_i + Ar_i / Z) (problems.ROW_TOL), 1e-4 relative L2
    against the larger of |g| and its terms' norms, Z to 1e-6."""
    wl = atlas[0]
    n = wl.n
    rows = atlas[7]
    Y = STATES["spread"](n)
    Y64 = Y.astype(np.float64)
    box = {}
    th = threading.Thread(target=lambda: box.update(z=oracle.Z(Y64)), daemon=True)
    th.start()
    row_ptr, col, val = synth.neighbour_csr(n, wl.k, 5000, seed=23)
    Pd = api.CSR(torch.tensor(row_ptr, device=gpu), torch.tensor(col, device=gpu),
                 torch.tensor(val, device=gpu))
    Yd = torch.tensor(Y, device=gpu)
    st = api.new_status(gpu)
    out = {}
    for alpha in (12.0, 1.0):
        g, Z, _ = api.kl_grad(Pd, Yd, alpha, status=st)
        out[alpha] = (g.cpu().numpy()[rows].astype(np.float64), Z.item())
    assert st.item() == 0
    Fa, Fr, _, Aa, Ar = oracle.forces_rows(oracle.CSR(row_ptr, col, val.astype(np.float64)), Y64,
                                           rows, scales=True)
    th.join()
    Z_ref = box["z"]
    for alpha, (g, Z) in out.items():
        g_ref = 4.0 * (alpha * Fa - Fr / Z_ref)
        den = max(np.linalg.norm(g_ref), 4 * alpha * np.linalg.norm(Fa),
                  4 * np.linalg.norm(Fr) / Z_ref)
        l2 = float(np.linalg.norm(g - g_ref) / den)
        re = row_err_scaled(g - g_ref, 4.0 * (alpha * Aa + Ar / Z_ref))
        zr = abs(Z / Z_ref - 1)
        record(f"combined_grad/atlas_n1m/alpha{alpha}", grad_rel_l2=l2, grad_max_row=re, Z_rel=zr)
        assert l2 < 1e-4
        assert re < ROW_TOL
        assert zr < 1e-6


def test_pca_full_size_properties(gpu):
    """PCA at the pca_n1m_g2000 size (1M x 2000 -> 50) in the benchmarked
    configuration, checked by properties of the exact answer computed in FP64
    on the host: the mean, orthonormal axes, the eigen-residual
    ||Ac^T Ac v_c - lambda_c v_c|| <= 1e-3 lambda_1 (eps sigma_1^2 scale of the
    BF16x3 products), sigma_c^2 = v_c^T Ac^T Ac v_c within 6e-5 sigma_1, and the
    scores of 200 sampled cells = (A_i - mean) V^T."""
    cfg = dict(synth.PCA_N1M_G2000)
    n, g, k = cfg["n"], cfg["g"], 50
    A = synth.pca_matrix_device(n, g, gpu, rank=cfg["rank"], n_clusters=cfg["n_clusters"],
                                noise=cfg["noise"], seed=cfg["seed"])
    omega = torch.tensor(synth.pca_omega(g), device=gpu)
    st = api.new_status(gpu)
    out = api.pca(A, k, n_power=2, omega=omega, status=st)
    torch.cuda.synchronize()
    assert st.item() == 0
    V = out["components"].cpu().numpy().astype(np.float64)
    sig = out["sigma"].cpu().numpy()
    mean = out["mean"].cpu().numpy()
    T = out["scores"]
    Ah = A.cpu().numpy()
    del A
    mu = np.zeros(g)
    for a in range(0, n, 1 << 17):
        mu += Ah[a:a + (1 << 17)].astype(np.float64).sum(0)
    mu /= n
    np.testing.assert_allclose(mean, mu, atol=1e-6 * np.abs(mu).max() + 1e-9)
    np.testing.assert_allclose(V @ V.T, np.eye(k), atol=2e-5)
    # C V^T accumulated over row chunks in FP64
    CV = np.zeros((g, k))
    for a in range(0, n, 1 << 16):
        Ac = Ah[a:a + (1 << 16)].astype(np.float64) - mu
        CV += Ac.T @ (Ac @ V.T)
    lam = (V * CV.T).sum(1)
    # sigma from the GPU's Rayleigh-Ritz step vs the FP64 Rayleigh quotient of its axes:
    # both carry the products' error, eps sigma_1 with eps ~ 3e-5
    assert np.all(np.abs(np.sqrt(lam) - sig) <= 6e-5 * sig[0])
    resid = np.linalg.norm(CV - V.T * lam[None, :], axis=0)
    assert (resid <= 1e-3 * lam[0]).all()
    rows = np.sort(np.random.default_rng(14).choice(n, 200, replace=False))
    Tr = (Ah[rows].astype(np.float64) - mu) @ V.T
    Tg = T.cpu().numpy()[rows].astype(np.float64)
    assert np.linalg.norm(Tg - Tr) / np.linalg.norm(Tr) < 1e-4


def test_umap_epoch_rows_at_full_size(gpu):
    """One epoch (e = 100 of 200) of the UMAP layout at the umap_layout_n1m size on
    a symmetric graph built on the host (12 random links per point, both
    directions, weights uniform in [0.05, 1]): 200 sampled rows against the
    oracle's update of those rows, within the per-point bound of
    tests/test_gpu_umap.py."""
    from oracle import umap_layout as U
    n, m = 1_000_000, 12
    rng = np.random.default_rng(15)
    src = np.repeat(np.arange(n, dtype=np.int64), m)
    dst = rng.integers(0, n, n * m)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    w = rng.uniform(0.05, 1.0, len(src)).astype(np.float32)
    key = np.concatenate([src * n + dst, dst * n + src])
    ww = np.concatenate([w, w])
    order = np.argsort(key, kind="stable")
    key, ww = key[order], ww[order]
    uniq, first = np.unique(key, return_index=True)
    val = np.maximum.reduceat(ww, first).astype(np.float32)
    row, col = uniq // n, (uniq % n).astype(np.int32)
    rp = np.concatenate([[0], np.cumsum(np.bincount(row, minlength=n))]).astype(np.int64)
    Y = rng.uniform(-10, 10, (n, 2)).astype(np.float32)
    a, b, e, n_epochs, n_neg, seed = 1.577, 0.895, 100, 200, 5, 3
    G = api.CSR.from_numpy(rp, col, val, gpu)
    Yd = torch.tensor(Y, device=gpu)
    st = api.new_status(gpu)
    api.umap_layout(G, Yd, n_epochs=n_epochs, a=a, b=b, n_neg=n_neg, seed=seed, epoch0=e,
                    n_run=1, status=st)
    torch.cuda.synchronize()
    assert st.item() == 0
    rows = np.sort(rng.choice(n, ROWS, replace=False))
    D = U.epoch_delta(rp, col, val, Y.astype(np.float64), e, a, b, n_neg, seed, rows=rows)
    alpha = 1.0 - e / n_epochs
    ref = Y[rows].astype(np.float64) + alpha * D
    got = Yd.cpu().numpy()[rows].astype(np.float64)
    deg = np.diff(rp)[rows].astype(np.float64)
    bound = alpha * 1e-5 * 4 * deg * (1 + n_neg) + 2.0 ** -22 * np.abs(Y[rows]).max(1)
    assert np.all(np.abs(got - ref).max(1) <= bound)
    assert np.abs(got - Y[rows]).max() > 1e-3

