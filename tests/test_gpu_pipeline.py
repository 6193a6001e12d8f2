"""The chained GPU pipeline (PCA -> exact t-SNE -> fuzzy graph -> UMAP layout) on a small
cells x genes matrix: each stage equals its stand-alone call (deterministic
kernels), the PCA stage matches the FP64 oracle, the embedding is finite and
its KL falls."""
import numpy as np
import pytest
import torch

from oracle import pca as OP
from paper_2605_13928_b300 import _lib as L
from paper_2605_13928_b300 import api, pipeline, synth

pytestmark = pytest.mark.gpu


def test_embed_cells_chains_the_stages(gpu):
    A = synth.pca_matrix(2500, 300, seed=synth.SEED_BASE + 60)
    Ad = torch.tensor(A, device=gpu)
    prm = L.default_params(n_iter=300, ee_iters=100, mom_switch=100, kl_every=50)
    out = pipeline.embed_cells(Ad, n_pcs=30, params=prm, graph_k=15, umap_epochs=50)
    assert out.status == 0
    # stage 1 equals the stand-alone PCA, and matches the oracle's singular values
    ref = api.pca(Ad, 30)
    assert torch.equal(out.scores, ref["scores"])
    sig_r = OP.pca(A, 30)["sigma"]
    assert np.all(np.abs(out.sigma.cpu().numpy() - sig_r) <= 6e-5 * sig_r[0])
    # stage 2: finite embedding whose KL falls after exaggeration
    Y = out.Y.cpu().numpy()
    assert np.isfinite(Y).all() and Y.std() > 1.0
    tr = out.kl_trace[:, 0]
    assert tr[-1] < tr[2]
    # stage 3: the graph of the scores equals the stand-alone graph
    idx, d2 = api.knn(out.scores.contiguous(), 15, mode=L.TSNE_KNN_BF16_RERANK)
    G, _, _, _ = api.knn_graph(idx, d2)
    for a, b in zip(out.graph.to_numpy(), G.to_numpy()):
        assert np.array_equal(a, b)
    # stage 4: the UMAP layout equals the stand-alone call from the same start
    U = pipeline.umap_init(out.scores.contiguous())
    api.umap_layout(G, U, n_epochs=50, seed=0)
    assert torch.equal(out.umap, U) and torch.isfinite(U).all()
