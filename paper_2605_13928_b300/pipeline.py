"""The GPU part of the single-cell pipeline the paper benchmarks (its Table 1,
steps 5-7), chained on one device through the libtsne.so C ABI:

  cells x genes matrix --PCA (tsne_pca)--> 50-D scores
      --kNN + perplexity affinities + exact t-SNE (tsne_run)--> 2-D embedding
      --fuzzy neighbour graph (tsne_knn / tsne_knn_graph)--> UMAP / Leiden graph
      --UMAP layout optimisation (tsne_umap_layout)--> 2-D UMAP layout

Argument marshalling only: every step runs in the library's kernels.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

from . import _lib as L
from . import api, synth


@dataclass
class Embedding:
    scores: torch.Tensor          # n x n_pcs PCA scores (device)
    components: torch.Tensor      # n_pcs x g principal axes (device)
    sigma: torch.Tensor           # n_pcs singular values (device, FP64)
    Y: torch.Tensor               # n x 2 t-SNE embedding (device)
    kl_trace: Optional[np.ndarray]
    status: int
    graph: Optional[api.CSR] = None
    umap: Optional[torch.Tensor] = None  # n x 2 UMAP layout (device)


def embed_cells(A: torch.Tensor, n_pcs: int = 50, params: Optional[L.TsneParams] = None,
                n_power: int = 2, seed: int = 0, graph_k: int = 0,
                umap_epochs: int = 0) -> Embedding:
    """PCA of A (n x g FP32 CUDA tensor) to n_pcs components, exact t-SNE of
    the scores with `params` (library defaults when None: perplexity 30,
    k = 90, 750 iterations), and, when graph_k >= 2, the fuzzy graph on the
    graph_k nearest neighbours of the scores; with umap_epochs > 0 also the
    UMAP layout of that graph, started from the first two PCA scores scaled
    into [-10, 10] (min_dist 0.1, spread 1, 5 negatives per taken entry)."""
    if params is None:
        params = L.default_params()
    pca = api.pca(A, n_pcs, n_power=n_power, seed=seed)
    X = pca["scores"].contiguous()
    n = X.shape[0]
    Y0 = torch.tensor(synth.initial_embedding(n, seed), device=A.device)
    Y, trace, status = api.run(X, Y0, params)
    G = None
    U = None
    if graph_k >= 2:
        idx, d2 = api.knn(X, graph_k, mode=L.TSNE_KNN_BF16_RERANK)
        G, _, _, _ = api.knn_graph(idx, d2)
        if umap_epochs > 0:
            U = umap_init(X)
            api.umap_layout(G, U, n_epochs=umap_epochs, seed=seed)
    return Embedding(pca["scores"], pca["components"], pca["sigma"], Y, trace, status, G, U)


def umap_init(scores: torch.Tensor) -> torch.Tensor:
    """Initial UMAP layout: the first two PCA scores, centred and scaled so that
    the larger coordinate range is [-10, 10] (a PCA start in place of a spectral
    one), computed by the library (tsne_umap_init)."""
    return api.umap_init(scores)
