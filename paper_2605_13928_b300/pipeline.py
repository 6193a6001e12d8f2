"""The GPU part of the single-cell pipeline the paper benchmarks (its Table 1,
steps 5-7), chained on one device through the libtsne.so C ABI:

  cells x genes matrix --PCA (tsne_pca)--> 50-D scores
      --kNN + perplexity affinities + exact t-SNE (tsne_run)--> 2-D embedding
      --fuzzy neighbour graph (tsne_knn / tsne_knn_graph)--> UMAP / Leiden graph

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


def embed_cells(A: torch.Tensor, n_pcs: int = 50, params: Optional[L.TsneParams] = None,
                n_power: int = 2, seed: int = 0, graph_k: int = 0) -> Embedding:
    """PCA of A (n x g FP32 CUDA tensor) to n_pcs components, exact t-SNE of
    the scores with `params` (library defaults when None: perplexity 30,
    k = 90, 750 iterations), and, when graph_k >= 2, the fuzzy graph on the
    graph_k nearest neighbours of the scores."""
    if params is None:
        params = L.default_params()
    pca = api.pca(A, n_pcs, n_power=n_power, seed=seed)
    X = pca["scores"].contiguous()
    n = X.shape[0]
    Y0 = torch.tensor(synth.initial_embedding(n, seed), device=A.device)
    Y, trace, status = api.run(X, Y0, params)
    G = None
    if graph_k >= 2:
        idx, d2 = api.knn(X, graph_k, mode=L.TSNE_KNN_BF16_RERANK)
        G, _, _, _ = api.knn_graph(idx, d2)
    return Embedding(pca["scores"], pca["components"], pca["sigma"], Y, trace, status, G)
