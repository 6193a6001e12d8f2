"""Seeded synthetic inputs: PCA-like Gaussian mixtures and initial embeddings.

This module draws inputs only; it holds none of the t-SNE arithmetic, and both
the CUDA path's tests and the CPU oracle take their inputs from it.  The paper's
workload (1M E18 mouse-brain cells after PCA, Sec. 3.3) is not available, so
these mixtures stand in for its PCA scores:

* cluster means mu_c ~ N(0, 16 I_D);
* point x = mu_c + eps with eps_d ~ N(0, 1/d) for d = 1..D (per-dimension
  standard deviation decaying as 1/sqrt(d), like PCA scores ordered by
  explained variance);
* anisotropic variant: eps = R_c diag(s_c / sqrt(d)) z with R_c a random
  orthogonal matrix (QR of a Gaussian matrix) and s_{c,d} ~ LogUniform[0.5, 2];
* cluster sizes from weights (equal, log-normal exp(N(0, sigma^2)), or Zipf
  r^-a), rounded to sum to N by largest remainder;
* rows shuffled, so cluster members are not contiguous in memory;
* the initial embedding Y0 ~ N(0, 1e-4 I_2) (standard deviation 0.01).

All generators use numpy's PCG64 seeded explicitly.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 20260513


def _largest_remainder(weights: np.ndarray, n: int) -> np.ndarray:
    w = np.asarray(weights, dtype=np.float64)
    w = w / w.sum()
    raw = w * n
    base = np.floor(raw).astype(np.int64)
    short = n - int(base.sum())
    order = np.argsort(-(raw - base), kind="stable")
    base[order[:short]] += 1
    return base


def cluster_sizes(n: int, n_clusters: int, kind: str, rng: np.random.Generator,
                  sigma: float = 1.0, zipf_a: float = 1.1) -> np.ndarray:
    if kind == "equal":
        w = np.ones(n_clusters)
    elif kind == "lognormal":
        w = np.exp(rng.normal(0.0, sigma, size=n_clusters))
    elif kind == "zipf":
        w = np.arange(1, n_clusters + 1, dtype=np.float64) ** (-zipf_a)
    else:
        raise ValueError(f"unknown size distribution {kind!r}")
    return _largest_remainder(w, n)


def mixture(n: int, n_clusters: int, d: int = 50, sizes: str = "equal", seed: int = SEED_BASE,
            anisotropic: bool = False, sigma: float = 1.0, zipf_a: float = 1.1,
            mean_std: float = 4.0) -> np.ndarray:
    """n x d float32 PCA-like scores drawn from a seeded Gaussian mixture."""
    rng = np.random.default_rng(seed)
    counts = cluster_sizes(n, n_clusters, sizes, rng, sigma=sigma, zipf_a=zipf_a)
    means = rng.normal(0.0, mean_std, size=(n_clusters, d))
    dim_std = 1.0 / np.sqrt(np.arange(1, d + 1, dtype=np.float64))
    X = np.empty((n, d), dtype=np.float32)
    o = 0
    for c in range(n_clusters):
        m = int(counts[c])
        if m == 0:
            continue
        z = rng.standard_normal(size=(m, d))
        if anisotropic:
            R, _ = np.linalg.qr(rng.standard_normal(size=(d, d)))
            s = np.exp(rng.uniform(math.log(0.5), math.log(2.0), size=d))
            eps = (z * (s * dim_std)) @ R.T
        else:
            eps = z * dim_std
        X[o:o + m] = (means[c] + eps).astype(np.float32)
        o += m
    perm = rng.permutation(n)
    return np.ascontiguousarray(X[perm])


def initial_embedding(n: int, seed: int, dim: int = 2, std: float = 1e-2) -> np.ndarray:
    """Y0 ~ N(0, std^2 I) as n x dim float32 (default covariance 1e-4 I)."""
    rng = np.random.default_rng(seed + 7919)
    return rng.normal(0.0, std, size=(n, dim)).astype(np.float32)


def embedding_state(n: int, n_clusters: int, centre_std: float, within_std: float, seed: int,
                    zipf_a: float = 1.1) -> np.ndarray:
    """An n x 2 float32 embedding shaped like a t-SNE state: n_clusters
    Zipf-sized clusters, centres ~ N(0, centre_std^2 I), points ~ N(centre,
    within_std^2 I), rows shuffled.  Small centre_std and within_std give the
    clumped layouts of early exaggeration (forces of many near-coincident points
    nearly cancel); large centre_std gives the spread layouts of late iterations
    (w spans many orders of magnitude)."""
    rng = np.random.default_rng(seed)
    counts = cluster_sizes(n, n_clusters, "zipf", rng, zipf_a=zipf_a)
    centres = rng.normal(0.0, centre_std, size=(n_clusters, 2))
    lab = np.repeat(np.arange(n_clusters), counts)
    Y = centres[lab] + rng.normal(0.0, within_std, size=(n, 2))
    return Y[rng.permutation(n)].astype(np.float32)


def neighbour_csr(n: int, k: int, window: int, seed: int):
    """A seeded sparse n x n matrix in CSR form with the shape of a kNN affinity
    matrix of spatially ordered points: k entries per row, columns j != i drawn
    within `window` of i (reflected at the ends, ascending per row, repeats
    possible), positive values summing to 1.  Returns (row_ptr int64, col
    int32, val float32).  An input generator only: no perplexity calibration or
    symmetrisation."""
    rng = np.random.default_rng(seed)
    i = np.arange(n, dtype=np.int64)[:, None]
    off = rng.integers(1, window + 1, size=(n, k), dtype=np.int64)
    off *= rng.choice(np.array([-1, 1], dtype=np.int64), size=(n, k))
    j = i + off
    j = np.where((j < 0) | (j >= n), i - off, j)
    col = np.sort(j.astype(np.int32), axis=1).reshape(-1)
    val = rng.exponential(1.0, size=n * k)
    val = (val / val.sum()).astype(np.float32)
    row_ptr = np.arange(n + 1, dtype=np.int64) * k
    return row_ptr, col, val


def batch_sizes(n_samples: int = 64, lo: int = 500, hi: int = 20000, seed: int = SEED_BASE + 3):
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_samples))).astype(np.int64)


def batch(n_samples: int = 64, lo: int = 500, hi: int = 20000, d: int = 50,
          seed: int = SEED_BASE + 3, sizes=None):
    """List of per-sample n_s x d mixtures with 5..20 equal-weight clusters each."""
    rng = np.random.default_rng(seed + 1)
    ns = batch_sizes(n_samples, lo, hi, seed) if sizes is None else np.asarray(sizes)
    out = []
    for s, n in enumerate(ns):
        nc = int(rng.integers(5, 21))
        out.append(mixture(int(n), nc, d=d, sizes="equal", seed=seed * 1000 + s))
    return out


@dataclasses.dataclass(frozen=True)
class Workload:
    """One named t-SNE workload: data recipe plus optimiser settings."""
    name: str
    n: int
    n_clusters: int
    sizes: str
    anisotropic: bool
    k: int = 90
    perplexity: float = 30.0
    n_iter: int = 750
    ee_iters: int = 250
    ee: float = 12.0
    mom0: float = 0.5
    mom1: float = 0.8
    seed: int = SEED_BASE
    d: int = 50

    def data(self) -> np.ndarray:
        return mixture(self.n, self.n_clusters, d=self.d, sizes=self.sizes, seed=self.seed,
                       anisotropic=self.anisotropic)

    def y0(self) -> np.ndarray:
        return initial_embedding(self.n, self.seed)


WORKLOADS = {
    "plain_n2000": Workload("plain_n2000", 2000, 8, "equal", False, n_iter=500, ee_iters=125,
                            seed=SEED_BASE + 0),
    "kl_n50k": Workload("kl_n50k", 50_000, 30, "lognormal", False, n_iter=1000,
                        seed=SEED_BASE + 1),
    "knn_n200k": Workload("knn_n200k", 200_000, 50, "zipf", False, seed=SEED_BASE + 2),
    "atlas_n1m": Workload("atlas_n1m", 1_000_000, 100, "zipf", True, seed=SEED_BASE + 4),
}


# ---------------------------------------------------------------- PCA input
# Stand-in for the scaled cells x genes matrix that the paper's pipeline hands
# to PCA (its Table 1, steps 4-5): a latent 50-D mixture (the same recipe as
# the t-SNE workloads) mapped to g genes through orthonormal loadings, plus
# per-entry Gaussian noise and per-gene offsets.  With a small `noise` the top
# `rank` principal axes are separated from the rest by a clear spectral gap.
PCA_N1M_G2000 = dict(n=1_000_000, g=2000, rank=50, n_clusters=100, noise=0.01,
                     seed=SEED_BASE + 5)


def pca_loadings(g: int, rank: int, seed: int) -> np.ndarray:
    """g x rank orthonormal loadings (QR of a seeded Gaussian matrix)."""
    rng = np.random.default_rng(seed + 101)
    Q, _ = np.linalg.qr(rng.normal(size=(g, rank)))
    return Q


def pca_matrix(n: int, g: int, rank: int = 50, n_clusters: int = 30, noise: float = 0.01,
               seed: int = SEED_BASE + 5, offset_std: float = 1.0, sizes: str = "zipf",
               chunk: int = 1 << 16) -> np.ndarray:
    """n x g float32: latent mixture (n x rank) @ loadings^T + noise * N(0, 1)
    + per-gene offsets ~ N(0, offset_std^2); generated in row chunks."""
    latent = mixture(n, n_clusters, d=rank, sizes=sizes, seed=seed).astype(np.float64)
    W = pca_loadings(g, rank, seed)
    rng = np.random.default_rng(seed + 202)
    offs = rng.normal(0.0, offset_std, size=g)
    out = np.empty((n, g), dtype=np.float32)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        blk = latent[a:b] @ W.T + offs[None, :]
        blk += noise * rng.standard_normal(size=(b - a, g))
        out[a:b] = blk
    return out


def pca_omega(g: int, L: int = 64, seed: int = SEED_BASE + 6) -> np.ndarray:
    """g x L float32 standard Gaussian test matrix of the randomized range finder."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(size=(g, L)).astype(np.float32)


def pca_matrix_device(n: int, g: int, device, rank: int = 50, n_clusters: int = 100,
                      noise: float = 0.01, seed: int = SEED_BASE + 5, offset_std: float = 1.0,
                      sizes: str = "zipf", chunk: int = 1 << 17):
    """The pca_matrix recipe generated on a CUDA device (torch, seeded), for
    sizes whose host generation would dominate a run (1M x 2000 = 8 GB): the
    latent mixture and the loadings come from the host generator, the noise
    from a seeded torch generator on the device."""
    import torch
    latent = torch.tensor(mixture(n, n_clusters, d=rank, sizes=sizes, seed=seed), device=device)
    W = torch.tensor(pca_loadings(g, rank, seed).astype(np.float32), device=device)
    offs = torch.tensor(np.random.default_rng(seed + 202).normal(0.0, offset_std, size=g)
                        .astype(np.float32), device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed + 303)
    out = torch.empty((n, g), dtype=torch.float32, device=device)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        blk = torch.randn((b - a, g), generator=gen, device=device, dtype=torch.float32)
        blk.mul_(noise).add_(latent[a:b] @ W.T).add_(offs)
        out[a:b] = blk
    return out
