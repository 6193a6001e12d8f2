"""FP64 CPU oracle of principal component analysis -- TEST INFRASTRUCTURE ONLY.

Only the tests, the package smoke check and the benchmark's CPU-baseline leg may
import this module.  It shares no code with the CUDA path and never calls it.

The single-cell pipeline runs PCA on the scaled cells x genes matrix before
the neighbour graph and the embeddings (the paper's Table 1, step 5); the
paper does not define it, so this is the plain definition (Pearson 1901;
Jolliffe 2002, Sec. 1.1), with library routines (a matrix product, a
symmetric eigensolver) as steps:

* column means mu_g = (1/n) sum_i A_ig, centred matrix Ac = A - 1 mu^T;
* scatter matrix C = Ac^T Ac (g x g);
* principal axes v_1..v_k: unit eigenvectors of C for its k largest
  eigenvalues lambda_1 >= ... >= lambda_k;
* singular values sigma_c = sqrt(lambda_c); explained variance
  lambda_c / (n - 1); explained-variance ratio lambda_c / trace(C);
* scores T = Ac V_k^T (n x k), components V_k (k x g, one axis per row);
* sign convention (an eigenvector is defined up to sign): every axis is
  flipped so that its entry of largest magnitude -- the lowest gene index
  among equal magnitudes -- is positive.

All arrays are float64 numpy.
"""
from __future__ import annotations

import numpy as np


def column_means(A):
    A = np.asarray(A, dtype=np.float64)
    return A.sum(axis=0) / A.shape[0]


def sign_fix(V):
    """Rows of V flipped so that each row's largest-magnitude entry (lowest
    index among ties) is positive."""
    V = np.array(V, dtype=np.float64, copy=True)
    idx = np.argmax(np.abs(V), axis=1)  # first index of the maximum
    s = np.sign(V[np.arange(V.shape[0]), idx])
    s[s == 0] = 1.0
    return V * s[:, None], s


def pca(A, k):
    """Exact k-component PCA of the rows of A (n x g).  Returns a dict with
    mean (g), components (k x g), sigma (k), scores (n x k),
    explained_variance (k), ratio (k) and total_var (trace(C) / (n - 1))."""
    A = np.asarray(A, dtype=np.float64)
    n, g = A.shape
    if not 1 <= k <= min(n, g):
        raise ValueError("need 1 <= k <= min(n, g)")
    mu = column_means(A)
    Ac = A - mu[None, :]
    C = Ac.T @ Ac
    lam, vec = np.linalg.eigh(C)  # ascending
    order = np.argsort(-lam, kind="stable")[:k]
    lam_k = np.maximum(lam[order], 0.0)
    V, _ = sign_fix(vec[:, order].T)
    T = Ac @ V.T
    tr = float(np.trace(C))
    return {"mean": mu, "components": V, "sigma": np.sqrt(lam_k), "scores": T,
            "explained_variance": lam_k / (n - 1), "ratio": lam_k / tr if tr > 0 else lam_k * 0,
            "total_var": tr / (n - 1)}


def transform(A, mean, components):
    """Scores of new rows: (A - mean) V^T."""
    A = np.asarray(A, dtype=np.float64)
    return (A - np.asarray(mean, np.float64)[None, :]) @ np.asarray(components, np.float64).T
