"""FP64 CPU oracle of the fuzzy neighbour graph -- TEST INFRASTRUCTURE ONLY.

Only the tests, the package smoke check and the benchmark's CPU-baseline leg may
import this module.  It shares no code with the CUDA path and never calls it.

The pipeline's step 6 builds the neighbour graph that UMAP and Leiden use (the
paper's Table 1); the paper does not define it, so this follows the fuzzy
simplicial set of McInnes, Healy & Melville (2018), Sec. 3.1:

* for point i with k nearest neighbours (self excluded) at Euclidean
  distances d_i1 <= ... <= d_ik:
  rho_i = the smallest positive d_ij (0 if every d_ij is 0);
  sigma_i solves  sum_j exp(-max(0, d_ij - rho_i) / sigma_i) = log2(k);
* directed weights w_ij = exp(-max(0, d_ij - rho_i) / sigma_i);
* symmetric graph (fuzzy set union): b_ij = w_ij + w_ji - w_ij w_ji, with
  w_ij = 0 where j is not among i's neighbours.

f(sigma) = sum_j exp(-max(0, d_ij - rho_i) / sigma) increases from the
number of d_ij <= rho_i (sigma -> 0) to k (sigma -> inf).  When that number is
at least log2(k) the target is out of reach: the row takes the sigma -> 0
limit (weight 1 on those neighbours, 0 on the others) and is flagged.
Reading: sigma is found by bisection on sigma itself (start 1, double while
f < target, then halve the bracket) to |f - log2 k| <= tol.
"""
from __future__ import annotations

import math

import numpy as np


def rho_sigma(d, tol=1e-12, max_iter=200):
    """Per-row (rho, sigma, flag) for Euclidean neighbour distances d (n x k)."""
    d = np.asarray(d, dtype=np.float64)
    n, k = d.shape
    target = math.log2(k)
    rho = np.zeros(n)
    sigma = np.zeros(n)
    flag = np.zeros(n, dtype=np.int8)
    for i in range(n):
        pos = d[i][d[i] > 0]
        r = pos.min() if len(pos) else 0.0
        rho[i] = r
        x = np.maximum(d[i] - r, 0.0)
        if np.count_nonzero(x == 0) >= target:
            flag[i] = 1
            continue
        lo, hi, s = 0.0, math.inf, 1.0
        done = False
        for _ in range(max_iter):
            f = np.exp(-x / s).sum()
            if abs(f - target) <= tol:
                done = True
                break
            if f > target:
                hi = s
            else:
                lo = s
            s = 2 * s if math.isinf(hi) else 0.5 * (lo + hi)
        sigma[i] = s
        flag[i] = 0 if done else 1
    return rho, sigma, flag


def weights(d, rho, sigma):
    """Directed membership strengths w_ij (sigma = 0: the limit, 1 where d <= rho)."""
    d = np.asarray(d, dtype=np.float64)
    x = np.maximum(d - np.asarray(rho)[:, None], 0.0)
    s = np.asarray(sigma)[:, None]
    with np.errstate(divide="ignore", invalid="ignore"):
        w = np.where(s > 0, np.exp(-x / np.where(s > 0, s, 1.0)), (x == 0).astype(np.float64))
    return w


def fuzzy_union(idx, w, n):
    """Symmetric graph b_ij = w_ij + w_ji - w_ij w_ji as CSR (row_ptr, col, val),
    columns ascending, no diagonal."""
    idx = np.asarray(idx)
    a = {}
    for i in range(idx.shape[0]):
        for jj, j in enumerate(idx[i]):
            a[(i, int(j))] = float(w[i, jj])
    b = {}
    for (i, j), v in a.items():
        u = a.get((j, i), 0.0)
        b[(i, j)] = v + u - v * u
        b[(j, i)] = b[(i, j)]
    rows = [[] for _ in range(n)]
    for (i, j), v in b.items():
        rows[i].append((j, v))
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    col, val = [], []
    for i in range(n):
        rows[i].sort()
        row_ptr[i + 1] = row_ptr[i] + len(rows[i])
        col.extend(j for j, _ in rows[i])
        val.extend(v for _, v in rows[i])
    return row_ptr, np.asarray(col, dtype=np.int32), np.asarray(val, dtype=np.float64)


def graph(X, k):
    """kNN (FP64 brute force, self excluded, ordered by (d^2, j)) + fuzzy graph."""
    from . import knn
    idx, d2 = knn(np.asarray(X, dtype=np.float64), k)
    d = np.sqrt(d2)
    rho, sigma, flag = rho_sigma(d)
    w = weights(d, rho, sigma)
    return fuzzy_union(idx, w, len(idx)), idx, d, rho, sigma, flag
