"""Shared seeded problems for the GPU parity tests: inputs from the synthetic
generator, expected values from the FP64 oracle only."""
import functools
import json
import os

import numpy as np

import oracle
from paper_2605_13928_b300 import synth


@functools.lru_cache(maxsize=None)
def mixture_P(n, n_clusters=8, k=30, perplexity=10.0, seed=0, d=10):
    """Oracle P (CSR, float64) of a seeded mixture of n points."""
    X = synth.mixture(n, n_clusters, d=d, sizes="equal", seed=synth.SEED_BASE + 100 + seed)
    k = min(k, n - 1)
    perp = min(perplexity, k / 3.0 if k >= 3 else 0.9 * k + 0.05)
    P, idx, d2, pc, beta, flag = oracle.affinities(X.astype(np.float64), k, perp)
    return X, P


def embedding(n, scale, seed=0):
    rng = np.random.default_rng(1234 + seed)
    return (rng.normal(size=(n, 2)) * scale).astype(np.float32)


def block_diag(Ps):
    """Concatenate per-sample CSR matrices into one block-diagonal CSR."""
    rp, cols, vals, off, e = [np.zeros(1, dtype=np.int64)], [], [], 0, 0
    for P in Ps:
        rp.append(P.row_ptr[1:] + e)
        cols.append(P.col.astype(np.int64) + off)
        vals.append(P.val)
        off += P.n
        e += P.nnz
    return oracle.CSR(np.concatenate(rp), np.concatenate(cols), np.concatenate(vals))


def record(name, **measured):
    """Appends the errors a parity test measured (not only its verdict) to the
    JSON-lines file $TSNE_PARITY_LOG names, if set: the source of the tables of
    measured errors per configuration."""
    path = os.environ.get("TSNE_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"test": name, **{k: float(v) for k, v in measured.items()}}) + "\n")


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# Per-row bound.  Each row of the GPU gradient sums FP32 terms: a term's own
# rounding is a few units of u = 2^-24 of its magnitude, and a sequential FP32
# running sum of m terms adds at most (m - 1) u times the sum of the terms'
# magnitudes.  The kernels' longest FP32 running sums hold at most 4096 terms
# before they are folded into compensated, fixed-point or FP64 sums (a column
# accumulator of the tiled fixed-point form over its tile's four row groups;
# 1024 in every other kernel: a column of one group pair, a 1024-column tile of
# the direct form), and the attraction's at most ~2k / 16 per lane, so for
# every row
#   |g_i - g_ref,i| <= 4 (alpha Aa_i + Ar_i / Z) * (4100 u + dZ) < 4 (alpha Aa_i + Ar_i / Z) * 3e-4,
# with Aa_i, Ar_i the sums of the attraction and repulsion terms' magnitudes
# (oracle.forces_rows(..., scales=True)) and dZ <= 1e-6 the relative error of Z.
# A worst case: rounding errors of random sign grow like sqrt(m) u, and the
# measured errors are about 1e-7 of that scale.  A wrong row (a tile-boundary
# or sentinel mistake) is off by order 1.
ROW_TOL = 3e-4


def row_err_scaled(diff, scale):
    """max_i |diff_i| / scale_i for rows (n x 2) of differences and per-row scales."""
    d = np.hypot(np.asarray(diff, dtype=np.float64)[:, 0], np.asarray(diff, dtype=np.float64)[:, 1])
    scale = np.asarray(scale, dtype=np.float64)
    return float(np.max(d / np.maximum(scale, 1e-300))) if len(d) else 0.0


def row_err(g, P, Y, alpha):
    """Largest per-row error of a gradient against the oracle, in units of the
    row's own scale 4 (alpha Aa_i + Ar_i / Z) (see ROW_TOL)."""
    Y64 = np.asarray(Y, dtype=np.float64)
    g_ref, Z = oracle.grad(P, Y64, alpha)
    _, _, _, Aa, Ar = oracle.forces_rows(P, Y64, scales=True)
    return row_err_scaled(np.asarray(g, dtype=np.float64) - g_ref, 4 * (alpha * Aa + Ar / Z))


def grad_err(g, P, Y, alpha):
    """Relative L2 error of a gradient against the oracle.

    The denominator is max(|g_ref|, |4 alpha Fa|, |4 Fr / Z|): when attraction and
    repulsion cancel (N = 2 at alpha = 1, or P = Q) the exact gradient is 0 and an
    FP32 result can only be judged against the size of the cancelling terms."""
    Y64 = np.asarray(Y, dtype=np.float64)
    g_ref, Z = oracle.grad(P, Y64, alpha)
    Fa, Fr, _ = oracle.forces_rows(P, Y64)
    den = max(np.linalg.norm(g_ref), 4 * alpha * np.linalg.norm(Fa), 4 * np.linalg.norm(Fr) / Z)
    return float(np.linalg.norm(np.asarray(g, dtype=np.float64) - g_ref) / max(den, 1e-300))
