"""FP64 CPU oracle of the UMAP layout optimisation -- TEST INFRASTRUCTURE ONLY.

Only the tests, the package smoke check and the benchmark's CPU-baseline leg may
import this module.  It shares no code with the CUDA path and never calls it.

The pipeline's step 7 lays the fuzzy neighbour graph out in 2-D with UMAP (the
paper's Table 1); the paper does not define the method, so this follows
McInnes, Healy & Melville (2018), Sec. 3.2 and their embedding optimisation
algorithm (Algorithm 5):

* low-dimensional membership  Phi(y_i, y_j) = 1 / (1 + a d^(2b)),  d = |y_i - y_j|,
  with (a, b) the least-squares fit of Phi to
  Psi(d) = 1 for d <= min_dist, exp(-(d - min_dist) / spread) beyond  (fit_ab);
* epoch e of n_epochs has the learning rate alpha_e = alpha0 (1 - e / n_epochs);
* every graph edge (i, j) of weight p is taken with probability p; a taken edge
  moves y_i along  grad_i log Phi(y_i, y_j)  and, for each of n_neg vertices c
  drawn uniformly, along  grad_i log(1 - Phi(y_i, y_c)):
      grad_i log Phi     = -2 a b d^(2b-2) / (1 + a d^(2b)) (y_i - y_j)
      grad_i log(1-Phi)  =  2 b / (d^2 (1 + a d^(2b)))     (y_i - y_c)

Readings where the paper is silent (the CUDA path takes the same ones):
1. edges are the directed entries (i, j) of the symmetric graph's CSR, so each
   undirected edge appears twice; only the source y_i moves;
2. epochs are synchronous: every term of epoch e uses the positions at the start
   of the epoch, and their sum is applied at its end (the order of the sequential
   loop is not defined for a parallel machine; this makes every epoch a pure
   function of its input);
3. the repulsive term uses d^2 + eps (eps = 1e-3) in its denominator, and a drawn
   c equal to i is skipped; the attractive term is 0 when d = 0;
4. each coordinate of every term is clipped to [-4, 4] before it is summed;
5. the draws are counter-based: h(t) = splitmix64 output for the counter
   t = (e << 40) + (q << 4) + s  xor  seed  (q = the edge's CSR entry, s = 0 for
   the edge's own draw, 1..n_neg for its negatives); the edge is taken when
   (h >> 40) 2^-24 < p, and negative s is vertex p0 + ((h >> 32) n_s >> 32) of
   the point's sample [p0, p0 + n_s).
"""
from __future__ import annotations

import numpy as np

EPS = 1e-3
CLIP = 4.0
MASK64 = (1 << 64) - 1


def splitmix64(x):
    """One output of splitmix64 (Steele, Lea & Flood 2014) for the state x, i.e.
    the generator's mix of x + 0x9E3779B97F4A7C15; works on Python ints or uint64
    arrays (arithmetic mod 2^64)."""
    if isinstance(x, np.ndarray):
        with np.errstate(over="ignore"):
            z = x.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            return z ^ (z >> np.uint64(31))
    z = (int(x) + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def draw(seed, e, q, s):
    """h for epoch e, CSR entry q (array), draw s (reading 5)."""
    q = np.asarray(q, dtype=np.uint64)
    t = (np.uint64(e) << np.uint64(40)) + (q << np.uint64(4)) + np.uint64(s)
    return splitmix64(t ^ np.uint64(seed & MASK64))


def taken(h, p):
    """Edge decision of reading 5: the 24-bit uniform below the FP32 weight."""
    u = (h >> np.uint64(40)).astype(np.float64) * 2.0 ** -24
    return u < np.asarray(p, dtype=np.float32).astype(np.float64)


def vertex(h, p0, n_s):
    """Negative vertex of reading 5 (exact integer multiply-shift)."""
    hi = h >> np.uint64(32)
    with np.errstate(over="ignore"):
        return np.asarray(p0, dtype=np.int64) + (
            (hi * np.asarray(n_s, dtype=np.uint64)) >> np.uint64(32)).astype(np.int64)


def fit_ab(min_dist=0.1, spread=1.0):
    """(a, b) of Sec. 3.2: least squares of 1 / (1 + a d^(2b)) against Psi on 300
    points of [0, 3 spread] (scipy's curve_fit)."""
    from scipy.optimize import curve_fit

    d = np.linspace(0.0, 3.0 * spread, 300)
    psi = np.where(d < min_dist, 1.0, np.exp(-(d - min_dist) / spread))

    def phi(x, a, b):
        return 1.0 / (1.0 + a * x ** (2.0 * b))

    (a, b), _ = curve_fit(phi, d, psi, p0=(1.0, 1.0))
    return float(a), float(b)


def attract_coef(d2, a, b):
    """Coefficient of (y_i - y_j) in grad_i log Phi (0 at d = 0)."""
    d2 = np.asarray(d2, dtype=np.float64)
    out = np.zeros_like(d2)
    nz = d2 > 0
    out[nz] = -2.0 * a * b * d2[nz] ** (b - 1.0) / (1.0 + a * d2[nz] ** b)
    return out


def repulse_coef(d2, a, b):
    """Coefficient of (y_i - y_c) in grad_i log(1 - Phi), with d^2 + eps."""
    d2 = np.asarray(d2, dtype=np.float64)
    return 2.0 * b / ((EPS + d2) * (1.0 + a * d2 ** b))


def epoch_delta(row_ptr, col, w, Y, e, a, b, n_neg, seed, pt_off=None, rows=None):
    """Summed, clipped terms of epoch e for the points `rows` (all by default):
    D[r] for r in rows (float64, len(rows) x 2).  Terms are added per point in
    CSR order, each edge's attractive term before its negatives."""
    n = len(row_ptr) - 1
    pt_off = np.array([0, n], dtype=np.int64) if pt_off is None else np.asarray(pt_off)
    rows = np.arange(n) if rows is None else np.asarray(rows)
    Y = np.asarray(Y, dtype=np.float64)
    D = np.zeros((len(rows), 2))
    for r, i in enumerate(rows):
        s = np.searchsorted(pt_off, i, side="right") - 1
        p0, n_s = int(pt_off[s]), int(pt_off[s + 1] - pt_off[s])
        q = np.arange(row_ptr[i], row_ptr[i + 1], dtype=np.int64)
        if len(q) == 0:
            continue
        sel = taken(draw(seed, e, q, 0), w[q])
        for qq in q[sel]:
            j = int(col[qq])
            diff = Y[i] - Y[j]
            D[r] += np.clip(attract_coef(diff @ diff, a, b) * diff, -CLIP, CLIP)
            for t in range(1, n_neg + 1):
                c = int(vertex(draw(seed, e, np.array([qq]), t), p0, n_s)[0])
                if c == i:
                    continue
                diff = Y[i] - Y[c]
                D[r] += np.clip(repulse_coef(diff @ diff, a, b) * diff, -CLIP, CLIP)
    return D


def epoch(row_ptr, col, w, Y, e, n_epochs, a, b, alpha0, n_neg, seed, pt_off=None):
    """Positions after epoch e (reading 2): Y + alpha_e * D."""
    alpha = alpha0 * (1.0 - e / n_epochs)
    return np.asarray(Y, dtype=np.float64) + alpha * epoch_delta(row_ptr, col, w, Y, e, a, b,
                                                                  n_neg, seed, pt_off)
