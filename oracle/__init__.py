"""FP64 CPU oracle of exact t-SNE -- TEST INFRASTRUCTURE ONLY.

Only the tests, the package smoke check and the benchmark's CPU-baseline leg may
import this module.  It shares no code with the CUDA path and never calls it.
Every function is a numpy front end to the plain C in ``tsne_oracle.c``; the C
file's header lists the definitions followed (textbook exact t-SNE: van der
Maaten & Hinton 2008; kNN-sparse P: van der Maaten 2014) and the readings
taken where they are silent.  All arrays are float64 / int64 / int32 numpy.
"""
import ctypes
import numpy as np

from .build import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build())
        P = ctypes.c_void_p
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        _lib.oracle_knn_rows.argtypes = [P, i64, i32, i32, P, i64, P, P]
        _lib.oracle_knn_rows.restype = None
        _lib.oracle_calibrate.argtypes = [P, i64, i32, f64, f64, i32, P, P, P]
        _lib.oracle_calibrate.restype = i64
        _lib.oracle_cond_at_beta.argtypes = [P, i64, i32, P, P]
        _lib.oracle_cond_at_beta.restype = None
        _lib.oracle_symmetrize.argtypes = [P, P, i64, i32, P, P, P]
        _lib.oracle_symmetrize.restype = i64
        _lib.oracle_Z.argtypes = [P, i64]
        _lib.oracle_Z.restype = f64
        _lib.oracle_grad.argtypes = [P, P, P, P, i64, f64, P]
        _lib.oracle_grad.restype = f64
        _lib.oracle_forces_rows.argtypes = [P, P, P, P, i64, P, i64, P, P, P, P, P]
        _lib.oracle_forces_rows.restype = None
        _lib.oracle_kl.argtypes = [P, P, P, P, i64, f64, f64]
        _lib.oracle_kl.restype = f64
        _lib.oracle_run.argtypes = [P, P, P, i64, P, P, P, i32, i32, f64, i32, f64, f64,
                                    f64, f64, i32, P]
        _lib.oracle_run.restype = None
        _lib.oracle_num_threads.argtypes = []
        _lib.oracle_num_threads.restype = i32
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return lib().oracle_num_threads()


class CSR:
    """Symmetric P as CSR: row_ptr int64[n+1], col int32[nnz] ascending per row, val float64."""

    def __init__(self, row_ptr, col, val):
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = _f64(val)
        self.n = len(self.row_ptr) - 1

    @property
    def nnz(self):
        return int(self.row_ptr[-1])

    def dense(self):
        D = np.zeros((self.n, self.n))
        for i in range(self.n):
            s, e = self.row_ptr[i], self.row_ptr[i + 1]
            D[i, self.col[s:e]] = self.val[s:e]
        return D

    @staticmethod
    def from_dense(D):
        D = np.asarray(D, dtype=np.float64)
        n = D.shape[0]
        rows, cols = np.nonzero(D)
        order = np.lexsort((cols, rows))
        rows, cols = rows[order], cols[order]
        row_ptr = np.zeros(n + 1, dtype=np.int64)
        np.add.at(row_ptr, rows + 1, 1)
        return CSR(np.cumsum(row_ptr), cols, D[rows, cols])


def knn(X, k, rows=None):
    """k nearest neighbours (self excluded) by (d2, index); returns (idx int32, d2 float64)."""
    X = _f64(X)
    n, d = X.shape
    rows_a = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    m = n if rows_a is None else len(rows_a)
    idx = np.empty((m, k), dtype=np.int32)
    d2 = np.empty((m, k), dtype=np.float64)
    lib().oracle_knn_rows(_p(X), n, d, k, _p(rows_a), m, _p(idx), _p(d2))
    return idx, d2


def calibrate(d2, perplexity, tol=1e-12, max_iter=200):
    """Per-row beta so exp(H(p_{.|i})) = perplexity; returns (pcond, beta, flag)."""
    d2 = _f64(d2)
    n, k = d2.shape
    pc = np.empty_like(d2)
    beta = np.empty(n)
    flag = np.empty(n, dtype=np.int8)
    lib().oracle_calibrate(_p(d2), n, k, float(perplexity), float(tol), int(max_iter),
                           _p(pc), _p(beta), _p(flag))
    return pc, beta, flag


def cond_at_beta(d2, beta):
    """p_{j|i} of every row at the given beta (Gibbs form; beta = inf: uniform on ties)."""
    d2 = _f64(d2)
    beta = _f64(beta)
    n, k = d2.shape
    pc = np.empty_like(d2)
    lib().oracle_cond_at_beta(_p(d2), n, k, _p(beta), _p(pc))
    return pc


def symmetrize(idx, pcond):
    """P = (P_cond + P_cond^T) / (2N) as CSR."""
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    pcond = _f64(pcond)
    n, k = idx.shape
    row_ptr = np.empty(n + 1, dtype=np.int64)
    col = np.empty(2 * n * k, dtype=np.int32)
    val = np.empty(2 * n * k, dtype=np.float64)
    nnz = lib().oracle_symmetrize(_p(idx), _p(pcond), n, k, _p(row_ptr), _p(col), _p(val))
    return CSR(row_ptr, col[:nnz].copy(), val[:nnz].copy())


def affinities(X, k, perplexity):
    idx, d2 = knn(X, k)
    pc, beta, flag = calibrate(d2, perplexity)
    return symmetrize(idx, pc), idx, d2, pc, beta, flag


def Z(Y):
    Y = _f64(Y)
    return lib().oracle_Z(_p(Y), Y.shape[0])


def grad(P, Y, alpha=1.0):
    """Exact dKL_alpha/dY (n x 2) and Z."""
    Y = _f64(Y)
    g = np.empty_like(Y)
    z = lib().oracle_grad(_p(P.row_ptr), _p(P.col), _p(P.val), _p(Y), Y.shape[0],
                          float(alpha), _p(g))
    return g, z


def forces_rows(P, Y, rows=None, scales=False):
    """Per-row attraction Fa, repulsion Fr and Z_i for the given rows (all if None).
    With scales=True also the sums of the terms' magnitudes (Aa, Ar), the scale
    of the rounding error of any floating-point evaluation of those sums."""
    Y = _f64(Y)
    rows_a = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    m = Y.shape[0] if rows_a is None else len(rows_a)
    Fa = np.empty((m, 2)); Fr = np.empty((m, 2)); Zi = np.empty(m)
    Aa = np.empty(m) if scales else None
    Ar = np.empty(m) if scales else None
    lib().oracle_forces_rows(_p(P.row_ptr), _p(P.col), _p(P.val), _p(Y), Y.shape[0],
                             _p(rows_a), m, _p(Fa), _p(Fr), _p(Zi), _p(Aa), _p(Ar))
    if scales:
        return Fa, Fr, Zi, Aa, Ar
    return Fa, Fr, Zi


def kl(P, Y, alpha=1.0, Zval=0.0):
    Y = _f64(Y)
    return lib().oracle_kl(_p(P.row_ptr), _p(P.col), _p(P.val), _p(Y), Y.shape[0],
                           float(alpha), float(Zval))


def run(P, Y0, n_iter, ee_iters, ee=12.0, mom_switch=None, mom0=0.5, mom1=0.8, eta=None,
        min_gain=0.01, kl_every=0, U0=None, gains0=None):
    """Full optimiser; returns (Y, U, gains, kl_trace)."""
    Y = _f64(Y0).copy()
    n = Y.shape[0]
    U = np.zeros_like(Y) if U0 is None else _f64(U0).copy()
    G = np.ones_like(Y) if gains0 is None else _f64(gains0).copy()
    if eta is None or eta <= 0:
        eta = n / 12.0
    if mom_switch is None:
        mom_switch = ee_iters
    m = n_iter // kl_every if kl_every > 0 else 0
    tr = np.zeros(max(m, 1))
    lib().oracle_run(_p(P.row_ptr), _p(P.col), _p(P.val), n, _p(Y), _p(U), _p(G), int(n_iter),
                     int(ee_iters), float(ee), int(mom_switch), float(mom0), float(mom1),
                     float(eta), float(min_gain), int(kl_every), _p(tr) if m > 0 else None)
    return Y, U, G, tr[:m]
