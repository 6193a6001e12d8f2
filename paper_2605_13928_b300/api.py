"""PyTorch front end of libtsne.so: argument marshalling only.

Tensors are CUDA tensors; their device pointers and the current torch stream
are handed to the C ABI (include/tsne.h), whose kernels do all the work.  The
library must be built (``build.py``); a missing library raises.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib as L

_ALIGN = 256


def _stream(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t: Optional[torch.Tensor]):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _need(t: torch.Tensor, dtype, name, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t


class Batch:
    """Back-to-back independent samples: HOST offsets pt_off[S+1]."""

    def __init__(self, sizes: Sequence[int]):
        sizes = np.asarray(sizes, dtype=np.int64)
        if sizes.ndim != 1 or len(sizes) < 1 or len(sizes) > L.TSNE_MAX_SAMPLES:
            raise ValueError("1..512 samples")
        self.pt_off = np.zeros(len(sizes) + 1, dtype=np.int64)
        self.pt_off[1:] = np.cumsum(sizes)
        self._c = L.TsneBatch(len(sizes), self.pt_off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))

    @property
    def n(self) -> int:
        return int(self.pt_off[-1])

    @property
    def S(self) -> int:
        return len(self.pt_off) - 1

    def sizes(self):
        return np.diff(self.pt_off)

    def c(self):
        return ctypes.byref(self._c)


def _bc(batch: Optional[Batch]):
    return batch.c() if batch is not None else None


def _nsamp(batch):
    return batch.S if batch is not None else 1


class CSR:
    """Symmetric P on the device: row_ptr int64[n+1], col int32[cap], val float32[cap]."""

    def __init__(self, row_ptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor):
        self.row_ptr = _need(row_ptr, torch.int64, "row_ptr")
        self.col = _need(col, torch.int32, "col")
        self.val = _need(val, torch.float32, "val")
        if self.col.numel() != self.val.numel():
            raise ValueError("col and val must have the same capacity")
        self.n = self.row_ptr.numel() - 1
        self._c = L.TsneCsr(self.n, 0, self.col.numel(), _ptr(self.row_ptr), _ptr(self.col),
                            _ptr(self.val))

    @staticmethod
    def from_numpy(row_ptr, col, val, device="cuda") -> "CSR":
        return CSR(torch.as_tensor(np.asarray(row_ptr, dtype=np.int64), device=device),
                   torch.as_tensor(np.asarray(col, dtype=np.int32), device=device),
                   torch.as_tensor(np.asarray(val, dtype=np.float32), device=device))

    @staticmethod
    def empty(n: int, cap: int, device="cuda") -> "CSR":
        return CSR(torch.zeros(n + 1, dtype=torch.int64, device=device),
                   torch.zeros(max(cap, 1), dtype=torch.int32, device=device),
                   torch.zeros(max(cap, 1), dtype=torch.float32, device=device))

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1].item())

    def to_numpy(self):
        nnz = self.nnz
        return (self.row_ptr.cpu().numpy(), self.col[:nnz].cpu().numpy(),
                self.val[:nnz].cpu().numpy())

    def c(self):
        return ctypes.byref(self._c)


class Workspace:
    """Caller-owned scratch for the library (256-byte aligned device bytes).

    tsne_step's device iteration counter lives in it, so a run keeps one
    Workspace for all its steps."""

    def __init__(self, nbytes: int, device="cuda"):
        self.nbytes = int(nbytes)
        self._buf = torch.empty(self.nbytes + _ALIGN, dtype=torch.uint8, device=device)
        base = self._buf.data_ptr()
        self.offset = (-base) % _ALIGN
        self.ptr = ctypes.c_void_p(base + self.offset)

    def ensure(self, nbytes: int) -> "Workspace":
        return self if nbytes <= self.nbytes else Workspace(nbytes, self._buf.device)


def workspace_size(op: int, n: int, d: int = 0, k: int = 0, batch: Optional[Batch] = None,
                   params: Optional[L.TsneParams] = None) -> int:
    return int(L.lib().tsne_workspace_size(op, n, d, k, _bc(batch),
                                           ctypes.byref(params) if params is not None else None))


def _ws(op, n, d, k, batch, params, ws: Optional[Workspace], device):
    need = workspace_size(op, n, d, k, batch, params)
    if ws is None or ws.nbytes < need:
        ws = Workspace(max(need, 1), device)
    return ws


def new_status(device="cuda") -> torch.Tensor:
    return torch.zeros(1, dtype=torch.int32, device=device)


# ----------------------------------------------------------------------------- gradient
def kl_grad(P: CSR, Y: torch.Tensor, alpha: float = 1.0, batch: Optional[Batch] = None,
            want_grad: bool = True, want_kl: bool = False, params: Optional[L.TsneParams] = None,
            ws: Optional[Workspace] = None, status: Optional[torch.Tensor] = None):
    """Exact dKL_alpha/dY (n x 2), Z per sample (float64) and KL_alpha per sample."""
    n = P.n
    _need(Y, torch.float32, "Y", (n, 2))
    dev = Y.device
    S = _nsamp(batch)
    grad = torch.empty_like(Y) if want_grad else None
    Z = torch.empty(S, dtype=torch.float64, device=dev)
    kl = torch.empty(S, dtype=torch.float64, device=dev) if want_kl else None
    ws = _ws(L.TSNE_OP_KL_GRAD, n, 0, 0, batch, params, ws, dev)
    rc = L.lib().tsne_kl_grad(P.c(), _bc(batch), _ptr(Y), float(alpha), _ptr(grad), _ptr(Z),
                              _ptr(kl), ctypes.byref(params) if params is not None else None,
                              ws.ptr, ws.nbytes, _ptr(status), _stream(dev))
    L.check(rc, "tsne_kl_grad")
    return grad, Z, kl


def kl_grad_noalloc(P: CSR, Y: torch.Tensor, alpha: float = 1.0, want_grad: bool = True,
                    want_kl: bool = False, status: Optional[torch.Tensor] = None):
    """tsne_kl_grad_noalloc: the exact gradient of one sample (n <= 65,536) using
    the library's fixed scratch array instead of a workspace, for callers that
    cannot allocate device memory.  Calls that overlap on the GPU share that
    array and race.  (This wrapper allocates its output tensors through torch;
    a caller without an allocator passes its own buffers to the C entry.)"""
    n = P.n
    _need(Y, torch.float32, "Y", (n, 2))
    dev = Y.device
    grad = torch.empty_like(Y) if want_grad else None
    Z = torch.empty(1, dtype=torch.float64, device=dev)
    kl = torch.empty(1, dtype=torch.float64, device=dev) if want_kl else None
    rc = L.lib().tsne_kl_grad_noalloc(P.c(), _ptr(Y), float(alpha), _ptr(grad), _ptr(Z), _ptr(kl),
                                      _ptr(status), _stream(dev))
    L.check(rc, "tsne_kl_grad_noalloc")
    return grad, Z, kl


def kl_grad_plain(P: CSR, Y: torch.Tensor, alpha: float = 1.0, batch: Optional[Batch] = None,
                  ws: Optional[Workspace] = None, status: Optional[torch.Tensor] = None):
    """The same gradient through the plain GPU form (comparison baseline)."""
    n = P.n
    _need(Y, torch.float32, "Y", (n, 2))
    dev = Y.device
    grad = torch.empty_like(Y)
    Z = torch.empty(_nsamp(batch), dtype=torch.float64, device=dev)
    ws = _ws(L.TSNE_OP_PLAIN, n, 0, 0, batch, None, ws, dev)
    rc = L.lib().tsne_kl_grad_plain(P.c(), _bc(batch), _ptr(Y), float(alpha), _ptr(grad), _ptr(Z),
                                    ws.ptr, ws.nbytes, _ptr(status), _stream(dev))
    L.check(rc, "tsne_kl_grad_plain")
    return grad, Z


def step_plain(P: CSR, Y: torch.Tensor, U: torch.Tensor, G: torch.Tensor, it: int,
               params: L.TsneParams, batch: Optional[Batch] = None,
               ws: Optional[Workspace] = None,
               status: Optional[torch.Tensor] = None) -> Workspace:
    """One optimiser iteration through the plain GPU form (comparison baseline)."""
    n = P.n
    for t, nm in ((Y, "Y"), (U, "U"), (G, "G")):
        _need(t, torch.float32, nm, (n, 2))
    dev = Y.device
    ws = _ws(L.TSNE_OP_PLAIN, n, 0, 0, batch, None, ws, dev)
    rc = L.lib().tsne_step_plain(P.c(), _bc(batch), _ptr(Y), _ptr(U), _ptr(G), int(it),
                                 ctypes.byref(params), ws.ptr, ws.nbytes, _ptr(status),
                                 _stream(dev))
    L.check(rc, "tsne_step_plain")
    return ws


def step(P: CSR, Y: torch.Tensor, U: torch.Tensor, G: torch.Tensor, it: int,
         params: L.TsneParams, batch: Optional[Batch] = None, Z: Optional[torch.Tensor] = None,
         kl: Optional[torch.Tensor] = None, ws: Optional[Workspace] = None,
         status: Optional[torch.Tensor] = None) -> Workspace:
    """One optimiser iteration in place on Y, U (velocity) and G (gains)."""
    n = P.n
    for t, nm in ((Y, "Y"), (U, "U"), (G, "G")):
        _need(t, torch.float32, nm, (n, 2))
    if Z is not None:
        _need(Z, torch.float64, "Z", (_nsamp(batch),))
    if kl is not None:
        _need(kl, torch.float64, "kl")
        if params.kl_every > 0 and kl.numel() < (params.n_iter // params.kl_every) * _nsamp(batch):
            raise ValueError("kl needs (n_iter // kl_every) * S entries")
    dev = Y.device
    ws = _ws(L.TSNE_OP_KL_GRAD, n, 0, 0, batch, params, ws, dev)
    rc = L.lib().tsne_step(P.c(), _bc(batch), _ptr(Y), _ptr(U), _ptr(G), int(it),
                           ctypes.byref(params), _ptr(Z), _ptr(kl), ws.ptr, ws.nbytes,
                           _ptr(status), _stream(dev))
    L.check(rc, "tsne_step")
    return ws


def step_reset(ws: Workspace, it: int = 0, device="cuda"):
    L.check(L.lib().tsne_step_reset(ws.ptr, ws.nbytes, int(it), _stream(device)),
            "tsne_step_reset")


# ----------------------------------------------------------------------------- kNN / P
def knn(X: torch.Tensor, k: int, batch: Optional[Batch] = None, mode: int = L.TSNE_KNN_FP32,
        cand_mult: float = 2.0, ws: Optional[Workspace] = None,
        status: Optional[torch.Tensor] = None):
    """k nearest neighbours within each sample: (idx int32 n x k, d2 float32 n x k)."""
    _need(X, torch.float32, "X")
    if X.dim() != 2:
        raise ValueError("X must be n x d")
    n, d = X.shape
    dev = X.device
    idx = torch.empty((n, k), dtype=torch.int32, device=dev)
    d2 = torch.empty((n, k), dtype=torch.float32, device=dev)
    ws = _ws(L.TSNE_OP_KNN, n, d, k, batch, L.default_params(knn_mode=mode, cand_mult=cand_mult),
             ws, dev)
    rc = L.lib().tsne_knn(_ptr(X), n, d, k, _bc(batch), int(mode), float(cand_mult), _ptr(idx),
                          _ptr(d2), ws.ptr, ws.nbytes, _ptr(status), _stream(dev))
    L.check(rc, "tsne_knn")
    return idx, d2


def affinities(idx: torch.Tensor, d2: torch.Tensor, perplexity: float,
               batch: Optional[Batch] = None, tol: float = 1e-5, max_iter: int = 200,
               ws: Optional[Workspace] = None, status: Optional[torch.Tensor] = None):
    """Calibrated, symmetrised P as CSR, per-row beta and the count of flagged rows."""
    _need(idx, torch.int32, "idx")
    n, k = idx.shape
    _need(d2, torch.float32, "d2", (n, k))
    dev = idx.device
    P = CSR.empty(n, 2 * n * k, dev)
    beta = torch.empty(n, dtype=torch.float32, device=dev)
    n_bad = torch.zeros(1, dtype=torch.int64, device=dev)
    ws = _ws(L.TSNE_OP_AFFINITIES, n, 0, k, batch, None, ws, dev)
    rc = L.lib().tsne_affinities(_ptr(idx), _ptr(d2), n, k, _bc(batch), float(perplexity),
                                 float(tol), int(max_iter), P.c(), _ptr(beta), _ptr(n_bad),
                                 ws.ptr, ws.nbytes, _ptr(status), _stream(dev))
    L.check(rc, "tsne_affinities")
    return P, beta, n_bad


def knn_graph(idx: torch.Tensor, d2: torch.Tensor, batch: Optional[Batch] = None,
              tol: float = 1e-5, max_iter: int = 200, ws: Optional[Workspace] = None,
              status: Optional[torch.Tensor] = None):
    """Fuzzy neighbour graph (UMAP's fuzzy simplicial set) from kNN lists:
    (G as CSR, rho, sigma, count of rows that could not reach log2 k)."""
    _need(idx, torch.int32, "idx")
    n, k = idx.shape
    _need(d2, torch.float32, "d2", (n, k))
    dev = idx.device
    G = CSR.empty(n, 2 * n * k, dev)
    rho = torch.empty(n, dtype=torch.float32, device=dev)
    sigma = torch.empty(n, dtype=torch.float32, device=dev)
    n_bad = torch.zeros(1, dtype=torch.int64, device=dev)
    ws = _ws(L.TSNE_OP_KNN_GRAPH, n, 0, k, batch, None, ws, dev)
    rc = L.lib().tsne_knn_graph(_ptr(idx), _ptr(d2), n, k, _bc(batch), float(tol), int(max_iter),
                                G.c(), _ptr(rho), _ptr(sigma), _ptr(n_bad), ws.ptr, ws.nbytes,
                                _ptr(status), _stream(dev))
    L.check(rc, "tsne_knn_graph")
    return G, rho, sigma, n_bad


def umap_ab(min_dist: float = 0.1, spread: float = 1.0):
    """(a, b) of UMAP's low-dimensional membership 1 / (1 + a d^(2b)), fitted by
    the library (tsne_umap_ab: FP64 Levenberg-Marquardt on the host)."""
    a, b = ctypes.c_double(0.0), ctypes.c_double(0.0)
    L.check(L.lib().tsne_umap_ab(float(min_dist), float(spread), ctypes.byref(a),
                                 ctypes.byref(b)), "tsne_umap_ab")
    return a.value, b.value


def umap_init(scores: torch.Tensor, ws: Optional[Workspace] = None,
              status: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Initial UMAP layout from PCA scores through tsne_umap_init: the first two
    columns, centred and scaled into [-10, 10]."""
    _need(scores, torch.float32, "scores")
    if scores.dim() != 2 or scores.shape[1] < 2 or scores.stride(1) != 1:
        raise ValueError("scores must be n x k (k >= 2) with unit column stride")
    n = scores.shape[0]
    dev = scores.device
    U = torch.empty((n, 2), dtype=torch.float32, device=dev)
    ws = _ws(L.TSNE_OP_UMAP_INIT, n, 0, 0, None, None, ws, dev)
    L.check(L.lib().tsne_umap_init(_ptr(scores), n, scores.stride(0), _ptr(U), ws.ptr, ws.nbytes,
                                   _ptr(status), _stream(dev)), "tsne_umap_init")
    return U


def umap_layout(G: CSR, Y: torch.Tensor, n_epochs: int = 200, a: Optional[float] = None,
                b: Optional[float] = None, min_dist: float = 0.1, spread: float = 1.0,
                alpha0: float = 1.0, n_neg: int = 5, seed: int = 0, epoch0: int = 0,
                n_run: Optional[int] = None, batch: Optional[Batch] = None,
                ws: Optional[Workspace] = None, status: Optional[torch.Tensor] = None) -> Workspace:
    """UMAP layout optimisation of the fuzzy graph G in place on Y (n x 2): epochs
    epoch0 .. epoch0 + n_run - 1 (all remaining by default) of an n_epochs
    schedule; (a, b) from umap_ab(min_dist, spread) unless given."""
    n = G.n
    _need(Y, torch.float32, "Y", (n, 2))
    if a is None or b is None:
        a, b = umap_ab(min_dist, spread)
    if n_run is None:
        n_run = n_epochs - epoch0
    ws = _ws(L.TSNE_OP_UMAP_LAYOUT, n, 0, 0, batch, None, ws, Y.device)
    rc = L.lib().tsne_umap_layout(G.c(), _bc(batch), _ptr(Y), int(n_epochs), int(epoch0),
                                  int(n_run), float(a), float(b), float(alpha0), int(n_neg),
                                  int(seed) & ((1 << 64) - 1), ws.ptr, ws.nbytes, _ptr(status),
                                  _stream(Y.device))
    L.check(rc, "tsne_umap_layout")
    return ws


def run(X, Y0, params: L.TsneParams, batch: Optional[Batch] = None, kl_trace: bool = True,
        stream: Optional[torch.cuda.Stream] = None):
    """Whole embedding through tsne_run.  X and Y0 may be numpy (host) arrays or
    CUDA tensors; returns (Y, kl_trace[n_iter // kl_every, S] or None, status)."""
    host = isinstance(X, np.ndarray)
    if host:
        Xa = np.ascontiguousarray(X, dtype=np.float32)
        Ya = np.array(Y0, dtype=np.float32, order="C", copy=True)
        n, d = Xa.shape
        px, py = Xa.ctypes.data_as(ctypes.c_void_p), Ya.ctypes.data_as(ctypes.c_void_p)
    else:
        Xa = _need(X, torch.float32, "X")
        n, d = Xa.shape
        Ya = _need(Y0, torch.float32, "Y0", (n, 2)).clone()
        px, py = _ptr(Xa), _ptr(Ya)
    S = _nsamp(batch)
    m = params.n_iter // params.kl_every if (kl_trace and params.kl_every > 0) else 0
    tr = np.zeros(max(m * S, 1), dtype=np.float64)
    st = ctypes.c_int32(0)
    s = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream
    rc = L.lib().tsne_run(px, n, d, _bc(batch), ctypes.byref(params), py,
                          tr.ctypes.data_as(ctypes.c_void_p) if m else None, ctypes.byref(st),
                          ctypes.c_void_p(s))
    L.check(rc, "tsne_run")
    return Ya, (tr[:m * S].reshape(m, S) if m else None), int(st.value)


# ----------------------------------------------------------------------------- PCA
def _tma_layout(A: torch.Tensor) -> torch.Tensor:
    """tsne_pca reads A by TMA: 16-byte aligned rows.  A matrix whose row
    stride is not a multiple of 4 floats is copied once into a padded one."""
    if A.stride(0) % 4 == 0 and A.data_ptr() % 16 == 0:
        return A
    n, g = A.shape
    P = torch.zeros((n, (g + 3) // 4 * 4), dtype=A.dtype, device=A.device)
    P[:, :g] = A
    return P[:, :g]


def pca(A: torch.Tensor, k: int = 50, n_power: int = 2, omega: Optional[torch.Tensor] = None,
        seed: int = 0, ws: Optional[Workspace] = None, status: Optional[torch.Tensor] = None):
    """k principal components of the rows of A (n x g float32, CUDA) through
    tsne_pca.  omega: g x 64 Gaussian test matrix (drawn from `seed` on the
    host when not given).  Returns a dict of CUDA tensors: scores (n x k),
    components (k x g), sigma, explained_variance (k, float64), mean (g,
    float64) and total_var (1, float64)."""
    if not isinstance(A, torch.Tensor) or not A.is_cuda or A.dtype != torch.float32 or A.dim() != 2:
        raise ValueError("A must be a 2-D float32 CUDA tensor")
    if A.stride(1) != 1:
        raise ValueError("A must have unit column stride")
    n, g = A.shape
    A = _tma_layout(A)
    lda = A.stride(0)
    dev = A.device
    if omega is None:
        rng = np.random.default_rng(seed)
        omega = torch.tensor(rng.standard_normal(size=(g, L.TSNE_PCA_SKETCH)).astype(np.float32),
                             device=dev)
    _need(omega, torch.float32, "omega", (g, L.TSNE_PCA_SKETCH))
    out = {"scores": torch.empty((n, k), dtype=torch.float32, device=dev),
           "components": torch.empty((k, g), dtype=torch.float32, device=dev),
           "sigma": torch.empty(k, dtype=torch.float64, device=dev),
           "explained_variance": torch.empty(k, dtype=torch.float64, device=dev),
           "mean": torch.empty(g, dtype=torch.float64, device=dev),
           "total_var": torch.empty(1, dtype=torch.float64, device=dev)}
    ws = _ws(L.TSNE_OP_PCA, n, g, 0, None, None, ws, dev)
    rc = L.lib().tsne_pca(_ptr(A), n, g, lda, int(k), int(n_power), _ptr(omega),
                          _ptr(out["scores"]), _ptr(out["components"]), _ptr(out["sigma"]),
                          _ptr(out["explained_variance"]), _ptr(out["mean"]),
                          _ptr(out["total_var"]), ws.ptr, ws.nbytes, _ptr(status), _stream(dev))
    L.check(rc, "tsne_pca")
    return out


def pca_transform(A: torch.Tensor, mean: torch.Tensor, components: torch.Tensor,
                  ws: Optional[Workspace] = None, status: Optional[torch.Tensor] = None):
    """Scores (A - mean) components^T of new rows through tsne_pca_transform."""
    if not isinstance(A, torch.Tensor) or not A.is_cuda or A.dtype != torch.float32 or A.dim() != 2:
        raise ValueError("A must be a 2-D float32 CUDA tensor")
    if A.stride(1) != 1:
        raise ValueError("A must have unit column stride")
    n, g = A.shape
    A = _tma_layout(A)
    k = components.shape[0]
    _need(mean, torch.float64, "mean", (g,))
    _need(components, torch.float32, "components", (k, g))
    dev = A.device
    scores = torch.empty((n, k), dtype=torch.float32, device=dev)
    ws = _ws(L.TSNE_OP_PCA_TRANSFORM, n, g, 0, None, None, ws, dev)
    rc = L.lib().tsne_pca_transform(_ptr(A), n, g, A.stride(0), _ptr(mean), _ptr(components), k,
                                    _ptr(scores), ws.ptr, ws.nbytes, _ptr(status), _stream(dev))
    L.check(rc, "tsne_pca_transform")
    return scores
