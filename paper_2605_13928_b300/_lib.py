"""ctypes loader of libtsne.so and the C structs of include/tsne.h.

Argument marshalling only.  The library must be present (built in-tree by
``build.py``); there is no fallback of any kind: without it every call raises.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtsne.so")

TSNE_OK = 0
ERRORS = {
    -1: "TSNE_ERR_ARG", -2: "TSNE_ERR_CAPACITY", -3: "TSNE_ERR_CUDA", -4: "TSNE_ERR_TIMEOUT",
    -5: "TSNE_ERR_NOT_CONVERGED", -6: "TSNE_ERR_WORKSPACE", -7: "TSNE_ERR_DEVICE",
    -8: "TSNE_ERR_DEVICE_STATUS",
}
TSNE_ERR_NOT_CONVERGED = -5
TSNE_STATUS_BAD_INDEX, TSNE_STATUS_CAPACITY, TSNE_STATUS_TIMEOUT, TSNE_STATUS_NONFINITE = 1, 2, 4, 8
TSNE_KNN_FP32, TSNE_KNN_BF16_RERANK = 0, 1
TSNE_OP_KNN, TSNE_OP_AFFINITIES, TSNE_OP_KL_GRAD, TSNE_OP_PLAIN = 1, 2, 3, 4
TSNE_OP_PCA, TSNE_OP_PCA_TRANSFORM, TSNE_OP_KNN_GRAPH, TSNE_OP_UMAP_LAYOUT = 5, 6, 7, 8
TSNE_OP_UMAP_INIT = 9
TSNE_PCA_SKETCH = 64
(TSNE_VARIANT_AUTO, TSNE_VARIANT_DIRECT, TSNE_VARIANT_DIRECT_L, TSNE_VARIANT_DIRECT_S,
 TSNE_VARIANT_SYM, TSNE_VARIANT_DIRECT_M, TSNE_VARIANT_SYM4, TSNE_VARIANT_FUSED,
 TSNE_VARIANT_SYM4_FX) = (-1, 0, 1, 2, 3, 4, 5, 6, 7)
TSNE_MAX_SAMPLES = 512

# Every symbol include/tsne.h declares (checked by the CPU test-suite).
EXPORTS = (
    "tsne_params_default", "tsne_strerror", "tsne_version", "tsne_workspace_size",
    "tsne_knn", "tsne_affinities", "tsne_kl_grad", "tsne_kl_grad_plain", "tsne_step_plain",
    "tsne_step",
    "tsne_step_reset", "tsne_run", "tsne_kl_grad_noalloc",
    "tsne_mon_start", "tsne_mon_mark", "tsne_mon_stop", "tsne_mon_count", "tsne_mon_samples",
    "tsne_mon_event", "tsne_mon_free", "tsne_pca", "tsne_pca_transform", "tsne_knn_graph",
    "tsne_umap_layout", "tsne_umap_ab", "tsne_umap_init",
)
TSNE_NOALLOC_MAX_N = 65536


class TsneCsr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("cap", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class TsneBatch(ctypes.Structure):
    _fields_ = [("n_samples", ctypes.c_int), ("pt_off", ctypes.POINTER(ctypes.c_int64))]


class TsneParams(ctypes.Structure):
    _fields_ = [("perplexity", ctypes.c_float), ("k", ctypes.c_int), ("knn_mode", ctypes.c_int),
                ("cand_mult", ctypes.c_float), ("calib_tol", ctypes.c_float),
                ("calib_max_iter", ctypes.c_int), ("n_iter", ctypes.c_int),
                ("ee_iters", ctypes.c_int), ("ee", ctypes.c_float), ("mom_switch", ctypes.c_int),
                ("mom0", ctypes.c_float), ("mom1", ctypes.c_float), ("lr", ctypes.c_float),
                ("min_gain", ctypes.c_float), ("kl_every", ctypes.c_int),
                ("variant", ctypes.c_int), ("use_graph", ctypes.c_int)]


class TsneError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({strerror(code)})")


_lib = None


def lib():
    """The loaded libtsne.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"libtsne.so not found at {LIB_PATH}; build it with "
                "`python -m paper_2605_13928_b300.build` (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        P, i32, i64, f32, sz = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_float,
                                ctypes.c_size_t)
        csr, bat, prm = (ctypes.POINTER(TsneCsr), ctypes.POINTER(TsneBatch),
                         ctypes.POINTER(TsneParams))
        sig = {
            "tsne_params_default": (None, [prm]),
            "tsne_strerror": (ctypes.c_char_p, [i32]),
            "tsne_version": (ctypes.c_char_p, []),
            "tsne_workspace_size": (sz, [i32, i64, i32, i32, bat, prm]),
            "tsne_kl_grad": (i32, [csr, bat, P, f32, P, P, P, prm, P, sz, P, P]),
            "tsne_kl_grad_plain": (i32, [csr, bat, P, f32, P, P, P, sz, P, P]),
            "tsne_step_plain": (i32, [csr, bat, P, P, P, i32, prm, P, sz, P, P]),
            "tsne_step": (i32, [csr, bat, P, P, P, i32, prm, P, P, P, sz, P, P]),
            "tsne_step_reset": (i32, [P, sz, i32, P]),
        }
        optional = {
            "tsne_knn": (i32, [P, i64, i32, i32, bat, i32, f32, P, P, P, sz, P, P]),
            "tsne_affinities": (i32, [P, P, i64, i32, bat, f32, f32, i32, csr, P, P, P, sz, P,
                                      P]),
            "tsne_run": (i32, [P, i64, i32, bat, prm, P, P, P, P]),
            "tsne_kl_grad_noalloc": (i32, [csr, P, f32, P, P, P, P, P]),
            "tsne_mon_start": (P, [i32, ctypes.c_double, ctypes.c_char_p, ctypes.POINTER(i32)]),
            "tsne_mon_mark": (i32, [P, ctypes.c_char_p]),
            "tsne_mon_stop": (i32, [P]),
            "tsne_mon_count": (i64, [P, i32]),
            "tsne_mon_samples": (i32, [P, P, i64]),
            "tsne_mon_event": (i32, [P, i64, ctypes.POINTER(ctypes.c_double), ctypes.c_char_p,
                                     i32]),
            "tsne_mon_free": (None, [P]),
            "tsne_pca": (i32, [P, i64, i32, i64, i32, i32, P, P, P, P, P, P, P, P, sz, P, P]),
            "tsne_pca_transform": (i32, [P, i64, i32, i64, P, P, i32, P, P, sz, P, P]),
            "tsne_knn_graph": (i32, [P, P, i64, i32, bat, f32, i32, csr, P, P, P, P, sz, P, P]),
            "tsne_umap_layout": (i32, [csr, bat, P, i32, i32, i32, f32, f32, f32, i32,
                                       ctypes.c_uint64, P, sz, P, P]),
            "tsne_umap_ab": (i32, [f32, f32, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double)]),
            "tsne_umap_init": (i32, [P, i64, i64, P, P, sz, P, P]),
        }
        for name, (res, args) in list(sig.items()) + list(optional.items()):
            if not hasattr(L, name):
                if name in sig:
                    raise RuntimeError(f"libtsne.so lacks {name}")
                continue
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def strerror(code: int) -> str:
    try:
        return lib().tsne_strerror(int(code)).decode()
    except Exception:
        return ERRORS.get(code, "unknown")


def check(code: int, where: str) -> int:
    if code != TSNE_OK and code != TSNE_ERR_NOT_CONVERGED:
        raise TsneError(code, where)
    return code


def default_params(**over) -> TsneParams:
    p = TsneParams()
    lib().tsne_params_default(ctypes.byref(p))
    for k, v in over.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p
