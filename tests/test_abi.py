"""CPU checks of the C ABI: libtsne.so builds, loads, exports every function
include/tsne.h declares, and rejects bad arguments on the host (no kernel is
launched by any call here)."""
import ctypes
import os
import re

import pytest

from paper_2605_13928_b300 import _lib as L
from paper_2605_13928_b300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "tsne.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(tsne_\w+)\s*\(", src, re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(L.EXPORTS) == names


def test_defaults_and_strings(lib):
    p = L.default_params()
    assert (p.perplexity, p.k, p.ee, p.ee_iters, p.mom0) == (30.0, 90, 12.0, 250, 0.5)
    assert abs(p.mom1 - 0.8) < 1e-7 and p.lr == 0.0
    assert p.knn_mode == L.TSNE_KNN_BF16_RERANK and p.cand_mult == 2.0
    assert lib.tsne_strerror(L.TSNE_OK) == b"ok"
    assert b"workspace" in lib.tsne_strerror(-6)
    assert b"sm_103a" in lib.tsne_version()


def test_workspace_size_grows_with_n(lib):
    a = lib.tsne_workspace_size(L.TSNE_OP_KL_GRAD, 1000, 0, 0, None, None)
    b = lib.tsne_workspace_size(L.TSNE_OP_KL_GRAD, 100000, 0, 0, None, None)
    assert 0 < a < b and a % 256 == 0
    assert lib.tsne_workspace_size(L.TSNE_OP_PLAIN, 1000, 0, 0, None, None) > 0


def test_symmetric_scratch_switches_to_fixed_point(lib):
    """The symmetric split's partial buffers take 16 B per point and group pair
    (O(N^2)); the tiled fixed-point form (SYM4_FX, and AUTO once its tiles fill
    the GPU eight times over) takes 16 B per point.  SYM4 keeps the buffers up to
    32 GiB and takes the fixed-point form beyond (about 2M points)."""
    KG = L.TSNE_OP_KL_GRAD

    def ws(n, variant):
        return lib.tsne_workspace_size(KG, n, 0, 0, None,
                                       ctypes.byref(L.default_params(variant=variant)))

    n = 1_000_000
    G = (n + 1023) // 1024
    bufs = 2 * 8 * (G * (G - 1) // 2) * 1024
    assert ws(n, L.TSNE_VARIANT_SYM4) - ws(n, L.TSNE_VARIANT_SYM4_FX) >= bufs - 16 * n
    assert ws(n, L.TSNE_VARIANT_AUTO) == ws(n, L.TSNE_VARIANT_SYM4_FX) < 200 * n  # O(N)
    # below 8 waves of tiles (three CTAs per SM) AUTO keeps the buffers
    n = 50_000
    assert ws(n, L.TSNE_VARIANT_AUTO) == ws(n, L.TSNE_VARIANT_SYM4) > ws(n, L.TSNE_VARIANT_SYM4_FX)
    n = 2_500_000
    # buffers would take 49 GB
    assert ws(n, L.TSNE_VARIANT_SYM4) == ws(n, L.TSNE_VARIANT_SYM4_FX) < 200 * n
    assert ws(n, L.TSNE_VARIANT_SYM) > 20 * 2 ** 30  # 2048-point groups: buffers, 24 GB


def test_host_argument_errors(lib):
    fake = ctypes.c_void_p(1 << 40)  # never dereferenced: every call below fails its checks
    csr = L.TsneCsr(10, 0, 20, fake, fake, fake)
    # missing P / Y / Z
    assert lib.tsne_kl_grad(None, None, fake, 1.0, None, fake, None, None, fake, 1 << 30,
                            None, None) == -1
    assert lib.tsne_kl_grad(ctypes.byref(csr), None, None, 1.0, None, fake, None, None, fake,
                            1 << 30, None, None) == -1
    # workspace too small / misaligned
    assert lib.tsne_kl_grad(ctypes.byref(csr), None, fake, 1.0, None, fake, None, None, fake,
                            16, None, None) == -6
    assert lib.tsne_kl_grad(ctypes.byref(csr), None, fake, 1.0, None, fake, None, None,
                            ctypes.c_void_p((1 << 40) + 8), 1 << 30, None, None) == -6
    # batch offsets that do not cover n, or a sample with a single point
    off = (ctypes.c_int64 * 3)(0, 4, 9)
    bt = L.TsneBatch(2, off)
    assert lib.tsne_kl_grad(ctypes.byref(csr), ctypes.byref(bt), fake, 1.0, None, fake, None,
                            None, fake, 1 << 30, None, None) == -1
    off1 = (ctypes.c_int64 * 3)(0, 9, 10)
    bt1 = L.TsneBatch(2, off1)
    assert lib.tsne_kl_grad(ctypes.byref(csr), ctypes.byref(bt1), fake, 1.0, None, fake, None,
                            None, fake, 1 << 30, None, None) == -1
    # step without params, negative iteration below -1
    p = L.default_params()
    assert lib.tsne_step(ctypes.byref(csr), None, fake, fake, fake, 0, None, None, None, fake,
                         1 << 30, None, None) == -1
    assert lib.tsne_step(ctypes.byref(csr), None, fake, fake, fake, -2, ctypes.byref(p), None,
                         None, fake, 1 << 30, None, None) == -1
    assert lib.tsne_step_reset(None, 0, 0, None) == -6


def test_umap_layout_host_argument_errors(lib):
    fake = ctypes.c_void_p(1 << 40)  # never dereferenced: every call below fails its checks
    csr = L.TsneCsr(10, 30, 30, fake, fake, fake)
    G = ctypes.byref(csr)

    def call(Y=fake, n_epochs=200, epoch0=0, n_run=1, a=1.5, b=0.9, alpha0=1.0, n_neg=5,
             ws=fake, ws_bytes=1 << 30, graph=G):
        return lib.tsne_umap_layout(graph, None, Y, n_epochs, epoch0, n_run, a, b, alpha0, n_neg,
                                    7, ws, ws_bytes, None, None)

    assert call(graph=None) == -1
    assert call(Y=None) == -1
    assert call(n_epochs=0) == -1
    assert call(n_epochs=1 << 24) == -1
    assert call(epoch0=-1) == -1
    assert call(n_run=-1) == -1
    assert call(epoch0=150, n_run=51) == -1
    assert call(a=0.0) == -1
    assert call(b=float("nan")) == -1
    assert call(alpha0=-1.0) == -1
    assert call(n_neg=16) == -1
    assert call(n_neg=-1) == -1
    assert call(ws_bytes=16) == -6  # workspace smaller than n positions
    assert call(ws=ctypes.c_void_p((1 << 40) + 8)) == -6
    assert call(n_run=0) == 0  # nothing to do: no launch
    assert lib.tsne_workspace_size(L.TSNE_OP_UMAP_LAYOUT, 1000, 0, 0, None, None) == 8192
    assert lib.tsne_workspace_size(L.TSNE_OP_UMAP_LAYOUT, 0, 0, 0, None, None) == 0


def test_umap_ab_matches_the_oracle_fit():
    """The library's (a, b) fit (tsne_umap_ab: FP64 Levenberg-Marquardt in C on
    the host) against the oracle's (scipy's curve_fit) on the same least-squares
    problem."""
    import numpy as np

    from oracle import umap_layout as U
    from paper_2605_13928_b300 import api
    for md, sp in ((0.1, 1.0), (0.5, 1.0), (0.0, 2.0), (0.25, 0.5)):
        np.testing.assert_allclose(api.umap_ab(md, sp), U.fit_ab(md, sp), rtol=1e-5)


def test_umap_ab_and_init_host_argument_errors(lib):
    a, b = ctypes.c_double(0.0), ctypes.c_double(0.0)
    assert lib.tsne_umap_ab(0.1, 0.0, ctypes.byref(a), ctypes.byref(b)) == -1
    assert lib.tsne_umap_ab(-0.1, 1.0, ctypes.byref(a), ctypes.byref(b)) == -1
    assert lib.tsne_umap_ab(float("nan"), 1.0, ctypes.byref(a), ctypes.byref(b)) == -1
    assert lib.tsne_umap_ab(0.1, 1.0, None, ctypes.byref(b)) == -1
    fake = ctypes.c_void_p(1 << 40)  # never dereferenced: the checks come first
    need = lib.tsne_workspace_size(L.TSNE_OP_UMAP_INIT, 1000, 0, 0, None, None)
    assert need > 0 and lib.tsne_workspace_size(L.TSNE_OP_UMAP_INIT, 0, 0, 0, None, None) == 0
    assert lib.tsne_umap_init(fake, 1000, 1, fake, fake, need, None, None) == -1  # ld < 2
    assert lib.tsne_umap_init(None, 1000, 50, fake, fake, need, None, None) == -1
    assert lib.tsne_umap_init(fake, 1000, 50, fake, fake, 16, None, None) == -6
    assert lib.tsne_umap_init(fake, 0, 50, fake, fake, need, None, None) == 0  # nothing to do


def test_pca_host_argument_errors(lib):
    fake = ctypes.c_void_p(1 << 40)  # never dereferenced: every call below fails its checks
    P = fake
    # n too small, g too small, k out of range, lda < g, missing pointers, no workspace
    assert lib.tsne_pca(P, 64, 64, 64, 10, 2, P, P, P, None, None, None, P, P, 1 << 30, None,
                        None) == -1
    assert lib.tsne_pca(P, 100, 63, 63, 10, 2, P, P, P, None, None, None, P, P, 1 << 30, None,
                        None) == -1
    assert lib.tsne_pca(P, 100, 64, 64, 65, 2, P, P, P, None, None, None, P, P, 1 << 30, None,
                        None) == -1
    assert lib.tsne_pca(P, 100, 64, 32, 10, 2, P, P, P, None, None, None, P, P, 1 << 30, None,
                        None) == -1
    assert lib.tsne_pca(P, 100, 64, 64, 10, 2, None, P, P, None, None, None, P, P, 1 << 30, None,
                        None) == -1
    assert lib.tsne_pca(P, 100, 64, 64, 10, 2, P, P, P, None, None, None, P, None, 0, None,
                        None) == -6
    assert lib.tsne_pca_transform(P, 0, 64, 64, P, P, 10, P, P, 1 << 30, None, None) == -1
    assert lib.tsne_pca_transform(P, 10, 64, 64, P, P, 65, P, P, 1 << 30, None, None) == -1
    assert lib.tsne_pca_transform(P, 10, 64, 64, None, P, 5, P, P, 1 << 30, None, None) == -1
    # A misaligned for TMA (row stride not a multiple of 4 floats)
    assert lib.tsne_pca(P, 100, 66, 66, 10, 2, P, P, P, None, None, None, P, P, 1 << 30, None,
                        None) == -1
    # workspace: sketches and partial products only (A is read in place)
    need = lib.tsne_workspace_size(L.TSNE_OP_PCA, 100000, 2000, 0, None, None)
    big = lib.tsne_workspace_size(L.TSNE_OP_PCA, 1000000, 2000, 0, None, None)
    assert 0 < need < big < (1 << 30)
    assert lib.tsne_workspace_size(L.TSNE_OP_PCA, 64, 2000, 0, None, None) == 0
    assert 0 < lib.tsne_workspace_size(L.TSNE_OP_PCA_TRANSFORM, 1000, 300, 0, None, None)
