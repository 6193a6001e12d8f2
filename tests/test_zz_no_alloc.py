"""tsne_kl_grad_noalloc, the allocation-free gradient entry point.

It serves callers that cannot allocate device memory: an application whose
own allocator owns all device memory, or a loop that cannot afford
cudaMalloc's implicit synchronisation.  Its scratch is a fixed array inside
the library, shared by every call and keeping the previous call's contents.
This test calls it through the C ABI twice in a row, on different inputs, and
compares each result with the workspace entry point tsne_kl_grad under the
tolerances of the other gradient tests (1e-4 relative L2 for the gradient,
1e-6 for Z and KL), the same at the size limit (the fullest scratch layout)
through the Python wrapper with no KL output, and checks that a size beyond
the array's limit is refused.  The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2605_13928_b300 import _lib as L
from paper_2605_13928_b300 import api
from problems import embedding, grad_err, mixture_P

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_workspace_entry_point_twice(gpu):
    lib = L.lib()
    cases = [(3001, 5.0, 12.0, 0), (1500, 0.5, 1.0, 1)]  # second call: smaller, new inputs
    for n, scale, alpha, seed in cases:
        X, P = mixture_P(n, seed=seed)
        Pd = api.CSR.from_numpy(P.row_ptr, P.col, P.val, gpu)
        Y = torch.tensor(embedding(n, scale, seed=40 + seed), device=gpu)
        g0, Z0, kl0 = api.kl_grad(Pd, Y, alpha, want_kl=True)
        g1 = torch.empty_like(Y)
        Z1 = torch.empty(1, dtype=torch.float64, device=gpu)
        kl1 = torch.empty(1, dtype=torch.float64, device=gpu)
        stream = ctypes.c_void_p(torch.cuda.current_stream(gpu).cuda_stream)
        rc = lib.tsne_kl_grad_noalloc(Pd.c(), _p(Y), float(alpha), _p(g1), _p(Z1), _p(kl1), None,
                                      stream)
        assert rc == 0
        torch.cuda.synchronize()
        a, b = g1.cpu().numpy(), g0.cpu().numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-4
        assert grad_err(a, P, Y.cpu().numpy(), alpha) < 1e-4
        assert abs(Z1.item() / Z0.item() - 1) < 1e-6
        assert abs(kl1.item() - kl0.item()) < 1e-6 * max(1.0, abs(kl0.item()))


def test_noalloc_at_its_size_limit_through_the_binding(gpu):
    """n = TSNE_NOALLOC_MAX_N, where the scratch layout is fullest (four column
    chunks of partial forces, about 5.5 of the 6 MiB), called through the Python
    wrapper without the KL value (kl = NULL), twice in a row on different
    embeddings, each against tsne_kl_grad under the same tolerances."""
    n = L.TSNE_NOALLOC_MAX_N
    X, P = mixture_P(n, k=12, perplexity=4.0, seed=2)
    Pd = api.CSR.from_numpy(P.row_ptr, P.col, P.val, gpu)
    for scale, alpha, seed in ((0.01, 12.0, 50), (20.0, 1.0, 51)):
        Y = torch.tensor(embedding(n, scale, seed=seed), device=gpu)
        g0, Z0, _ = api.kl_grad(Pd, Y, alpha)
        g1, Z1, kl1 = api.kl_grad_noalloc(Pd, Y, alpha)
        torch.cuda.synchronize()
        assert kl1 is None
        a, b = g1.cpu().numpy(), g0.cpu().numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-4
        assert abs(Z1.item() / Z0.item() - 1) < 1e-6


def test_noalloc_rejects_sizes_beyond_its_limit(gpu):
    n = L.TSNE_NOALLOC_MAX_N + 1
    fake = ctypes.c_void_p(1 << 40)  # never dereferenced: the size check comes first
    csr = L.TsneCsr(n, 0, 0, fake, fake, fake)
    rc = L.lib().tsne_kl_grad_noalloc(ctypes.byref(csr), fake, 1.0, None, fake, None, None, None)
    assert rc == -2  # TSNE_ERR_CAPACITY
