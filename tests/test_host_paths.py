"""Host-side error paths and state handling, on CPU: fault injection through
the C ABI (no kernel runs) and checkpoint round trips."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2605_13928_b300 import _lib as L
from paper_2605_13928_b300 import build as B
from paper_2605_13928_b300 import checkpoint


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.lib()


def test_fault_injection_returns_the_named_code(lib, monkeypatch):
    fake = ctypes.c_void_p(1 << 40)  # never dereferenced: the injected code returns first
    csr = L.TsneCsr(10, 0, 20, fake, fake, fake)
    monkeypatch.setenv("TSNE_FAULT", "tsne_step:-1,tsne_kl_grad:-3")
    assert lib.tsne_kl_grad(ctypes.byref(csr), None, fake, 1.0, None, fake, None, None, fake,
                            1 << 30, None, None) == -3
    p = L.default_params()
    assert lib.tsne_step(ctypes.byref(csr), None, fake, fake, fake, 0, ctypes.byref(p), None, None,
                         fake, 1 << 30, None, None) == -1
    monkeypatch.setenv("TSNE_FAULT", "tsne_knn:-4")
    assert lib.tsne_knn(fake, 100, 5, 3, None, 0, 2.0, fake, fake, None, 0, None, None) == -4
    monkeypatch.setenv("TSNE_FAULT", "tsne_run:-7")
    assert lib.tsne_run(fake, 100, 5, None, ctypes.byref(p), fake, None, None, None) == -7
    with pytest.raises(L.TsneError) as err:
        L.check(-4, "tsne_knn")
    assert err.value.code == -4 and "TIMEOUT" in str(err.value)


def test_checkpoint_round_trip(tmp_path):
    rng = np.random.default_rng(0)
    Y, U, G = (torch.tensor(rng.normal(size=(50, 2)).astype(np.float32)) for _ in range(3))
    prm = L.default_params(n_iter=321, ee=8.0, kl_every=7, variant=L.TSNE_VARIANT_SYM4)
    path = str(tmp_path / "state.npz")
    checkpoint.save(path, Y, U, G, 123, prm)
    st = checkpoint.load(path)
    assert torch.equal(st.Y, Y) and torch.equal(st.U, U) and torch.equal(st.G, G)
    assert st.iteration == 123
    for name, _ in L.TsneParams._fields_:
        assert getattr(st.params, name) == getattr(prm, name), name


def test_neighbour_csr_shape():
    """The host generator of kNN-shaped P matrices (used by the 1M gradient test
    and the bench's oracle timings): k ascending columns per row, none on the
    diagonal, all within the window and inside [0, n), positive values summing
    to 1, reproducible from the seed."""
    from paper_2605_13928_b300 import synth
    n, k, win = 5000, 30, 200
    rp, col, val = synth.neighbour_csr(n, k, win, seed=3)
    assert rp.dtype == np.int64 and col.dtype == np.int32 and val.dtype == np.float32
    assert np.array_equal(rp, np.arange(n + 1) * k)
    c = col.reshape(n, k).astype(np.int64)
    i = np.arange(n)[:, None]
    assert (np.diff(c, axis=1) >= 0).all()
    assert (c != i).all() and (np.abs(c - i) <= win).all()
    assert c.min() >= 0 and c.max() < n
    assert (val > 0).all() and abs(float(val.astype(np.float64).sum()) - 1.0) < 1e-5
    rp2, col2, val2 = synth.neighbour_csr(n, k, win, seed=3)
    assert np.array_equal(col, col2) and np.array_equal(val, val2)
