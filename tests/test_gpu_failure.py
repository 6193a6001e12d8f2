"""Failure detection on the GPU without a fault: bounded device waits that run
out report TSNE_STATUS_TIMEOUT and the context stays usable; checkpoints
resume bitwise identically."""
import numpy as np
import pytest
import torch

from paper_2605_13928_b300 import _lib as L
from paper_2605_13928_b300 import api, checkpoint
from problems import block_diag, embedding, mixture_P

pytestmark = pytest.mark.gpu


def _batch(gpu):
    sizes = [30000, 600, 700, 500, 900]
    Ps = [mixture_P(n, seed=40 + i, k=15, perplexity=5.0)[1] for i, n in enumerate(sizes)]
    Pb = block_diag(Ps)
    return api.CSR.from_numpy(Pb.row_ptr, Pb.col, Pb.val, gpu), api.Batch(sizes)


def test_wait_limit_runs_out_and_is_reported(gpu, monkeypatch):
    Pd, batch = _batch(gpu)
    n = batch.n
    prm = L.default_params(variant=L.TSNE_VARIANT_FUSED, kl_every=0)
    Y0 = torch.tensor(embedding(n, 1.0, seed=3), device=gpu)
    # update slots of the fused launch wait for their sample; with a one-cycle
    # limit the slots of the 30,000-point sample give up before it completes
    monkeypatch.setenv("TSNE_WAIT_LIMIT", "1")
    st = api.new_status(gpu)
    Y, U, G = Y0.clone(), torch.zeros_like(Y0), torch.ones_like(Y0)
    api.step(Pd, Y, U, G, 0, prm, batch=batch, status=st)
    torch.cuda.synchronize()
    assert st.item() & L.TSNE_STATUS_TIMEOUT
    # the context is still usable and a normal limit completes cleanly
    monkeypatch.delenv("TSNE_WAIT_LIMIT")
    st2 = api.new_status(gpu)
    Y, U, G = Y0.clone(), torch.zeros_like(Y0), torch.ones_like(Y0)
    api.step(Pd, Y, U, G, 0, prm, batch=batch, status=st2)
    torch.cuda.synchronize()
    assert st2.item() == 0 and torch.isfinite(Y).all() and not torch.equal(Y, Y0)


def test_knn_wait_limit_runs_out_and_is_reported(gpu, monkeypatch):
    """The tcgen05 kNN's pipeline waits (TMA producer, MMA issuer, epilogue)
    with a one-cycle limit give up: TSNE_STATUS_TIMEOUT is set; the producer
    still waits, on its own long bound, for the copies it has issued and the MMA
    issuer for its committed MMAs before tensor memory is freed and the CTA
    exits.  The context stays usable: the next call with the default limit is
    clean and bit-identical to the FP32 brute-force path."""
    from paper_2605_13928_b300 import synth
    n, k = 5000, 90
    X = synth.mixture(n, 8, d=50, seed=synth.SEED_BASE + n + 50)
    Xd = torch.tensor(X, device=gpu)
    monkeypatch.setenv("TSNE_WAIT_LIMIT", "1")
    st = api.new_status(gpu)
    api.knn(Xd, k, mode=L.TSNE_KNN_BF16_RERANK, status=st)
    torch.cuda.synchronize()
    assert st.item() & L.TSNE_STATUS_TIMEOUT
    monkeypatch.delenv("TSNE_WAIT_LIMIT")
    st2 = api.new_status(gpu)
    idx, d2 = api.knn(Xd, k, mode=L.TSNE_KNN_BF16_RERANK, status=st2)
    idx32, d232 = api.knn(Xd, k)
    torch.cuda.synchronize()
    assert st2.item() == 0
    assert torch.equal(idx, idx32) and torch.equal(d2, d232)


def test_checkpoint_resume_is_bitwise(gpu, tmp_path):
    X, P = mixture_P(3000)
    Pd = api.CSR.from_numpy(P.row_ptr, P.col, P.val, gpu)
    prm = L.default_params(ee_iters=4, mom_switch=4, kl_every=0, n_iter=10)
    Y0 = torch.tensor(embedding(3000, 1e-2, seed=1), device=gpu)
    Y, U, G = Y0.clone(), torch.zeros_like(Y0), torch.ones_like(Y0)
    for it in range(10):
        api.step(Pd, Y, U, G, it, prm)
    Yb, Ub, Gb = Y0.clone(), torch.zeros_like(Y0), torch.ones_like(Y0)
    for it in range(6):
        api.step(Pd, Yb, Ub, Gb, it, prm)
    path = str(tmp_path / "ck.npz")
    checkpoint.save(path, Yb, Ub, Gb, 6, prm)
    st = checkpoint.load(path, gpu)
    for it in range(st.iteration, 10):
        api.step(Pd, st.Y, st.U, st.G, it, st.params)
    assert torch.equal(st.Y, Y) and torch.equal(st.U, U) and torch.equal(st.G, G)
