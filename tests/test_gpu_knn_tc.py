"""GPU parity of the BF16 tensor-core kNN (tcgen05 distance GEMM, candidate
filter, exact FP32 re-rank of cand_mult * k candidates).

Once the true k nearest are among the candidates, the re-rank uses the FP32
brute-force kernel's operation order, so its output is bit-identical to the
FP32 path; where the BF16 distances drop a true neighbour from the candidate
set the row differs.  The tests require:
* neighbour sets equal to the FP64 oracle's modulo ties within 1e-6 relative,
  on every row, for the mixture workloads at cand_mult = 2 (recall 1);
* bit-identical output to the FP32 path on those rows;
* integer inputs (exact BF16 and FP32 distances) bit-exact against the oracle.
The candidate recall on the knn_n200k workload (5,000-row subsample against
the oracle) is checked to be 1 as well.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_13928_b300 import _lib as L
from paper_2605_13928_b300 import api, synth
from test_gpu_knn_affinity import _check_knn

pytestmark = pytest.mark.gpu

BF16 = L.TSNE_KNN_BF16_RERANK


@pytest.mark.parametrize("n,d,k", [(91, 50, 90), (2000, 50, 90), (1500, 3, 30), (700, 17, 12),
                                   (1030, 64, 90), (5000, 50, 90)])
def test_bf16_knn_matches_oracle_and_fp32_path(gpu, n, d, k):
    X = synth.mixture(n, 8, d=d, seed=synth.SEED_BASE + n + d)
    Xd = torch.tensor(X, device=gpu)
    st = api.new_status(gpu)
    idx, d2 = api.knn(Xd, k, mode=BF16, status=st)
    idx32, d232 = api.knn(Xd, k)
    torch.cuda.synchronize()
    assert st.item() == 0
    _check_knn(X, idx.cpu().numpy(), d2.cpu().numpy(), k, name=f"knn_bf16/n{n}/d{d}/k{k}")
    assert torch.equal(idx, idx32) and torch.equal(d2, d232)


def test_bf16_knn_integer_grid_bit_exact(gpu):
    g = np.array([[a, b, c] for a in range(6) for b in range(6) for c in range(4)], np.float32)
    X = np.concatenate([g, g[::7]])
    k = 20
    idx, d2 = api.knn(torch.tensor(X, device=gpu), k, mode=BF16)
    idx_r, d2_r = oracle.knn(X.astype(np.float64), k)
    assert np.array_equal(idx.cpu().numpy(), idx_r)
    assert np.array_equal(d2.cpu().numpy().astype(np.float64), d2_r)


def test_bf16_knn_batched(gpu):
    sizes = [100, 91, 3000, 333, 129]
    Xs = [synth.mixture(s, 5, d=50, seed=synth.SEED_BASE + 150 + i) for i, s in enumerate(sizes)]
    X = np.concatenate(Xs)
    batch = api.Batch(sizes)
    Xd = torch.tensor(X, device=gpu)
    idx, d2 = api.knn(Xd, 90, batch=batch, mode=BF16)
    idx32, d232 = api.knn(Xd, 90, batch=batch)
    assert torch.equal(idx, idx32) and torch.equal(d2, d232)
    idx = idx.cpu().numpy()
    for s in range(len(sizes)):
        a, b = batch.pt_off[s], batch.pt_off[s + 1]
        assert idx[a:b].min() >= a and idx[a:b].max() < b


def test_bf16_knn_recall_knn_n200k_subsample(gpu):
    wl = synth.WORKLOADS["knn_n200k"]
    X = wl.data()
    idx, d2 = api.knn(torch.tensor(X, device=gpu), wl.k, mode=BF16)
    rows = np.sort(np.random.default_rng(5).choice(wl.n, 5000, replace=False))
    _check_knn(X, idx.cpu().numpy(), d2.cpu().numpy(), wl.k, rows=rows,
               name="knn_bf16/knn_n200k/5000_rows")


@pytest.mark.parametrize("d", [50, 64])  # folded (d <= 61) and unfolded candidate filter
def test_bf16_knn_prunes_under_concentration_and_ties(gpu, d):
    """Inputs that stress the candidate prunes: one isotropic Gaussian, whose
    distances pile up near each row's threshold (every row prunes several times
    and the early-exit radix passes must narrow a crowded bin), and 50 positions
    repeated 60 times, whose buffers hold long runs of equal keys (the passes
    cannot split them and the prune falls back to the exact select)."""
    rng = np.random.default_rng(77 + d)
    A = rng.normal(size=(6000, d)).astype(np.float32)
    B = np.repeat(rng.normal(size=(50, d)).astype(np.float32) * 3.0, 60, axis=0)
    for X, same_as_fp32 in ((A, True), (B, False)):
        Xd = torch.tensor(X, device=gpu)
        st = api.new_status(gpu)
        idx, d2 = api.knn(Xd, 90, mode=BF16, status=st)
        torch.cuda.synchronize()
        assert st.item() == 0
        _check_knn(X, idx.cpu().numpy(), d2.cpu().numpy(), 90)
        if same_as_fp32:  # no ties: the FP32 path's output, bit for bit
            idx32, d232 = api.knn(Xd, 90)
            assert torch.equal(idx, idx32) and torch.equal(d2, d232)
