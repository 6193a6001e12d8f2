"""GPU parity of the PCA path (tsne_pca, tsne_pca_transform) against the FP64
oracle (oracle/pca.py).

Error budget.  Every product with A runs on the tensor cores with both
operands split into BF16 hi + lo (each value kept to ~2^-17 relative) and
FP32 accumulation: a product x.v carries an error of at most ~3 * 2^-18
|x||v| per term plus the FP32 accumulation, so
* transform: |T - T_ref| <= 4e-5 (|Ac| |V|^T) elementwise (K <= 400 terms);
* fit: the sketch products perturb B = Q^T Ac by eps ||Ac|| with eps ~ 3e-5,
  so singular values move by at most eps sigma_1 and an axis c turns by at
  most eps sigma_1 / gap_c (Wedin), gap_c its distance to the neighbouring
  singular values.  Axes are compared one by one where that bound is below
  0.02 and through the projector onto the top-k subspace otherwise.
The randomized iteration adds (sigma_65 / sigma_k)^(2q+1) to the subspace
error; the inputs below have a gap that makes it negligible.
"""
import numpy as np
import pytest
import torch

from oracle import pca as O
from paper_2605_13928_b300 import _lib as L
from paper_2605_13928_b300 import api, synth

pytestmark = pytest.mark.gpu

EPS = 3e-5


def _gpu_pca(A, k, n_power=2, seed=1, gpu=None):
    Ad = torch.tensor(A, device=gpu)
    st = api.new_status(gpu)
    out = api.pca(Ad, k, n_power=n_power, seed=seed, status=st)
    torch.cuda.synchronize()
    res = {key: v.cpu().numpy().astype(np.float64) for key, v in out.items()}
    res["status"] = int(st.item())
    return res


def _check_fit(A, k, got, ref, eps=EPS):
    assert got["status"] == 0
    s_ref = ref["sigma"]
    s1 = s_ref[0]
    np.testing.assert_allclose(got["mean"], ref["mean"], atol=1e-6 * max(1.0, np.abs(A).max()))
    np.testing.assert_allclose(got["total_var"][0], ref["total_var"], rtol=1e-5)
    assert np.all(np.abs(got["sigma"] - s_ref) <= 2 * eps * s1 + 1e-9)
    np.testing.assert_allclose(got["explained_variance"], got["sigma"] ** 2 / (A.shape[0] - 1),
                               rtol=1e-12)
    V, Vr = got["components"], ref["components"]
    # orthonormal axes, sign convention, subspace
    np.testing.assert_allclose(V @ V.T, np.eye(k), atol=1e-4)
    for row in V:
        assert row[np.argmax(np.abs(row))] > 0
    P, Pr = V.T @ V, Vr.T @ Vr
    full = O.pca(A, min(k + 1, min(A.shape)))
    gap_k = full["sigma"][k - 1] - full["sigma"][k] if k < len(full["sigma"]) else s1
    assert np.abs(P - Pr).max() <= max(4 * eps * s1 / gap_k, 1e-4)
    # axis by axis where the perturbation bound is small
    sig = full["sigma"]
    checked = 0
    for c in range(k):
        lo = sig[c - 1] - sig[c] if c > 0 else np.inf
        hi = sig[c] - sig[c + 1] if c + 1 < len(sig) else np.inf
        bound = 4 * eps * s1 / min(lo, hi)
        if bound > 0.02:
            continue
        cosang = abs(V[c] @ Vr[c])
        assert cosang >= 1 - bound ** 2 - 1e-6, (c, cosang, bound)
        sgn = np.sign(V[c] @ Vr[c])
        tref = ref["scores"][:, c]
        err = np.linalg.norm(got["scores"][:, c] - sgn * tref) / np.linalg.norm(tref)
        assert err <= 2 * bound + 2 * eps * s1 / sig[c], (c, err)
        checked += 1
    return checked


def test_transform_matches_oracle_ragged_tiles(gpu):
    rng = np.random.default_rng(7)
    n, g, k = 1000, 300, 50  # 8 row tiles (last one 104 rows), 5 K blocks (last ragged)
    A = (rng.normal(size=(n, g)) * 2 + rng.normal(size=g) * 5).astype(np.float32)
    mean = A.astype(np.float64).mean(axis=0) + rng.normal(size=g) * 0.1
    comp = rng.normal(size=(k, g)).astype(np.float32)
    T = api.pca_transform(torch.tensor(A, device=gpu), torch.tensor(mean, device=gpu),
                          torch.tensor(comp, device=gpu)).cpu().numpy().astype(np.float64)
    Tr = O.transform(A, mean, comp)
    Ac = np.abs(A.astype(np.float64) - mean[None, :])
    bound = 4e-5 * (Ac @ np.abs(comp.astype(np.float64)).T) + 1e-6
    assert np.all(np.abs(T - Tr) <= bound)


@pytest.mark.parametrize("k", [1, 7, 16])
def test_transform_few_components(gpu, k):
    rng = np.random.default_rng(k)
    n, g = 257, 129
    A = rng.normal(size=(n, g)).astype(np.float32)
    mean = rng.normal(size=g)
    comp = rng.normal(size=(k, g)).astype(np.float32)
    T = api.pca_transform(torch.tensor(A, device=gpu), torch.tensor(mean, device=gpu),
                          torch.tensor(comp, device=gpu)).cpu().numpy().astype(np.float64)
    Tr = O.transform(A, mean, comp)
    Ac = np.abs(A.astype(np.float64) - mean[None, :])
    assert np.all(np.abs(T - Tr) <= 4e-5 * (Ac @ np.abs(comp.astype(np.float64)).T) + 1e-6)


def test_fit_known_spectrum_exact_rank(gpu):
    """A = U S V^T + 1 m^T of rank 64 = the sketch width: the sketch spans the
    whole range, so the result is exact up to arithmetic."""
    rng = np.random.default_rng(3)
    n, g, r, k = 5000, 256, 64, 50
    U, _ = np.linalg.qr(rng.normal(size=(n, r)) - 0.0)
    U -= U.mean(axis=0)
    U, _ = np.linalg.qr(U)
    V, _ = np.linalg.qr(rng.normal(size=(g, r)))
    S = 300.0 * 0.93 ** np.arange(r)
    m = rng.normal(size=g)
    A = (U @ np.diag(S) @ V.T + m).astype(np.float32)
    got = _gpu_pca(A, k, gpu=gpu)
    ref = O.pca(A, k)
    # axes 35..50 have gaps below the per-axis bound's reach (sigma ratio 0.93)
    assert _check_fit(A, k, got, ref) >= 30


def test_fit_mixture_workload_recipe(gpu):
    A = synth.pca_matrix(3000, 300, seed=synth.SEED_BASE + 50)
    k = 50
    got = _gpu_pca(A, k, gpu=gpu)
    ref = O.pca(A, k)
    checked = _check_fit(A, k, got, ref)
    assert checked >= 20


def test_fit_rank_deficient_top_axes(gpu):
    """Rank 20 < 64: the sketch is rank deficient; shifted CholeskyQR keeps
    the top axes right."""
    rng = np.random.default_rng(4)
    n, g, r, k = 2000, 200, 20, 10
    A = (rng.normal(size=(n, r)) * (2.0 ** -np.arange(r) * 30)) @ rng.normal(size=(r, g))
    A = (A + rng.normal(size=g)).astype(np.float32)
    got = _gpu_pca(A, k, gpu=gpu)
    ref = O.pca(A, k)
    assert _check_fit(A, k, got, ref) >= 6  # the last axes (sigma ~ 10) sit below the bound


@pytest.mark.parametrize("n,g,k", [(65, 64, 1), (65, 64, 64), (130, 70, 5)])
def test_fit_smallest_shapes(gpu, n, g, k):
    rng = np.random.default_rng(n + g + k)
    A = (rng.normal(size=(n, g)) * np.linspace(3, 0.5, g)).astype(np.float32)
    got = _gpu_pca(A, k, n_power=3, gpu=gpu)
    ref = O.pca(A, k)
    assert got["status"] == 0
    # a 64-column sketch of a <= 65-row matrix spans its whole row space
    np.testing.assert_allclose(got["sigma"], ref["sigma"], rtol=2e-4, atol=2e-4 * ref["sigma"][0])


def test_fit_is_deterministic(gpu):
    A = synth.pca_matrix(2000, 200, seed=synth.SEED_BASE + 51)
    Ad = torch.tensor(A, device=gpu)
    a = api.pca(Ad, 30, seed=2)
    b = api.pca(Ad, 30, seed=2)
    for key in a:
        assert torch.equal(a[key], b[key]), key


def test_fit_then_transform_reproduces_scores(gpu):
    A = synth.pca_matrix(1500, 256, seed=synth.SEED_BASE + 52)
    Ad = torch.tensor(A, device=gpu)
    out = api.pca(Ad, 40)
    T2 = api.pca_transform(Ad, out["mean"], out["components"])
    T1 = out["scores"]
    rel = (T2 - T1).norm() / T1.norm()
    assert rel.item() < 1e-4


def test_pca_argument_errors(gpu):
    A = torch.zeros((64, 64), device=gpu)
    with pytest.raises(L.TsneError):
        api.pca(A, 10)  # n < 65
    A = torch.zeros((100, 63), device=gpu)
    with pytest.raises(L.TsneError):
        api.pca(A, 10)  # g < 64
    A = torch.zeros((100, 100), device=gpu)
    with pytest.raises(L.TsneError):
        api.pca(A, 65)  # k > 64


def test_fit_on_a_strided_view_equals_the_contiguous_fit(gpu):
    """A read in place with a row stride lda > g (a column slice of a wider
    matrix) gives bit-identical results to the contiguous copy."""
    A = synth.pca_matrix(1000, 200, seed=synth.SEED_BASE + 53)
    wide = torch.zeros((1000, 256), device=gpu)
    wide[:, :200] = torch.tensor(A, device=gpu)
    view = wide[:, :200]
    assert view.stride(0) == 256
    a = api.pca(view, 20, seed=4)
    b = api.pca(torch.tensor(A, device=gpu), 20, seed=4)
    for key in a:
        assert torch.equal(a[key], b[key]), key


def test_fit_without_power_iterations(gpu):
    """n_power = 0 (one pass of the range finder): with a gap after sigma_k the
    sketch already captures the top axes; sigma within the loose bound."""
    A = synth.pca_matrix(2000, 256, seed=synth.SEED_BASE + 54, noise=0.001)
    got = _gpu_pca(A, 20, n_power=0, gpu=gpu)
    ref = O.pca(A, 20)
    assert got["status"] == 0
    assert np.all(np.abs(got["sigma"] - ref["sigma"]) <= 1e-3 * ref["sigma"][0])


def test_wide_matrix_uses_several_k_segments(gpu):
    """g = 2600 > 2048: the rows product accumulates in two K segments summed in
    FP64; transform and fit stay within the same bounds."""
    rng = np.random.default_rng(8)
    n, g, k = 700, 2600, 12
    A = (rng.normal(size=(n, g)) + rng.normal(size=g)).astype(np.float32)
    mean = A.astype(np.float64).mean(axis=0)
    comp = rng.normal(size=(k, g)).astype(np.float32)
    T = api.pca_transform(torch.tensor(A, device=gpu), torch.tensor(mean, device=gpu),
                          torch.tensor(comp, device=gpu)).cpu().numpy().astype(np.float64)
    Tr = O.transform(A, mean, comp)
    Ac = np.abs(A.astype(np.float64) - mean[None, :])
    assert np.all(np.abs(T - Tr) <= 4e-5 * (Ac @ np.abs(comp.astype(np.float64)).T) + 1e-6)
    B = synth.pca_matrix(1500, 2100, seed=synth.SEED_BASE + 55)
    got = _gpu_pca(B, 30, gpu=gpu)
    ref = O.pca(B, 30)
    assert _check_fit(B, 30, got, ref) >= 10


def test_no_accumulation_drift_on_positive_data(gpu):
    """All-positive data and axes: every product and partial sum is positive,
    so a drift of the tensor cores' FP32 accumulation would show as a
    systematic underestimate; with K segments of 2048 summed in FP64 the mean
    relative error stays below 1e-5 at K = 8192."""
    rng = np.random.default_rng(9)
    n, g = 2048, 8192
    A = rng.uniform(0.5, 1.5, size=(n, g)).astype(np.float32)
    V = rng.uniform(0.5, 1.5, size=(64, g)).astype(np.float32)
    T = api.pca_transform(torch.tensor(A, device=gpu), torch.zeros(g, dtype=torch.float64,
                                                                   device=gpu),
                          torch.tensor(V, device=gpu)).cpu().numpy().astype(np.float64)
    ref = A.astype(np.float64) @ V.astype(np.float64).T
    rel = (T - ref) / ref
    assert abs(rel.mean()) < 1e-5 and np.abs(rel).max() < 1e-4
