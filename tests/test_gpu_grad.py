"""GPU parity of the exact KL gradient path against the FP64 oracle.

Tolerances: the gradient must match the oracle to 1e-4 relative L2 (per
sample; relative to the attraction / repulsion term norms where those cancel,
see problems.grad_err) and, row by row, to 3e-4 of the row's own scale
4 (alpha Aa_i + Ar_i / Z) (problems.ROW_TOL: a worst-case FP32 summation bound,
so that a few wrong rows cannot hide under the norm of thousands); Z to 1e-6
relative; KL to 1e-6 absolute.  The FP32 kernels
accumulate per shared-memory tile in FP32 and across tiles in FP64, so the
error budget is dominated by FP32 rounding of the per-pair terms (~1e-7
relative each) and of the approximate reciprocal (~1 ulp).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_13928_b300 import _lib as L
from paper_2605_13928_b300 import api
from problems import (ROW_TOL, block_diag, embedding, grad_err, mixture_P, record, rel_l2,
                      row_err, row_err_scaled)

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-4


def _dev_csr(P, dev):
    return api.CSR.from_numpy(P.row_ptr, P.col, P.val, dev)


def _oracle_grad(P, Y, alpha):
    # the oracle takes the FP32 positions exactly as the GPU sees them
    return oracle.grad(P, Y.astype(np.float64), alpha)


# TSNE_VARIANT_DIRECT: the tile shape AUTO picks by problem size, with the
# small-problem forces launch (attraction rows and direct items in one kernel)
VARIANTS = [L.TSNE_VARIANT_DIRECT, L.TSNE_VARIANT_DIRECT_S, L.TSNE_VARIANT_DIRECT_L,
            L.TSNE_VARIANT_SYM, L.TSNE_VARIANT_DIRECT_M, L.TSNE_VARIANT_SYM4,
            L.TSNE_VARIANT_SYM4_FX]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("n", [2, 3, 31, 257, 1000, 2049, 4096, 6001])
@pytest.mark.parametrize("scale", [1e-2, 1.0, 30.0])
def test_grad_matches_oracle(gpu, n, scale, variant):
    X, P = mixture_P(n)
    Y = embedding(n, scale, seed=n)
    prm = L.default_params(variant=variant)
    for alpha in (1.0, 12.0):
        g, Z, kl = api.kl_grad(_dev_csr(P, gpu), torch.tensor(Y, device=gpu), alpha, params=prm,
                               want_kl=True)
        g_ref, Z_ref = _oracle_grad(P, Y, alpha)
        ge, re = grad_err(g.cpu().numpy(), P, Y, alpha), row_err(g.cpu().numpy(), P, Y, alpha)
        kl_ref = oracle.kl(P, Y.astype(np.float64), alpha, Z_ref)
        record(f"grad/variant{variant}/n{n}/scale{scale}/alpha{alpha}", grad_rel_l2=ge,
               grad_max_row=re, Z_rel=abs(Z.item() / Z_ref - 1), kl_abs=abs(kl.item() - kl_ref),
               kl_scaled=abs(kl.item() - kl_ref) / max(1.0, abs(kl_ref)))
        assert ge < GRAD_TOL
        assert re < ROW_TOL
        assert abs(Z.item() / Z_ref - 1) < 1e-6
        assert abs(kl.item() - kl_ref) < 1e-6 * max(1.0, abs(kl_ref))


@pytest.mark.parametrize("n", [6500, 9000, 15000])
def test_auto_mid_sizes_match_oracle(gpu, n):
    """AUTO between 4e7 and 4e8 pairs (256-row items with 256-column tiles, in the
    small-problem forces launch) and at 15,000 points, just below the symmetric
    split, against the oracle's gradient, Z and KL."""
    X, P = mixture_P(n, seed=n)
    Y = embedding(n, 5.0, seed=n + 3)
    for alpha in (1.0, 12.0):
        g, Z, kl = api.kl_grad(_dev_csr(P, gpu), torch.tensor(Y, device=gpu), alpha,
                               params=L.default_params(), want_kl=True)
        g_ref, Z_ref = _oracle_grad(P, Y, alpha)
        ge, re = grad_err(g.cpu().numpy(), P, Y, alpha), row_err(g.cpu().numpy(), P, Y, alpha)
        kl_ref = oracle.kl(P, Y.astype(np.float64), alpha, Z_ref)
        record(f"grad_auto/n{n}/alpha{alpha}", grad_rel_l2=ge, grad_max_row=re,
               Z_rel=abs(Z.item() / Z_ref - 1), kl_abs=abs(kl.item() - kl_ref))
        assert ge < GRAD_TOL
        assert re < ROW_TOL
        assert abs(Z.item() / Z_ref - 1) < 1e-6
        assert abs(kl.item() - kl_ref) < 1e-6 * max(1.0, abs(kl_ref))


def test_grad_plain_form_matches_oracle(gpu):
    n = 3000
    X, P = mixture_P(n)
    Y = embedding(n, 5.0)
    g, Z = api.kl_grad_plain(_dev_csr(P, gpu), torch.tensor(Y, device=gpu), 12.0)
    g_ref, Z_ref = _oracle_grad(P, Y, 12.0)
    assert rel_l2(g.cpu().numpy(), g_ref) < GRAD_TOL
    assert abs(Z.item() / Z_ref - 1) < 1e-5


def test_batched_samples_match_per_sample_oracle(gpu):
    sizes = [2, 700, 3, 1500, 257, 40, 4500, 2048]
    Ps = [mixture_P(s, seed=i)[1] for i, s in enumerate(sizes)]
    Pb = block_diag(Ps)
    Y = embedding(sum(sizes), 3.0, seed=7)
    batch = api.Batch(sizes)
    for variant in VARIANTS:
        prm = L.default_params(variant=variant)
        g, Z, kl = api.kl_grad(_dev_csr(Pb, gpu), torch.tensor(Y, device=gpu), 4.0, batch=batch,
                               params=prm, want_kl=True)
        g = g.cpu().numpy()
        for s, P in enumerate(Ps):
            a, b = batch.pt_off[s], batch.pt_off[s + 1]
            g_ref, Z_ref = _oracle_grad(P, Y[a:b], 4.0)
            ge, re = grad_err(g[a:b], P, Y[a:b], 4.0), row_err(g[a:b], P, Y[a:b], 4.0)
            kl_ref = oracle.kl(P, Y[a:b].astype(np.float64), 4.0, Z_ref)
            record(f"batched_grad/variant{variant}/sample{s}", grad_rel_l2=ge, grad_max_row=re,
                   Z_rel=abs(Z[s].item() / Z_ref - 1), kl_abs=abs(kl[s].item() - kl_ref))
            assert ge < GRAD_TOL, s
            assert re < ROW_TOL, s
            assert abs(Z[s].item() / Z_ref - 1) < 1e-6
            assert abs(kl[s].item() - kl_ref) < 1e-6 * max(1.0, abs(kl_ref))


# Sizes whose last group of points (1024 for the SYM4 forms, 2048 for SYM) ends in
# each of its 256-point blocks: the group pairs against it have 1 .. W non-empty
# column blocks (skipped blocks, or per-warp column sums in the partial-buffer
# form), and its diagonal item 1 .. W non-empty blocks (triangles of a partial
# block, half visits against empty ones).
PARTIAL_SIZES = {
    L.TSNE_VARIANT_SYM4: [1024 + 200, 1024 + 300, 1024 + 600, 1024 + 800, 2048 + 1, 3072 + 255],
    L.TSNE_VARIANT_SYM4_FX: [1024 + 200, 1024 + 300, 1024 + 600, 1024 + 800, 3072 + 257],
    L.TSNE_VARIANT_SYM: [2048 + 100, 2048 + 700, 2048 + 1300, 2048 + 1900, 4096 + 513],
}


@pytest.mark.parametrize("variant", list(PARTIAL_SIZES))
def test_partial_last_groups_match_oracle(gpu, variant):
    sizes = PARTIAL_SIZES[variant]
    prm = L.default_params(variant=variant)
    for n in sizes:
        X, P = mixture_P(n, seed=n)
        Y = embedding(n, 2.0, seed=n + 1)
        g, Z, _ = api.kl_grad(_dev_csr(P, gpu), torch.tensor(Y, device=gpu), 12.0, params=prm)
        g = g.cpu().numpy()
        _, Z_ref = _oracle_grad(P, Y, 12.0)
        ge, re = grad_err(g, P, Y, 12.0), row_err(g, P, Y, 12.0)
        record(f"partial_groups/variant{variant}/n{n}", grad_rel_l2=ge, grad_max_row=re,
               Z_rel=abs(Z.item() / Z_ref - 1))
        assert ge < GRAD_TOL, n
        assert re < ROW_TOL, n
        assert abs(Z.item() / Z_ref - 1) < 1e-6, n
    # the same samples in one call, with two tiny ones between them
    bsizes = sizes[:2] + [2, 257] + sizes[2:]
    Ps = [mixture_P(s, seed=s)[1] for s in bsizes]
    Y = embedding(sum(bsizes), 2.0, seed=5)
    batch = api.Batch(bsizes)
    g, Z, _ = api.kl_grad(_dev_csr(block_diag(Ps), gpu), torch.tensor(Y, device=gpu), 12.0,
                          batch=batch, params=prm)
    g = g.cpu().numpy()
    for s, P in enumerate(Ps):
        a, b = batch.pt_off[s], batch.pt_off[s + 1]
        _, Z_ref = _oracle_grad(P, Y[a:b], 12.0)
        ge, re = grad_err(g[a:b], P, Y[a:b], 12.0), row_err(g[a:b], P, Y[a:b], 12.0)
        record(f"partial_groups_batched/variant{variant}/sample{s}", grad_rel_l2=ge,
               grad_max_row=re, Z_rel=abs(Z[s].item() / Z_ref - 1))
        assert ge < GRAD_TOL, s
        assert re < ROW_TOL, s
        assert abs(Z[s].item() / Z_ref - 1) < 1e-6, s


@pytest.mark.parametrize("variant", VARIANTS)
def test_grad_is_deterministic(gpu, variant):
    n = 5000
    X, P = mixture_P(n)
    Y = torch.tensor(embedding(n, 2.0), device=gpu)
    Pd = _dev_csr(P, gpu)
    prm = L.default_params(variant=variant)
    g1, Z1, _ = api.kl_grad(Pd, Y, 12.0, params=prm)
    g2, Z2, _ = api.kl_grad(Pd, Y, 12.0, params=prm)
    assert torch.equal(g1, g2) and torch.equal(Z1, Z2)


def test_symmetric_and_direct_forms_agree_at_scale(gpu):
    # 40,000 points: 20 groups, 190 symmetric items; no oracle needed beyond the
    # sampled rows (exact FP64 forces for 300 rows against all points).
    n = 40000
    rng = np.random.default_rng(9)
    Y = (rng.normal(size=(n, 2)) * 15).astype(np.float32)
    Pempty = oracle.CSR(np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0))
    Pd = _dev_csr(Pempty, gpu)
    Yd = torch.tensor(Y, device=gpu)
    out = {}
    for v in (L.TSNE_VARIANT_DIRECT_L, L.TSNE_VARIANT_SYM):
        g, Z, _ = api.kl_grad(Pd, Yd, 1.0, params=L.default_params(variant=v))
        out[v] = (g.cpu().numpy().astype(np.float64), Z.item())
    rows = np.sort(rng.choice(n, 300, replace=False))
    _, Fr, Zi, _, Ar = oracle.forces_rows(Pempty, Y.astype(np.float64), rows, scales=True)
    Z_ref = oracle.Z(Y.astype(np.float64))
    for v, (g, Z) in out.items():
        assert abs(Z / Z_ref - 1) < 1e-6
        # with P empty, g = -4 Fr / Z
        assert rel_l2(g[rows], -4 * Fr / Z_ref) < GRAD_TOL
        assert row_err_scaled(g[rows] + 4 * Fr / Z_ref, 4 * Ar / Z_ref) < ROW_TOL


@pytest.mark.parametrize("scale", [1e-3, 3e3])
@pytest.mark.parametrize("variant", [L.TSNE_VARIANT_SYM, L.TSNE_VARIANT_SYM4,
                                     L.TSNE_VARIANT_SYM4_FX])
def test_symmetric_split_across_scales(gpu, scale, variant):
    """Tightly packed points (forces ~ n |y|) and widely spread ones (forces
    ~ 1e-5) keep the gradient tolerance on sampled rows against the oracle's
    exact FP64 sums, with partial buffers and with the fixed-point sums (scale
    2^(62 - bitlen(n)): absolute resolution 2^-48 here).  Z: 1e-6, except when
    the points are packed so tightly that every w is within 1e-6 of 1; the
    kernels' FP32 running sums of 256 such terms then round away deviations
    below half an ulp, an error bounded by 255 u = 1.5e-5 (u = 2^-24)."""
    n = 20000
    rng = np.random.default_rng(21)
    Y = (rng.normal(size=(n, 2)) * scale).astype(np.float32)
    Pempty = oracle.CSR(np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0))
    g, Z, _ = api.kl_grad(_dev_csr(Pempty, gpu), torch.tensor(Y, device=gpu), 1.0,
                          params=L.default_params(variant=variant))
    rows = np.sort(rng.choice(n, 200, replace=False))
    _, Fr, _, _, Ar = oracle.forces_rows(Pempty, Y.astype(np.float64), rows, scales=True)
    Z_ref = oracle.Z(Y.astype(np.float64))
    assert abs(Z.item() / Z_ref - 1) < (1e-6 if scale >= 1 else 255 * 2.0 ** -24)
    g = g.cpu().numpy().astype(np.float64)
    assert rel_l2(g[rows], -4 * Fr / Z_ref) < GRAD_TOL
    assert row_err_scaled(g[rows] + 4 * Fr / Z_ref, 4 * Ar / Z_ref) < ROW_TOL


@pytest.mark.parametrize("sizes", [[20000], [16384], [3000], [9000, 16385, 3000, 12288]])
def test_tiled_fixed_point_form(gpu, sizes):
    """The fixed-point form in tiles of 4 x 4 group pairs (full tiles, diagonal
    tiles, the tiles of a partial last block of groups, a last group of one
    point), on single samples and on a batch: per sample Z to 1e-6, and F_r of
    sampled rows against the oracle (relative L2 and per row, ROW_TOL); the
    result is bitwise reproducible."""
    n = sum(sizes)
    rng = np.random.default_rng(len(sizes) + 3)
    Y = (rng.normal(size=(n, 2)) * 20).astype(np.float32)
    Pd = api.CSR(torch.zeros(n + 1, dtype=torch.int64, device=gpu),
                 torch.zeros(1, dtype=torch.int32, device=gpu),
                 torch.zeros(1, dtype=torch.float32, device=gpu))
    batch = api.Batch(sizes) if len(sizes) > 1 else None
    prm = L.default_params(variant=L.TSNE_VARIANT_SYM4_FX)
    Yd = torch.tensor(Y, device=gpu)
    g, Z, _ = api.kl_grad(Pd, Yd, 1.0, batch=batch, params=prm)
    g2, Z2, _ = api.kl_grad(Pd, Yd, 1.0, batch=batch, params=prm)
    assert torch.equal(g, g2) and torch.equal(Z, Z2)
    g = g.cpu().numpy().astype(np.float64)
    off = np.concatenate([[0], np.cumsum(sizes)])
    for s in range(len(sizes)):
        a, b = off[s], off[s + 1]
        Ys = Y[a:b].astype(np.float64)
        Pe = oracle.CSR(np.zeros(b - a + 1, dtype=np.int64), np.zeros(0, dtype=np.int32),
                        np.zeros(0))
        rows = np.sort(rng.choice(b - a, 150, replace=False))
        _, Fr, _, _, Ar = oracle.forces_rows(Pe, Ys, rows, scales=True)
        Z_ref = oracle.Z(Ys)
        assert abs(Z[s].item() / Z_ref - 1) < 1e-6
        gs = g[a:b][rows]
        assert rel_l2(gs, -4 * Fr / Z_ref) < GRAD_TOL
        assert row_err_scaled(gs + 4 * Fr / Z_ref, 4 * Ar / Z_ref) < ROW_TOL


@pytest.mark.parametrize("variant", [L.TSNE_VARIANT_SYM4_FX, L.TSNE_VARIANT_FUSED])
@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_nonfinite_positions_raise_status(gpu, variant, bad):
    """A non-finite position makes partial forces non-finite: the fixed-point
    form leaves them out of its sums and raises TSNE_STATUS_NONFINITE from
    kl_grad; a step raises it when the updated positions are non-finite."""
    n = 5000
    X, P = mixture_P(n)
    Y = embedding(n, 2.0)
    Y[17, 0] = bad
    st = api.new_status(gpu)
    Yd = torch.tensor(Y, device=gpu)
    prm = L.default_params(variant=variant)
    if variant == L.TSNE_VARIANT_FUSED:
        api.step(_dev_csr(P, gpu), Yd, torch.zeros_like(Yd), torch.ones_like(Yd), 0, prm,
                 status=st)
    else:
        api.kl_grad(_dev_csr(P, gpu), Yd, 1.0, params=prm, status=st)
    torch.cuda.synchronize()
    assert st.item() & L.TSNE_STATUS_NONFINITE


def _state(n, seed):
    """A seeded optimiser state (Y, velocity, gains) generated on the host."""
    rng = np.random.default_rng(seed)
    Y = rng.normal(0.0, 1e-2 * (1 + seed % 3), size=(n, 2))
    U = rng.normal(0.0, 1e-3, size=(n, 2))
    G = rng.uniform(0.5, 2.0, size=(n, 2))
    return Y.astype(np.float32), U.astype(np.float32), G.astype(np.float32)


def test_step_matches_oracle_iteration(gpu):
    """One optimiser iteration at each schedule phase (exaggeration and momentum
    0.5 at it < 2, then 1 and 0.8) from the same host-generated state on both
    sides."""
    n = 1500
    X, P = mixture_P(n)
    prm = L.default_params(ee_iters=2, mom_switch=2, lr=0.0, kl_every=0)
    Pd = _dev_csr(P, gpu)
    for it in range(4):
        Ys, Us, Gs = _state(n, 30 + it)
        Y, U, G = (torch.tensor(a, device=gpu) for a in (Ys, Us, Gs))
        Yo, Uo, Go = (a.astype(np.float64) for a in (Ys, Us, Gs))
        mu = 0.5 if it < 2 else 0.8
        Yr, Ur, Gr, _ = oracle.run(P, Yo, n_iter=1, ee_iters=1 if it < 2 else 0, ee=12.0,
                                   mom_switch=1 if it < 2 else 0, mom0=mu, mom1=mu, eta=n / 12.0,
                                   U0=Uo, gains0=Go)
        api.step(Pd, Y, U, G, it, prm)
        du_ref = Ur - Uo * mu
        same_gain = np.isclose(G.cpu().numpy(), Gr, rtol=1e-6)
        assert same_gain.mean() > 0.999
        m = same_gain.all(axis=1)
        assert rel_l2(U.cpu().numpy()[m] - Uo[m] * mu, du_ref[m]) < GRAD_TOL


def test_plain_step_matches_oracle_iteration(gpu):
    """The plain GPU form's whole iteration (tsne_step_plain), the comparison
    baseline of the metric's "vs plain", from the same host states as above; its
    FP32 running sums over all n columns allow only the relative L2 bound."""
    n = 1500
    X, P = mixture_P(n)
    prm = L.default_params(ee_iters=2, mom_switch=2, lr=0.0, kl_every=0)
    Pd = _dev_csr(P, gpu)
    for it in range(4):
        Ys, Us, Gs = _state(n, 30 + it)
        Y, U, G = (torch.tensor(a, device=gpu) for a in (Ys, Us, Gs))
        Yo, Uo, Go = (a.astype(np.float64) for a in (Ys, Us, Gs))
        mu = 0.5 if it < 2 else 0.8
        Yr, Ur, Gr, _ = oracle.run(P, Yo, n_iter=1, ee_iters=1 if it < 2 else 0, ee=12.0,
                                   mom_switch=1 if it < 2 else 0, mom0=mu, mom1=mu, eta=n / 12.0,
                                   U0=Uo, gains0=Go)
        api.step_plain(Pd, Y, U, G, it, prm)
        same_gain = np.isclose(G.cpu().numpy(), Gr, rtol=1e-6)
        assert same_gain.mean() > 0.999
        m = same_gain.all(axis=1)
        assert rel_l2(U.cpu().numpy()[m] - Uo[m] * mu, (Ur - Uo * mu)[m]) < GRAD_TOL
        np.testing.assert_allclose(Y.cpu().numpy()[m], Yo[m] + U.cpu().numpy()[m], rtol=0,
                                   atol=1e-6 * np.abs(Yo).max())


@pytest.mark.parametrize("variant", [L.TSNE_VARIANT_AUTO, L.TSNE_VARIANT_SYM])
def test_step_device_counter_equals_host_iterations(gpu, variant):
    n = 4100
    X, P = mixture_P(n)
    Y0 = torch.tensor(embedding(n, 1e-2, seed=5), device=gpu)
    prm = L.default_params(ee_iters=2, mom_switch=3, kl_every=2, n_iter=6, variant=variant)
    Pd = _dev_csr(P, gpu)
    outs = []
    for mode in ("host", "device"):
        Y, U, G = Y0.clone(), torch.zeros_like(Y0), torch.ones_like(Y0)
        kl = torch.zeros(3, dtype=torch.float64, device=gpu)
        ws = None
        if mode == "device":
            ws = api.Workspace(api.workspace_size(L.TSNE_OP_KL_GRAD, n, params=prm), gpu)
            api.step_reset(ws, 0, gpu)
        for it in range(6):
            ws = api.step(Pd, Y, U, G, it if mode == "host" else -1, prm, kl=kl, ws=ws)
        outs.append((Y, U, G, kl))
    for a, b in zip(outs[0], outs[1]):
        assert torch.equal(a, b)
    assert (outs[0][3] > 0).all()


def test_bad_column_index_sets_status_and_is_skipped(gpu):
    n = 300
    X, P = mixture_P(n)
    col = P.col.copy()
    col[5] = n + 1000  # outside [0, n): the attraction kernel must skip it and flag it
    Pbad = oracle.CSR(P.row_ptr, col, P.val)
    st = api.new_status(gpu)
    g, Z, _ = api.kl_grad(_dev_csr(Pbad, gpu), torch.tensor(embedding(n, 1.0), device=gpu), 1.0,
                          status=st)
    torch.cuda.synchronize()
    assert st.item() & L.TSNE_STATUS_BAD_INDEX
    assert torch.isfinite(g).all()


BATCH_SIZES = [600, 2048, 1500, 3000, 700, 91]


def _batched_problem(gpu, seed=0):
    Ps = [mixture_P(n, seed=10 + i)[1] for i, n in enumerate(BATCH_SIZES)]
    Pb = block_diag(Ps)
    return Ps, Pb, _dev_csr(Pb, gpu), api.Batch(BATCH_SIZES)


@pytest.mark.parametrize("variant", [L.TSNE_VARIANT_FUSED, L.TSNE_VARIANT_AUTO,
                                     L.TSNE_VARIANT_SYM4])
def test_batched_step_matches_oracle_per_sample(gpu, variant):
    """One iteration of a batch: the persistent launch (TSNE_VARIANT_FUSED), the
    per-term kernels as AUTO runs them here (one forces launch of attraction rows
    and small direct items, then the update kernel, which sums each sample's Z
    partials itself) and the symmetric split: every sample's update equals the
    oracle's iteration from the same host-generated state."""
    Ps, Pb, Pd, batch = _batched_problem(gpu)
    n = batch.n
    prm = L.default_params(variant=variant, ee_iters=2, mom_switch=2, kl_every=0)
    for it in range(3):
        Ys, Us, Gs = _state(n, 40 + it)
        Y, U, G = (torch.tensor(a, device=gpu) for a in (Ys, Us, Gs))
        Yo, Uo, Go = (a.astype(np.float64) for a in (Ys, Us, Gs))
        api.step(Pd, Y, U, G, it, prm, batch=batch)
        mu = 0.5 if it < 2 else 0.8
        Un, Gn = U.cpu().numpy(), G.cpu().numpy()
        for s, P in enumerate(Ps):
            a, b = batch.pt_off[s], batch.pt_off[s + 1]
            Yr, Ur, Gr, _ = oracle.run(P, Yo[a:b], n_iter=1, ee_iters=1 if it < 2 else 0, ee=12.0,
                                       mom_switch=1 if it < 2 else 0, mom0=mu, mom1=mu,
                                       eta=(b - a) / 12.0, U0=Uo[a:b], gains0=Go[a:b])
            same = np.isclose(Gn[a:b], Gr, rtol=1e-6).all(axis=1)
            du = rel_l2(Un[a:b][same] - Uo[a:b][same] * mu, (Ur - Uo[a:b] * mu)[same])
            tag = "fused_step" if variant == L.TSNE_VARIANT_FUSED else f"batched_step/v{variant}"
            record(f"{tag}/it{it}/sample{s}", update_rel_l2=du, gains_same=same.mean())
            assert same.mean() > 0.99
            assert du < GRAD_TOL


@pytest.mark.parametrize("variant", [L.TSNE_VARIANT_FUSED, L.TSNE_VARIANT_AUTO])
def test_batched_device_counter_and_kl_trace(gpu, variant):
    """Device-counter steps (iter = -1) equal host-numbered steps bitwise, and the
    KL trace and Z agree with tsne_kl_grad's at alpha = 1 of the same Y (for AUTO
    the trace comes from the update kernel's own reduction)."""
    Ps, Pb, Pd, batch = _batched_problem(gpu)
    n, S = batch.n, batch.S
    prm = L.default_params(variant=variant, ee_iters=3, mom_switch=3, kl_every=2, n_iter=6)
    Y0 = torch.tensor(embedding(n, 1e-2, seed=6), device=gpu)
    outs = []
    for mode in ("host", "device"):
        Y, U, G = Y0.clone(), torch.zeros_like(Y0), torch.ones_like(Y0)
        kl = torch.zeros(3 * S, dtype=torch.float64, device=gpu)
        Z = torch.zeros(S, dtype=torch.float64, device=gpu)
        ws = api.Workspace(api.workspace_size(L.TSNE_OP_KL_GRAD, n, batch=batch, params=prm), gpu)
        api.step_reset(ws, 0, gpu)
        Ysnap = None
        for it in range(6):
            if it == 5:
                Ysnap = Y.clone()
            api.step(Pd, Y, U, G, it if mode == "host" else -1, prm, batch=batch, Z=Z, kl=kl, ws=ws)
        outs.append((Y, U, G, kl, Z, Ysnap))
    for a_, b_ in zip(outs[0][:5], outs[1][:5]):
        assert torch.equal(a_, b_)
    # last KL slot (iteration 5) is KL(P||Q) of the Y the iteration started from
    Ysnap = outs[0][5]
    _, Zr, klr = api.kl_grad(Pd, Ysnap, 1.0, batch=batch, want_kl=True,
                             params=L.default_params(variant=L.TSNE_VARIANT_DIRECT_S))
    kl_last = outs[0][3].view(3, S)[2]
    assert torch.allclose(kl_last, klr, rtol=0, atol=1e-6)
    assert torch.allclose(outs[0][4], Zr, rtol=1e-6, atol=0)


def test_fused_equals_per_term_step(gpu):
    """The fused launch and the per-term kernels (same direct form, different
    chunking) give the same iteration within the gradient tolerance."""
    Ps, Pb, Pd, batch = _batched_problem(gpu)
    n = batch.n
    Y0 = torch.tensor(embedding(n, 3.0, seed=2), device=gpu)
    res = []
    for v in (L.TSNE_VARIANT_FUSED, L.TSNE_VARIANT_DIRECT_S):
        Y, U, G = Y0.clone(), torch.zeros_like(Y0), torch.ones_like(Y0)
        api.step(Pd, Y, U, G, 0, L.default_params(variant=v), batch=batch)
        res.append((Y - Y0).cpu().numpy())
    assert rel_l2(res[0], res[1]) < GRAD_TOL


def test_step_captured_as_a_threads_first_call_equals_eager_steps(gpu):
    """The attraction runs on a per-thread side stream forked from the caller's
    stream and joined back.  A fresh host thread whose first library call is
    inside a CUDA-graph capture (global capture mode) creates that stream during
    the capture; the replayed graph must equal the same steps run eagerly."""
    import threading

    n = 3000
    X, P = mixture_P(n)
    Pd = _dev_csr(P, gpu)
    prm = L.default_params(ee_iters=3, mom_switch=3, kl_every=0, n_iter=6,
                           variant=L.TSNE_VARIANT_SYM4)
    Y0 = torch.tensor(embedding(n, 1e-2, seed=9), device=gpu)
    Ye, Ue, Ge = Y0.clone(), torch.zeros_like(Y0), torch.ones_like(Y0)
    for it in range(6):
        api.step(Pd, Ye, Ue, Ge, it, prm)
    torch.cuda.synchronize()

    out = {}

    def body():
        try:
            torch.cuda.set_device(gpu)
            Y, U, G = Y0.clone(), torch.zeros_like(Y0), torch.ones_like(Y0)
            ws = api.Workspace(api.workspace_size(L.TSNE_OP_KL_GRAD, n, params=prm), gpu)
            st = api.new_status(gpu)
            s = torch.cuda.Stream(gpu)
            s.wait_stream(torch.cuda.current_stream(gpu))
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                for it in range(6):
                    api.step(Pd, Y, U, G, it, prm, ws=ws, status=st)
            g.replay()
            torch.cuda.synchronize()
            out["Y"], out["st"] = Y.clone(), int(st.item())
        except Exception as e:  # reported on the main thread
            out["err"] = repr(e)

    t = threading.Thread(target=body)
    t.start()
    t.join()
    assert "err" not in out, out.get("err")
    assert out["st"] == 0
    assert torch.equal(out["Y"], Ye)


def test_concurrent_threads_each_fork_their_own_side_stream(gpu):
    """Two host threads compute symmetric-kernel gradients at the same time, each
    on its own stream (and so each with its own side stream for the attraction);
    every result equals the same call made alone."""
    import threading

    n = 5000
    X, P = mixture_P(n)
    Pd = _dev_csr(P, gpu)
    prm = L.default_params(variant=L.TSNE_VARIANT_SYM4)
    Ys = [torch.tensor(embedding(n, 1.0, seed=s), device=gpu) for s in (21, 22)]
    ref = []
    for Y in Ys:
        g, Z, kl = api.kl_grad(Pd, Y, 12.0, want_kl=True, params=prm)
        torch.cuda.synchronize()
        ref.append((g.clone(), Z.clone(), kl.clone()))
    out = [None, None]
    errs = []

    def body(r):
        try:
            torch.cuda.set_device(gpu)
            s = torch.cuda.Stream(gpu)
            res = []
            with torch.cuda.stream(s):
                for _ in range(5):
                    g, Z, kl = api.kl_grad(Pd, Ys[r], 12.0, want_kl=True, params=prm)
                    res.append((g, Z, kl))
            s.synchronize()
            out[r] = res
        except Exception as e:  # reported on the main thread
            errs.append(repr(e))

    ts = [threading.Thread(target=body, args=(r,)) for r in (0, 1)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errs, errs
    for r in (0, 1):
        for g, Z, kl in out[r]:
            assert torch.equal(g, ref[r][0]) and torch.equal(Z, ref[r][1])
            assert torch.equal(kl, ref[r][2])
