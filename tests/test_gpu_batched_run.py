"""The batched configuration run as configured: 64 independent samples with sizes
log-uniform on [500, 20000] (about 282,000 points), each a 50-D mixture of
5-20 equal clusters, k = 90, perplexity 30, 750 iterations (exaggeration 12
and momentum 0.5 for 250, then 1 and 0.8, learning rate n_s / 12 per sample),
driven through tsne_step with the device iteration counter, steps captured in
CUDA graphs of 25, with the autotuned repulsion form.

At iterations 250, 500 and 750, on the embedding the run has reached, every
sample's exact gradient against the FP64 oracle: the GPU's gradient with the
oracle's own P of that sample (built by the oracle from the sample's X) against
oracle.grad on the same P and Y, 1e-4 relative L2 (against the larger of the
gradient's and its two terms' norms, as problems.grad_err: near convergence the
terms cancel) and per row (problems.ROW_TOL), and Z_s to 1e-6.  The states Y_t are the run's own (the
oracle cannot run 64 trajectories); no force, Z or gradient computed on the GPU
enters the oracle.  The run also keeps every sample finite with no status bit,
and its KL trace (summed over the samples) falls after early exaggeration.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_13928_b300 import _lib as L
from paper_2605_13928_b300 import api, autotune, synth
from problems import ROW_TOL, record, rel_l2, row_err_scaled

pytestmark = pytest.mark.gpu

CHECKS = (250, 500, 750)


@pytest.fixture(scope="module")
def batched_oracle_P():
    Xs = synth.batch()
    Ps = [oracle.affinities(X.astype(np.float64), 90, 30.0)[0] for X in Xs]
    return Xs, Ps


def _check_sample(P, Yd, a, b, alpha, gpu, variant, tag):
    Y = Yd[a:b].contiguous()
    Pd = api.CSR.from_numpy(P.row_ptr, P.col, P.val, gpu)
    g, Z, _ = api.kl_grad(Pd, Y, alpha, params=L.default_params(variant=variant))
    Y64 = Y.cpu().numpy().astype(np.float64)
    g_ref, Z_ref = oracle.grad(P, Y64, alpha)
    Fa, Fr, _, Aa, Ar = oracle.forces_rows(P, Y64, scales=True)
    g = g.cpu().numpy().astype(np.float64)
    # relative L2 as in problems.grad_err: against the larger of |g_ref| and the
    # two terms' norms, since near convergence they cancel and |g_ref| shrinks
    den = max(np.linalg.norm(g_ref), 4 * alpha * np.linalg.norm(Fa), 4 * np.linalg.norm(Fr) / Z_ref)
    l2 = float(np.linalg.norm(g - g_ref) / den)
    row = row_err_scaled(g - g_ref, 4 * (alpha * Aa + Ar / Z_ref))
    zr = abs(Z.item() / Z_ref - 1)
    record(tag, grad_rel_l2=l2, grad_rel_l2_plain=rel_l2(g, g_ref), grad_max_row=row, Z_rel=zr)
    return l2, row, zr


def test_batched64_750_iterations_checked_per_sample(gpu, batched_oracle_P):
    Xs, Ps = batched_oracle_P
    sizes = [len(x) for x in Xs]
    batch = api.Batch(sizes)
    n = batch.n
    X = torch.tensor(np.concatenate(Xs), device=gpu)
    st = api.new_status(gpu)
    idx, d2 = api.knn(X, 90, batch=batch, mode=L.TSNE_KNN_BF16_RERANK, status=st)
    P, _, n_bad = api.affinities(idx, d2, 30.0, batch=batch, status=st)
    del idx, d2, X
    best = autotune.tune(sizes, gpu)
    prm = L.default_params(variant=best["variant"], n_iter=750, ee_iters=250, mom_switch=250,
                           kl_every=50)
    Y = torch.tensor(np.concatenate([synth.initial_embedding(s, 11 + i)
                                     for i, s in enumerate(sizes)]), device=gpu)
    U, G = torch.zeros_like(Y), torch.ones_like(Y)
    kl = torch.zeros(15 * len(sizes), dtype=torch.float64, device=gpu)
    ws = api.Workspace(api.workspace_size(L.TSNE_OP_KL_GRAD, n, batch=batch, params=prm), gpu)
    api.step_reset(ws, 0, gpu)
    chunk = 25
    s_cap = torch.cuda.Stream(gpu)
    s_cap.wait_stream(torch.cuda.current_stream(gpu))
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s_cap):
        with torch.cuda.graph(graph, stream=s_cap):
            for _ in range(chunk):
                api.step(P, Y, U, G, -1, prm, batch=batch, kl=kl, ws=ws, status=st)
    torch.cuda.current_stream(gpu).wait_stream(s_cap)
    done = 0
    worst = [0.0, 0.0, 0.0]
    while done < 750:
        graph.replay()
        done += chunk
        if done not in CHECKS:
            continue
        torch.cuda.synchronize()
        assert st.item() == 0 and torch.isfinite(Y).all(), done
        alpha = 12.0 if done < 250 else 1.0
        for s, Ps_ in enumerate(Ps):
            a, b = batch.pt_off[s], batch.pt_off[s + 1]
            res = _check_sample(Ps_, Y, a, b, alpha, gpu, best["variant"],
                                f"batched64_run/it{done}/sample{s}")
            worst = [max(w, r) for w, r in zip(worst, res)]
            assert res[0] < 1e-4 and res[1] < ROW_TOL and res[2] < 1e-6, (done, s, res)
    record("batched64_run/worst", grad_rel_l2=worst[0], grad_max_row=worst[1], Z_rel=worst[2])
    trace = kl.cpu().numpy().reshape(15, len(sizes))
    assert np.isfinite(trace).all()
    assert trace[-1].sum() < trace[5].sum()
