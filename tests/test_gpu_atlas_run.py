"""The atlas workload run as configured: N = 1,000,000 cells (50-D mixture of 100
Zipf(1.1)-sized anisotropic clusters), k = 90, perplexity 30, 2-D output, 750
iterations (exaggeration 12 and momentum 0.5 for the first 250, then 1 and 0.8,
learning rate N / 12), driven through tsne_step with the device iteration
counter in the launch configuration bench.py times (AUTO repulsion), with the
gradient checked against the FP64 oracle on 1,000 sampled rows every 50
iterations.

At each of the 15 checkpoints (after 50, 100, ..., 750 iterations), on the
embedding Y_t the run has reached:

* the repulsive forces F_r = -Z g / 4 of a gradient with an empty P, for 1,000
  seeded rows, against the oracle's exact FP64 sums over all 1M points: 1e-4
  relative L2 and, row by row, 3e-4 of the row's term-magnitude sum
  (problems.ROW_TOL);
* the GPU's FP64 Z against the sampled rows' own sums Z_i: sum_i Z_i < Z, and
  Z within six standard errors of the sample mean of Z_i times N;
* the exact Z, by the oracle's full FP64 O(N^2) pass, at the first and the last
  checkpoint (1e-6 relative); the first pass runs on the host cores while the
  GPU continues;
* the full gradient with the real P: finite, sum_i g_i ~ 0;
* no status bit, finite Y, and the KL trace (alpha = 1, every 50 iterations)
  finite and lower at the end than at the end of early exaggeration.

Y_t is the run's own state: no host program can produce a 1M-point t-SNE
trajectory.  It serves only as the point at which both sides evaluate the
repulsion; no force, Z or gradient computed on the GPU enters the oracle.  The
update arithmetic that produced Y_t is pinned separately, one iteration at a
time from host-generated states (test_gpu_grad.test_step_matches_oracle_iteration).

When $TSNE_PARITY_LOG names a file, the measured errors of every checkpoint
are appended to it as JSON lines.
"""
import json
import os
import threading

import numpy as np
import pytest
import torch

import oracle
from paper_2605_13928_b300 import _lib as L
from paper_2605_13928_b300 import api, synth
from problems import ROW_TOL, row_err_scaled

pytestmark = pytest.mark.gpu

EVERY = 50
ROWS = 1000


def _log(rec):
    path = os.environ.get("TSNE_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(rec) + "\n")


def test_atlas_750_iterations_checked_every_50(gpu):
    wl = synth.WORKLOADS["atlas_n1m"]
    n = wl.n
    X = wl.data()
    st = api.new_status(gpu)
    Xd = torch.tensor(X, device=gpu)
    idx, d2 = api.knn(Xd, wl.k, mode=L.TSNE_KNN_BF16_RERANK, status=st)
    P, _, n_bad = api.affinities(idx, d2, wl.perplexity, status=st)
    del idx, d2, Xd, X
    prm = L.default_params(n_iter=wl.n_iter, ee_iters=wl.ee_iters, mom_switch=wl.ee_iters,
                           k=wl.k, perplexity=wl.perplexity, kl_every=EVERY)
    Y = torch.tensor(wl.y0(), device=gpu)
    U, G = torch.zeros_like(Y), torch.ones_like(Y)
    n_kl = wl.n_iter // EVERY
    kl = torch.zeros(n_kl, dtype=torch.float64, device=gpu)
    Zs = torch.zeros(1, dtype=torch.float64, device=gpu)
    ws = api.Workspace(api.workspace_size(L.TSNE_OP_KL_GRAD, n, params=prm), gpu)
    api.step_reset(ws, 0, gpu)
    Pe = api.CSR(torch.zeros(n + 1, dtype=torch.int64, device=gpu),
                 torch.zeros(1, dtype=torch.int32, device=gpu),
                 torch.zeros(1, dtype=torch.float32, device=gpu))
    gws = api.Workspace(api.workspace_size(L.TSNE_OP_KL_GRAD, n), gpu)
    Pempty = oracle.CSR(np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32),
                        np.zeros(0))
    exact_z = {}  # checkpoint -> (thread, result holder, GPU Z)

    def start_exact_z(t, Y64, z_gpu):
        box = {}
        th = threading.Thread(target=lambda: box.update(z=oracle.Z(Y64)), daemon=True)
        th.start()
        exact_z[t] = (th, box, z_gpu)

    checkpoints = list(range(EVERY, wl.n_iter + 1, EVERY))
    for t in range(1, wl.n_iter + 1):
        api.step(P, Y, U, G, -1, prm, Z=Zs, kl=kl, ws=ws, status=st)
        if t not in checkpoints:
            continue
        g, Z, _ = api.kl_grad(Pe, Y, 1.0, ws=gws)
        gP, _, _ = api.kl_grad(P, Y, 1.0 if t > wl.ee_iters else wl.ee)
        torch.cuda.synchronize()
        assert st.item() == 0, f"status {st.item()} at iteration {t}"
        Yh = Y.cpu().numpy()
        assert np.isfinite(Yh).all()
        Y64 = Yh.astype(np.float64)
        z_gpu = Z.item()
        if t in (checkpoints[0], checkpoints[-1]):
            start_exact_z(t, Y64, z_gpu)
        rows = np.sort(np.random.default_rng(1000 + t).choice(n, ROWS, replace=False))
        _, Fr, Zi, _, Ar = oracle.forces_rows(Pempty, Y64, rows, scales=True)
        Fr_gpu = -g.cpu().numpy()[rows].astype(np.float64) * z_gpu / 4.0
        l2 = float(np.linalg.norm(Fr_gpu - Fr) / np.linalg.norm(Fr))
        rowe = row_err_scaled(Fr_gpu - Fr, Ar)
        z_est = n * Zi.mean()
        z_se = n * Zi.std(ddof=1) / np.sqrt(ROWS)
        gp = gP.cpu().numpy().astype(np.float64)
        gsum = float(np.abs(gp.sum(0)).max() / np.abs(gp).sum(0).max())
        rec = {"iteration": t, "extent": float(np.abs(Y64).max()), "Fr_rel_l2": l2,
               "Fr_max_row_err": rowe, "Z_gpu": z_gpu, "Z_sampled_estimate": z_est,
               "Z_sampled_se": z_se, "grad_sum_rel": gsum}
        _log(rec)
        print(json.dumps(rec))
        assert l2 < 1e-4, rec
        assert rowe < ROW_TOL, rec
        assert Zi.sum() < z_gpu and abs(z_gpu - z_est) <= 6 * z_se, rec
        assert np.isfinite(gp).all() and gsum < 1e-4, rec
    for t, (th, box, z_gpu) in exact_z.items():
        th.join()
        err = abs(z_gpu / box["z"] - 1)
        _log({"iteration": t, "Z_exact": box["z"], "Z_gpu": z_gpu, "Z_rel_err": err})
        print(json.dumps({"iteration": t, "Z_exact": box["z"], "Z_rel_err": err}))
        assert err < 1e-6
    trace = kl.cpu().numpy()
    _log({"kl_trace": trace.tolist()})
    assert np.isfinite(trace).all()
    assert trace[-1] < trace[wl.ee_iters // EVERY]
