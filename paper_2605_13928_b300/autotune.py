"""Autotuner of the repulsion kernel shape (tsne_params.variant).

For a problem shape (sample sizes) it times every candidate variant through
the library -- one optimiser step through tsne_step on a random embedding
with a random P of a perplexity-30 graph's density (the attraction's cost
differs between the fused and the per-term kernels) -- with CUDA events, and
keeps the fastest.  Results are cached in a JSON file keyed by
GPU name, SM count and the sizes' profile (number of samples, largest sample
and total pairs in powers-of-two buckets), so each shape is tuned once per
machine.  The cache path is $TSNE_AUTOTUNE_CACHE or
~/.cache/tsne_b300/autotune.json.
"""
from __future__ import annotations

import json
import math
import os
from typing import Dict, Optional, Sequence

import numpy as np
import torch

from . import _lib as L
from . import api

CANDIDATES_SINGLE = (L.TSNE_VARIANT_DIRECT, L.TSNE_VARIANT_DIRECT_L, L.TSNE_VARIANT_DIRECT_S,
                     L.TSNE_VARIANT_DIRECT_M, L.TSNE_VARIANT_SYM, L.TSNE_VARIANT_SYM4,
                     L.TSNE_VARIANT_SYM4_FX)
CANDIDATES_BATCH = CANDIDATES_SINGLE + (L.TSNE_VARIANT_FUSED,)
# part of the cache key: results cached for another candidate list are not reused
CANDIDATES_VERSION = 2
NAMES = {L.TSNE_VARIANT_DIRECT: "direct_by_size", L.TSNE_VARIANT_DIRECT_L: "direct_256x8_1024", L.TSNE_VARIANT_DIRECT_S: "direct_128x4_256",
         L.TSNE_VARIANT_DIRECT_M: "direct_256x4_512", L.TSNE_VARIANT_SYM: "symmetric_2048",
         L.TSNE_VARIANT_SYM4: "symmetric_1024", L.TSNE_VARIANT_FUSED: "fused_batched",
         L.TSNE_VARIANT_SYM4_FX: "symmetric_1024_tiled_fixed_point"}


def cache_path() -> str:
    return os.environ.get("TSNE_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "tsne_b300",
                                       "autotune.json"))


def shape_key(sizes: Sequence[int], device=None) -> str:
    props = torch.cuda.get_device_properties(device or torch.cuda.current_device())
    sizes = np.asarray(sizes, dtype=np.int64)
    b = lambda x: int(math.log2(max(int(x), 1)))  # noqa: E731
    pairs = float((sizes.astype(np.float64) ** 2).sum())
    return (f"{props.name}|sms={props.multi_processor_count}|S={len(sizes)}|"
            f"nmax=2^{b(sizes.max())}|pairs=2^{b(pairs)}|nnz/row={NNZ_PER_ROW}|"
            f"candidates={CANDIDATES_VERSION}")


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, data):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


NNZ_PER_ROW = 140  # a symmetrised kNN graph with k = 90 holds ~1.5 k entries per row


def synthetic_P(sizes: Sequence[int], device, seed: int = 0, per_row: int = NNZ_PER_ROW):
    """A CSR with the density of a perplexity-30 P (per_row random columns of
    the row's own sample, sorted), so that the attraction's cost is timed too."""
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    cols, off = [], 0
    for s in sizes:
        m = min(per_row, max(s - 1, 1))
        c = torch.randint(0, s, (s, m), generator=g, device=device, dtype=torch.int64)
        cols.append((c.sort(dim=1).values + off).to(torch.int32))
        off += s
    col = torch.cat([c.reshape(-1) for c in cols])
    counts = torch.cat([torch.full((s,), c.shape[1], dtype=torch.int64, device=device)
                        for s, c in zip(sizes, cols)])
    row_ptr = torch.zeros(off + 1, dtype=torch.int64, device=device)
    row_ptr[1:] = torch.cumsum(counts, 0)
    val = torch.full((col.numel(),), 1.0 / col.numel(), dtype=torch.float32, device=device)
    return api.CSR(row_ptr, col, val)


def time_variant(variant: int, sizes: Sequence[int], device, reps: int = 3,
                 seed: int = 0) -> float:
    """Median ms of one tsne_step with the given variant on a random embedding
    and a P of realistic density."""
    sizes = [int(s) for s in sizes]
    n = sum(sizes)
    batch = api.Batch(sizes) if len(sizes) > 1 else None
    rng = np.random.default_rng(seed)
    Y = torch.tensor((rng.normal(size=(n, 2)) * 10).astype(np.float32), device=device)
    U = torch.zeros_like(Y)
    G = torch.ones_like(Y)
    P = synthetic_P(sizes, device, seed)
    prm = L.default_params(variant=variant, ee_iters=0, mom_switch=0, kl_every=0)
    ws = api.Workspace(api.workspace_size(L.TSNE_OP_KL_GRAD, n, batch=batch, params=prm), device)
    Yw = Y.clone()
    api.step(P, Yw, U, G, 0, prm, batch=batch, ws=ws)  # warm-up (and code load)
    times = []
    for _ in range(reps):
        Yw.copy_(Y)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        api.step(P, Yw, U, G, 0, prm, batch=batch, ws=ws)
        e1.record()
        torch.cuda.synchronize(device)
        times.append(e0.elapsed_time(e1))
    return float(np.median(times))


def tune(sizes: Sequence[int], device=None, candidates: Optional[Sequence[int]] = None,
         use_cache: bool = True, reps: int = 3) -> Dict:
    """Best variant for these sample sizes: {"variant", "name", "ms", "timings"}."""
    device = torch.device(device) if device is not None else torch.device("cuda", 0)
    key = shape_key(sizes, device)
    path = cache_path()
    data = _load(path) if use_cache else {}
    if use_cache and key in data:
        return data[key]
    if candidates is None:
        candidates = CANDIDATES_BATCH if len(sizes) > 1 else CANDIDATES_SINGLE
    timings = {}
    for v in candidates:
        try:
            timings[NAMES.get(v, str(v))] = (v, time_variant(v, sizes, device, reps=reps))
        except (L.TsneError, RuntimeError):
            continue  # a variant that cannot serve this shape
    if not timings:
        raise RuntimeError("no variant could be timed")
    name, (v, ms) = min(timings.items(), key=lambda kv: kv[1][1])
    result = {"variant": int(v), "name": name, "ms": ms,
              "timings": {k: t for k, (_, t) in timings.items()}}
    if use_cache:
        data[key] = result
        _store(path, data)
    return result


def tuned_params(sizes: Sequence[int], device=None, **over) -> L.TsneParams:
    """Default parameters with the autotuned repulsion variant for these sizes."""
    best = tune(sizes, device)
    return L.default_params(variant=best["variant"], **over)
