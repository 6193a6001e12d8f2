"""The autotuner picks a variant that runs, caches it per shape, and reuses it."""
import json

import pytest

from paper_2605_13928_b300 import _lib as L
from paper_2605_13928_b300 import autotune

pytestmark = pytest.mark.gpu


def test_autotune_picks_and_caches(gpu, tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("TSNE_AUTOTUNE_CACHE", str(path))
    sizes = [700, 1800, 2500, 900]
    best = autotune.tune(sizes, gpu, reps=2)
    assert best["variant"] in autotune.CANDIDATES_BATCH
    assert best["ms"] == min(best["timings"].values())
    data = json.loads(path.read_text())
    assert autotune.shape_key(sizes, gpu) in data
    again = autotune.tune(sizes, gpu)
    assert again == best
    single = autotune.tune([20000], gpu, reps=2)
    assert single["variant"] in autotune.CANDIDATES_SINGLE
    prm = autotune.tuned_params([20000], gpu, kl_every=0)
    assert prm.variant == single["variant"]
