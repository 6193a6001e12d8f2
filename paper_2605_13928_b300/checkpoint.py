"""Checkpoint and resume of an optimisation in progress.

The state of an exact t-SNE run is the embedding Y, the velocity U, the gains
G, the next iteration number and the parameters; P and the sample layout are
rebuilt from the data (or kept by the caller).  Because every kernel sums in a
fixed order, a run resumed from a checkpoint continues bitwise identically to
one that was never interrupted.
"""
from __future__ import annotations

import dataclasses
import os
from typing import Optional

import numpy as np
import torch

from . import _lib as L


@dataclasses.dataclass
class RunState:
    Y: torch.Tensor
    U: torch.Tensor
    G: torch.Tensor
    iteration: int
    params: L.TsneParams


def save(path: str, Y: torch.Tensor, U: torch.Tensor, G: torch.Tensor, iteration: int,
         params: L.TsneParams) -> None:
    """Writes the state to `path` (.npz), atomically."""
    fields = {name: getattr(params, name) for name, _ in params._fields_}
    tmp = path + ".tmp.npz"
    np.savez(tmp, Y=Y.detach().cpu().numpy(), U=U.detach().cpu().numpy(),
             G=G.detach().cpu().numpy(), iteration=np.int64(iteration),
             param_names=np.array(list(fields.keys())),
             param_values=np.array([float(v) for v in fields.values()]))
    os.replace(tmp, path)


def load(path: str, device: Optional[torch.device] = None) -> RunState:
    with np.load(path) as z:
        params = L.TsneParams()
        for name, value in zip(z["param_names"].tolist(), z["param_values"].tolist()):
            kind = dict(L.TsneParams._fields_)[name]
            setattr(params, name, int(value) if kind is not L.ctypes.c_float else float(value))
        mk = (lambda a: torch.tensor(a, device=device)) if device is not None else torch.tensor
        return RunState(mk(z["Y"]), mk(z["U"]), mk(z["G"]), int(z["iteration"]), params)
