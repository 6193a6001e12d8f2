"""GPU telemetry monitor: the four verbs of the paper's CudaMon package
(Sec. 2) -- start a sampler for a device at a period, mark named
timestamps, stop it, and parse the trace -- over the libtsne.so C ABI
(tsne_mon_*), whose background thread queries NVML read-only.

    mon = Monitor.start(period=0.2, device=0, csv="trace.csv")
    mon.timestamp("knn")
    ...
    mon.stop()
    trace = mon.parse()          # or parse_csv("trace.csv")

A trace holds `samples` (a dict of numpy columns: t, gpu_util, mem_util,
mem_used_mb, temp_c, power_w, sm_mhz) and `events` (a list of (t, name)),
times in seconds since start.  `summary()` gives per-phase means between
consecutive events, which is how the paper reads its traces (Sec. 3).
"""
from __future__ import annotations

import csv as _csv
import ctypes
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import numpy as np

from . import _lib as L

COLUMNS = ("t", "gpu_util", "mem_util", "mem_used_mb", "temp_c", "power_w", "sm_mhz")


@dataclass
class Trace:
    samples: Dict[str, np.ndarray]
    events: List[Tuple[float, str]] = field(default_factory=list)

    def summary(self) -> List[Dict]:
        """Mean of every column over each phase [event_i, event_{i+1}) (the
        last phase ends at the last sample); fields that failed (-1) are
        left out of the means."""
        t = self.samples["t"]
        marks = list(self.events) + [(float(t[-1]) + 1e-9 if len(t) else 0.0, "")]
        out = []
        for (t0, name), (t1, _) in zip(marks[:-1], marks[1:]):
            sel = (t >= t0) & (t < t1)
            row = {"phase": name, "t0": t0, "t1": t1, "samples": int(sel.sum())}
            for c in COLUMNS[1:]:
                v = self.samples[c][sel]
                v = v[v >= 0]
                row[c] = float(v.mean()) if len(v) else None
            out.append(row)
        return out


class Monitor:
    """One sampler thread in libtsne.so; see the module docstring."""

    def __init__(self, handle):
        self._h = handle

    @classmethod
    def start(cls, period: float = 1.0, device: int = 0, csv: Optional[str] = None) -> "Monitor":
        err = ctypes.c_int(0)
        h = L.lib().tsne_mon_start(int(device), float(period),
                                   csv.encode() if csv else None, ctypes.byref(err))
        if not h:
            raise L.TsneError(err.value, "tsne_mon_start")
        return cls(h)

    def timestamp(self, name: str) -> None:
        L.check(L.lib().tsne_mon_mark(self._h, name.encode()), "tsne_mon_mark")

    def stop(self) -> None:
        L.check(L.lib().tsne_mon_stop(self._h), "tsne_mon_stop")

    def parse(self) -> Trace:
        lib = L.lib()
        n = int(lib.tsne_mon_count(self._h, 0))
        buf = np.zeros((max(n, 1), len(COLUMNS)), np.float64)
        if n:
            L.check(lib.tsne_mon_samples(self._h, buf.ctypes.data, n), "tsne_mon_samples")
        buf = buf[:n]
        events = []
        name = ctypes.create_string_buffer(256)
        t = ctypes.c_double(0)
        for i in range(int(lib.tsne_mon_count(self._h, 1))):
            L.check(lib.tsne_mon_event(self._h, i, ctypes.byref(t), name, 256), "tsne_mon_event")
            events.append((t.value, name.value.decode()))
        return Trace({c: buf[:, j].copy() for j, c in enumerate(COLUMNS)}, events)

    def close(self) -> None:
        if self._h:
            L.lib().tsne_mon_free(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.stop()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def parse_csv(path: str) -> Trace:
    """Read a trace file written by Monitor.start(csv=...)."""
    rows, events = [], []
    with open(path) as f:
        r = _csv.reader(f)
        next(r)
        for rec in r:
            if rec[0] == "sample":
                rows.append([float(x) for x in rec[1:8]])
            elif rec[0] == "event":
                events.append((float(rec[1]), rec[8]))
    a = np.asarray(rows, np.float64).reshape(-1, len(COLUMNS))
    return Trace({c: a[:, j].copy() for j, c in enumerate(COLUMNS)}, events)
